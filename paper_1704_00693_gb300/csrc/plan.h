// Tiling plans for a chain segment (host side).
#pragma once

#include <stdint.h>

#include <vector>

#include "internal.h"

namespace opstile {

// What the planner needs to know about one argument of a loop.
struct PArg {
  int kind;     // OPS_ARG_*
  int dat;      // dat handle (DAT args)
  bool reads;   // READ / RW / INC
  bool writes;  // WRITE / RW / INC
  int slo[3];   // stencil extent: min(0, most negative offset) per dimension
  int shi[3];   //                 max(0, most positive offset) per dimension
};

struct PLoop {
  int rng[6];   // [x0, x1) x [y0, y1) x [z0, z1)
  std::vector<PArg> args;
};

struct SkewedPlan {
  int ndim = 0;
  int tile[3] = {1, 1, 1};
  int ntiles[3] = {1, 1, 1};
  // ranges[d][2 * (t * nloops + l)] = start, [... + 1] = end of loop l in tile t along d
  std::vector<int> ranges[3];
  std::vector<Phase> phases;
  int nbarriers = 0;
  int skew[3] = {0, 0, 0};
  int64_t points = 0;
};

// Algorithm 1 (Sec. 4.B) with the readings documented in plan.cpp.
void build_skewed_ranges(const std::vector<PLoop>& loops, int ndats, int ndim, const int tile[3], SkewedPlan& out);
// Algorithm 2 order (tiles lexicographic, x fastest; loops in order inside a
// tile) with a grid barrier only before a phase that conflicts with a phase
// since the previous barrier.
void build_phases(const std::vector<PLoop>& loops, SkewedPlan& plan);

// Overlapped tiling (Sec. 4.D applied to one tile): grow each loop's part of
// the tile backwards by what later loops of the tile read.
struct OverlapTile {
  int owned[6];
  std::vector<int> box;      // 6 ints per loop (empty box: lo == hi)
  std::vector<int> foot;     // 6 ints per dat: live-in box (lo > hi if unread)
};
void build_overlap_tile(const std::vector<PLoop>& loops, int ndats, int ndim, const int owned[6], OverlapTile& out);

}  // namespace opstile
