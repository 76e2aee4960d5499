// Tiling plans for a chain segment (host side).
#pragma once

#include <stdint.h>

#include <string>
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
  std::vector<int> phase_tile;  // linear tile index (x fastest) of each phase
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

// Wavefront execution of a skewed plan: the phases of plan.phases, each
// waiting only for the earlier phases it conflicts with.  deps[dep_off[q] ..
// dep_off[q + 1]) are the phases before q in plan order that touch a dat q
// touches, where at least one of the two writes it and the touched regions
// (reads widened by the stencil) intersect.  Candidates are found through a
// per-(dat, index) access list along dimension `axis` and then checked
// exactly, so the list is complete (every conflicting earlier phase) and
// holds nothing else.  Phase q is split into nchunk[q] work units of at most
// `per_unit` of the kernel's enumeration units (P rows of NT points, or
// flattened groups of NT x P points for boxes narrower than 128).
// Work units are numbered (the order a kernel hands them out) by the key
// level + slope * tile, then tile, then plan order, where the level of a
// phase is the longest dependency path that ends at it and tile is its
// linear tile index.  Every dependency has a smaller key (its level is
// smaller and its tile no later), so this is a topological order for any
// slope >= 0.  Slope 0 runs level by level over all tiles (loop by loop, as
// untiled); a slope >= the number of levels is Algorithm 2's tile-by-tile
// order; in between, about nlevels / slope tiles are in flight at once, each
// at a different level -- a wavefront over the tiles.
struct WavePlan {
  int axis = 0;
  std::vector<int> dep_off, deps;
  std::vector<int> nchunk, ustart;  // per phase
  std::vector<int> level;           // per phase
  int nlevels = 0;
  std::vector<int> uphase;          // per work unit: its phase
  int64_t nunits = 0;
};
void build_wavefront(const std::vector<PLoop>& loops, int ndats, const SkewedPlan& plan, int axis, int P, int NT,
                     int per_unit, int slope, WavePlan& out);

// Overlapped tiling (Sec. 4.D applied to one tile): grow each loop's part of
// the tile backwards by what later loops of the tile read.
struct OverlapTile {
  int owned[6];
  std::vector<int> box;      // 6 ints per loop (empty box: lo == hi)
  std::vector<int> foot;     // 6 ints per dat: live-in box (lo > hi if unread)
};
void build_overlap_tile(const std::vector<PLoop>& loops, int ndats, int ndim, const int owned[6], OverlapTile& out);

// Tile wavefront (OPS_MODE_TILEWAVE): the tiles of Algorithm 1 cut in every
// dimension; one CTA runs all the loops of a tile in order (the inner loop
// of Algorithm 2), and tiles run concurrently.  Algorithm 1 orders every
// conflicting pair of accesses the same way in each dimension on its own (an
// earlier loop's access never falls in a later tile than a later loop's
// access to the same data), so program order only needs tile T's loop l to
// run after the phases of the tiles one step back in any subset of
// dimensions (T - delta, delta in {0,1}^ndim, delta != 0) that conflict with
// it: those are earlier loops l' < l.  need[(class, delta, l)] = 1 + the
// latest such l' (0: none), a count of completed loops of tile T - delta.
// build_tile_wave checks both premises on the plan, per dimension: that the
// order holds for every pair of accesses (monotonicity) and that no access
// reaches data an access two or more tiles back touches.  Tiles whose
// per-dimension neighbourhoods have identical relative ranges share a class.
// Tickets hand out tiles strip by strip (strips of `band` tiles along x; 0:
// one strip), and inside a strip by the sum of their tile coordinates
// (then z, y, x): every predecessor is in the same or an earlier strip and
// has a smaller sum, so the earliest unfinished tile never waits on a later
// one.  Narrow strips keep the tiles in flight together in one compact
// region, whose data (the tiles' and their skew halos, shared between
// neighbours) then fits L2.
struct TileWavePlan {
  int ndim = 0, ndirs = 0;
  int dirs[7][3] = {};
  int ncls[3] = {1, 1, 1};
  std::vector<int> cls[3];        // per dimension: class of each tile index
  std::vector<uint16_t> need;     // [(class * ndirs + dir) * nloops + l]
  std::vector<int> order;         // ticket -> linear tile index (x fastest)
  int nloops = 0;
  int64_t pairs = 0;              // conflicting argument pairs examined
  int bad_dim = -1;               // on failure: the dimension whose tiles are too small
  // Steps of a tile: runs of consecutive loops, none of which shares a dat
  // with an earlier loop of its run where either writes it, so a run's
  // loops need no barrier between them; groups[g] .. groups[g + 1] are the
  // loops of step g (groups.back() = nloops)
  std::vector<int> groups;
};
// max_group caps the loops of one step (1: a step per loop)
bool build_tile_wave(const std::vector<PLoop>& loops, const SkewedPlan& plan, TileWavePlan& out, std::string* why,
                     int max_group = 8, int band = 0);

}  // namespace opstile
