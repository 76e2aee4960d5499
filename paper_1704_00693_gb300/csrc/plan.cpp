// Run-time dependency analysis of a queued chain segment.
//
// build_skewed_ranges is Algorithm 1 of Sec. 4.B.  The union of the loops'
// ranges is cut into tiles of `tile[d]` points per dimension; walking the
// loops from last to first, every tile of every loop gets a range that starts
// where the same loop's previous tile ended and ends far enough right to
//   - produce what later loops of the same tile read (read-after-write),
//   - not leave for the next tile a read or write of a value that a later
//     loop of this tile overwrites (write-after-read / write-after-write),
// or, with no dependency, at the tile boundary.  Readings of the printed
// algorithm: ranges are half-open; a tile's start is the previous tile's
// final end (prose step 3), so tiles are completed in increasing order per
// (loop, dimension); the default end of 0-based tile t is
// min(loop end, union start + (t+1) * tile); ends are clamped to at least the
// start and the last tile ends at the loop's end; m / p are the most negative
// / most positive stencil offsets, or 0; WAR/WAW looks at every dat argument
// (a written one has a point stencil, m = 0: the WAW case); empty ranges do
// not update the dependency records, which are never reset.  Dimensions are
// independent; tiles run lexicographically with x fastest.
#include "plan.h"

#include <algorithm>
#include <array>
#include <climits>
#include <map>

namespace opstile {

namespace {
constexpr int kNone = INT_MIN / 4;  // "no dependency recorded" / minus infinity
constexpr int kFar = INT_MAX / 4;
}  // namespace

void build_skewed_ranges(const std::vector<PLoop>& loops, int ndats, int ndim, const int tile[3], SkewedPlan& out) {
  const int L = (int)loops.size();
  out.ndim = ndim;
  for (int d = 0; d < 3; ++d) {
    out.tile[d] = 1;
    out.ntiles[d] = 1;
    out.ranges[d].clear();
    out.skew[d] = 0;
  }
  for (int d = 0; d < ndim; ++d) {
    int ustart = kFar, uend = -kFar;
    for (const PLoop& lp : loops) {
      ustart = std::min(ustart, lp.rng[2 * d]);
      uend = std::max(uend, lp.rng[2 * d + 1]);
    }
    const int ts = std::max(1, tile[d]);
    const int T = uend > ustart ? (uend - ustart - 1) / ts + 1 : 1;
    out.tile[d] = ts;
    out.ntiles[d] = T;
    std::vector<int>& R = out.ranges[d];
    R.assign((size_t)2 * T * L, 0);
    // dependency records per (tile, dat): end of reads / writes by later loops
    std::vector<int> rd_end((size_t)T * ndats, kNone), rd_start((size_t)T * ndats, kFar);
    std::vector<int> wr_end((size_t)T * ndats, kNone), wr_start((size_t)T * ndats, kFar);
    for (int l = L - 1; l >= 0; --l) {
      const PLoop& lp = loops[l];
      const int lo = lp.rng[2 * d], hi = lp.rng[2 * d + 1];
      for (int t = 0; t < T; ++t) {
        const int start = t == 0 ? lo : R[2 * ((t - 1) * L + l) + 1];
        int end = kNone;
        if (t == T - 1) {
          end = hi;
        } else {
          for (const PArg& a : lp.args) {  // read-after-write
            if (a.kind != OPS_ARG_DAT || !a.writes) continue;
            const int re = rd_end[(size_t)t * ndats + a.dat];
            if (re != kNone) end = std::min(hi, std::max(end, re));
          }
          for (const PArg& a : lp.args) {  // write-after-read / write-after-write
            if (a.kind != OPS_ARG_DAT) continue;
            const int we = wr_end[(size_t)t * ndats + a.dat];
            if (we != kNone) end = std::min(hi, std::max(end, we - a.slo[d]));
          }
        }
        if (end == kNone) end = std::min(hi, ustart + (t + 1) * ts);
        if (end < start) end = start;
        R[2 * (t * L + l)] = start;
        R[2 * (t * L + l) + 1] = end;
        if (end <= start) continue;
        for (const PArg& a : lp.args) {
          if (a.kind != OPS_ARG_DAT) continue;
          const size_t k = (size_t)t * ndats + a.dat;
          if (a.reads) {
            rd_end[k] = std::max(rd_end[k], end + a.shi[d]);
            rd_start[k] = std::min(rd_start[k], start + a.slo[d]);
          }
          if (a.writes) {
            wr_end[k] = std::max(wr_end[k], end);
            wr_start[k] = std::min(wr_start[k], start);
          }
        }
      }
    }
    // skew: spread of the loops' tile ends, largest over all but the last tile
    int sk = 0;
    for (int t = 0; t + 1 < T; ++t) {
      int mn = kFar, mx = -kFar;
      for (int l = 0; l < L; ++l) {
        const int s = R[2 * (t * L + l)], e = R[2 * (t * L + l) + 1];
        if (e <= s) continue;
        mn = std::min(mn, e);
        mx = std::max(mx, e);
      }
      if (mx >= mn) sk = std::max(sk, mx - mn);
    }
    out.skew[d] = sk;
  }
}

namespace {
bool boxes_meet(const int* a, const int* b) {
  for (int d = 0; d < 3; ++d)
    if (a[2 * d] >= b[2 * d + 1] || b[2 * d] >= a[2 * d + 1]) return false;
  return true;
}
void grow(const int* box, const PArg& a, int* out) {
  for (int d = 0; d < 3; ++d) {
    out[2 * d] = box[2 * d] + a.slo[d];
    out[2 * d + 1] = box[2 * d + 1] + a.shi[d];
  }
}
// Does phase q (loop lq over box bq) touch data that phase p (loop lp over
// box bp) writes, or write data that p touches?
bool conflict(const PLoop& lp, const int* bp, const PLoop& lq, const int* bq) {
  int gp[6], gq[6];
  for (const PArg& a : lp.args) {
    if (a.kind != OPS_ARG_DAT) continue;
    for (const PArg& b : lq.args) {
      if (b.kind != OPS_ARG_DAT || b.dat != a.dat) continue;
      if (!a.writes && !b.writes) continue;
      // region of the dat touched by each phase (reads widened by the stencil)
      if (a.reads) grow(bp, a, gp);
      else for (int i = 0; i < 6; ++i) gp[i] = bp[i];
      if (b.reads) grow(bq, b, gq);
      else for (int i = 0; i < 6; ++i) gq[i] = bq[i];
      if (boxes_meet(gp, gq)) return true;
    }
  }
  return false;
}
}  // namespace

void build_phases(const std::vector<PLoop>& loops, SkewedPlan& plan) {
  const int L = (int)loops.size();
  plan.phases.clear();
  plan.phase_tile.clear();
  plan.nbarriers = 0;
  plan.points = 0;
  std::vector<int> epoch;  // phases since the last barrier
  for (int tz = 0; tz < plan.ntiles[2]; ++tz)
    for (int ty = 0; ty < plan.ntiles[1]; ++ty)
      for (int tx = 0; tx < plan.ntiles[0]; ++tx)
        for (int l = 0; l < L; ++l) {
          Phase P;
          P.loop = l;
          P.barrier = 0;
          const int t[3] = {tx, ty, tz};
          bool empty = false;
          for (int d = 0; d < 3; ++d) {
            if (d < plan.ndim) {
              const std::vector<int>& R = plan.ranges[d];
              P.box[2 * d] = R[2 * (t[d] * L + l)];
              P.box[2 * d + 1] = R[2 * (t[d] * L + l) + 1];
            } else {
              P.box[2 * d] = loops[l].rng[2 * d];
              P.box[2 * d + 1] = loops[l].rng[2 * d + 1];
            }
            if (P.box[2 * d + 1] <= P.box[2 * d]) empty = true;
          }
          if (empty) continue;
          bool need = false;
          for (int e : epoch) {
            const Phase& Q = plan.phases[e];
            if (conflict(loops[Q.loop], Q.box, loops[l], P.box)) {
              need = true;
              break;
            }
          }
          if (need) {
            P.barrier = 1;
            ++plan.nbarriers;
            epoch.clear();
          }
          epoch.push_back((int)plan.phases.size());
          int64_t n = 1;
          for (int d = 0; d < 3; ++d) n *= (int64_t)(P.box[2 * d + 1] - P.box[2 * d]);
          plan.points += n;
          plan.phases.push_back(P);
          plan.phase_tile.push_back((tz * plan.ntiles[1] + ty) * plan.ntiles[0] + tx);
        }
}

namespace {
// enumeration units of one box, as the kernels count them (see run_units)
int64_t box_units(const int* b, int P, int NT) {
  const int64_t nx = b[1] - b[0], ny = b[3] - b[2], nz = b[5] - b[4];
  if (nx <= 0 || ny <= 0 || nz <= 0) return 0;
  if (nx >= 128) return ((nx + NT - 1) / NT) * ((ny + P - 1) / P) * nz;
  const int64_t g = (int64_t)NT * P;
  return (nx * ny * nz + g - 1) / g;
}
}  // namespace

void build_wavefront(const std::vector<PLoop>& loops, int ndats, const SkewedPlan& plan, int axis, int P, int NT,
                     int per_unit, int slope, WavePlan& out) {
  const int nph = (int)plan.phases.size();
  out.axis = axis;
  out.dep_off.assign(nph + 1, 0);
  out.deps.clear();
  out.nchunk.assign(nph, 0);
  out.ustart.assign(nph, 0);
  out.nunits = 0;
  // the index range along the axis that any phase touches
  int lo = kFar, hi = -kFar;
  for (const Phase& ph : plan.phases)
    for (const PArg& a : loops[ph.loop].args) {
      if (a.kind != OPS_ARG_DAT) continue;
      lo = std::min(lo, ph.box[2 * axis] + a.slo[axis]);
      hi = std::max(hi, ph.box[2 * axis + 1] + a.shi[axis]);
    }
  const int n = hi > lo ? hi - lo : 0;
  // acc[dat * n + i]: phases so far that touch index i of the dat along the axis
  std::vector<std::vector<int>> acc((size_t)ndats * n);
  std::vector<int> seen(nph, -1), cand;
  for (int q = 0; q < nph; ++q) {
    const Phase& Q = plan.phases[q];
    const PLoop& lq = loops[Q.loop];
    cand.clear();
    for (const PArg& a : lq.args) {
      if (a.kind != OPS_ARG_DAT) continue;
      const int r0 = Q.box[2 * axis] + (a.reads ? a.slo[axis] : 0) - lo;
      const int r1 = Q.box[2 * axis + 1] + (a.reads ? a.shi[axis] : 0) - lo;
      for (int i = r0; i < r1; ++i)
        for (int p : acc[(size_t)a.dat * n + i])
          if (seen[p] != q) {
            seen[p] = q;
            cand.push_back(p);
          }
    }
    std::sort(cand.begin(), cand.end());
    for (int p : cand)
      if (conflict(loops[plan.phases[p].loop], plan.phases[p].box, lq, Q.box)) out.deps.push_back(p);
    out.dep_off[q + 1] = (int)out.deps.size();
    for (const PArg& a : lq.args) {
      if (a.kind != OPS_ARG_DAT) continue;
      const int r0 = Q.box[2 * axis] + (a.reads ? a.slo[axis] : 0) - lo;
      const int r1 = Q.box[2 * axis + 1] + (a.reads ? a.shi[axis] : 0) - lo;
      for (int i = r0; i < r1; ++i) {
        std::vector<int>& v = acc[(size_t)a.dat * n + i];
        if (v.empty() || v.back() != q) v.push_back(q);
      }
    }
    const int64_t u = box_units(Q.box, P, NT);
    out.nchunk[q] = (int)std::max<int64_t>(1, (u + per_unit - 1) / std::max(1, per_unit));
  }
  // levels, then the units by (level + slope * tile, tile, plan order)
  out.level.assign(nph, 0);
  out.nlevels = 0;
  for (int q = 0; q < nph; ++q) {
    for (int k = out.dep_off[q]; k < out.dep_off[q + 1]; ++k)
      out.level[q] = std::max(out.level[q], out.level[out.deps[k]] + 1);
    out.nlevels = std::max(out.nlevels, out.level[q] + 1);
  }
  std::vector<std::array<int64_t, 3>> keyed(nph);
  for (int q = 0; q < nph; ++q) {
    const int64_t t = plan.phase_tile[q];
    keyed[q] = {out.level[q] + (int64_t)std::max(0, slope) * t, t, q};
  }
  std::sort(keyed.begin(), keyed.end());
  std::vector<int> order(nph);
  for (int q = 0; q < nph; ++q) order[q] = (int)keyed[q][2];
  out.uphase.clear();
  for (int q : order) {
    out.ustart[q] = (int)out.uphase.size();
    out.uphase.insert(out.uphase.end(), out.nchunk[q], q);
  }
  out.nunits = (int64_t)out.uphase.size();
}

// Overlapped tile (Sec. 4.D, read dependencies only): the last loops keep the
// tile's owned box; an earlier loop that writes a dat read by later loops of
// the tile widens its box to everything those reads touch (clipped to its own
// range); what is read but not produced inside the tile is the live-in
// footprint.
void build_overlap_tile(const std::vector<PLoop>& loops, int ndats, int ndim, const int owned[6], OverlapTile& out) {
  const int L = (int)loops.size();
  for (int i = 0; i < 6; ++i) out.owned[i] = owned[i];
  out.box.assign((size_t)6 * L, 0);
  std::vector<int> rb((size_t)6 * ndats);
  for (int k = 0; k < ndats; ++k)
    for (int d = 0; d < 3; ++d) {
      rb[6 * k + 2 * d] = kFar;
      rb[6 * k + 2 * d + 1] = -kFar;
    }
  for (int l = L - 1; l >= 0; --l) {
    const PLoop& lp = loops[l];
    int box[6];
    bool empty = false;
    for (int d = 0; d < 3; ++d) {
      const int lo = lp.rng[2 * d], hi = lp.rng[2 * d + 1];
      int blo, bhi;
      if (d < ndim) {
        blo = std::max(lo, owned[2 * d]);
        bhi = std::min(hi, owned[2 * d + 1]);
        if (bhi <= blo) {
          blo = kFar;
          bhi = -kFar;
        }
        for (const PArg& a : lp.args) {
          if (a.kind != OPS_ARG_DAT || !a.writes) continue;
          const int rlo = rb[6 * a.dat + 2 * d], rhi = rb[6 * a.dat + 2 * d + 1];
          if (rhi <= rlo) continue;
          blo = std::min(blo, std::max(lo, rlo));
          bhi = std::max(bhi, std::min(hi, rhi));
        }
      } else {
        blo = lo;
        bhi = hi;
      }
      box[2 * d] = blo;
      box[2 * d + 1] = bhi;
      if (bhi <= blo) empty = true;
    }
    int* ob = &out.box[(size_t)6 * l];
    if (empty) {
      for (int i = 0; i < 6; ++i) ob[i] = 0;
      continue;
    }
    for (int i = 0; i < 6; ++i) ob[i] = box[i];
    for (const PArg& a : lp.args) {
      if (a.kind != OPS_ARG_DAT || !a.reads) continue;
      for (int d = 0; d < 3; ++d) {
        rb[6 * a.dat + 2 * d] = std::min(rb[6 * a.dat + 2 * d], box[2 * d] + a.slo[d]);
        rb[6 * a.dat + 2 * d + 1] = std::max(rb[6 * a.dat + 2 * d + 1], box[2 * d + 1] + a.shi[d]);
      }
    }
  }
  out.foot = rb;
}

// ---------------------------------------------------------------------------
// Tile wavefront (see plan.h)
// ---------------------------------------------------------------------------
namespace {
// One conflicting pair of accesses: argument `a` of loop `l` (the later loop)
// and argument `b` of loop `lp` < l on the same dat, at least one writing it.
struct APair {
  int l, a, lp, b;
};
// The interval of dimension d an argument touches in tile t (reads widened
// by the stencil); empty (lo >= hi) when the loop's range there is empty.
inline void touched(const SkewedPlan& P, int L, int d, int t, int l, const PArg& a, int* lo, int* hi) {
  const std::vector<int>& R = P.ranges[d];
  const int s = R[2 * (t * L + l)], e = R[2 * (t * L + l) + 1];
  if (e <= s) {
    *lo = 0;
    *hi = 0;
    return;
  }
  *lo = s + (a.reads ? a.slo[d] : 0);
  *hi = e + (a.reads ? a.shi[d] : 0);
}
inline bool meet(int alo, int ahi, int blo, int bhi) { return alo < ahi && blo < bhi && alo < bhi && blo < ahi; }
}  // namespace

bool build_tile_wave(const std::vector<PLoop>& loops, const SkewedPlan& P, TileWavePlan& out, std::string* why,
                     int max_group, int band) {
  const int L = (int)loops.size();
  const int nd = P.ndim;
  out = TileWavePlan();
  out.ndim = nd;
  out.nloops = L;
  if (L >= 65535) {
    *why = "too many loops in one segment";
    return false;
  }
  // conflicting argument pairs (later loop first)
  std::vector<APair> pairs;
  for (int l = 0; l < L; ++l)
    for (int a = 0; a < (int)loops[l].args.size(); ++a) {
      const PArg& A = loops[l].args[a];
      if (A.kind != OPS_ARG_DAT) continue;
      for (int lp = 0; lp < l; ++lp)
        for (int b = 0; b < (int)loops[lp].args.size(); ++b) {
          const PArg& B = loops[lp].args[b];
          if (B.kind != OPS_ARG_DAT || B.dat != A.dat || !(A.writes || B.writes)) continue;
          pairs.push_back(APair{l, a, lp, b});
        }
    }
  out.pairs = (int64_t)pairs.size();
  // Per dimension, for every pair and tile t: the later access in tile t
  // must not touch what the earlier one touches in tiles after t (the order
  // of Algorithm 2 would then run them the wrong way round), nor what it
  // touches two or more tiles back (no wait covers that distance).  The
  // tiles of one loop partition its range in order, so the union of its
  // touched intervals over a run of consecutive tiles is one interval.
  for (int d = 0; d < nd; ++d) {
    const int T = P.ntiles[d];
    const std::vector<int>& R = P.ranges[d];
    for (const APair& q : pairs) {
      const PArg& A = loops[q.l].args[q.a];
      const PArg& B = loops[q.lp].args[q.b];
      const int blo0 = R[2 * (0 * L + q.lp)], bhi_all = R[2 * ((T - 1) * L + q.lp) + 1];
      const int bs = B.reads ? B.slo[d] : 0, be = B.reads ? B.shi[d] : 0;
      for (int t = 0; t < T; ++t) {
        int alo, ahi;
        touched(P, L, d, t, q.l, A, &alo, &ahi);
        if (alo >= ahi) continue;
        if (t + 1 < T) {
          const int e = R[2 * (t * L + q.lp) + 1];  // the earlier loop's later tiles: [e, end)
          if (e < bhi_all && meet(alo, ahi, e + bs, bhi_all + be)) {
            *why = "an access of a later loop falls in an earlier tile than a conflicting access of an earlier loop";
            return false;
          }
        }
        if (t >= 2) {
          const int e2 = R[2 * ((t - 2) * L + q.lp) + 1];  // the earlier loop's tiles up to t - 2: [start, e2)
          if (e2 > blo0 && meet(alo, ahi, blo0 + bs, e2 + be)) {
            *why = "the skew reaches two tiles back: tiles are too small for this chain";
            out.bad_dim = d;
            return false;
          }
        }
        // the same two checks with the roles of the tiles exchanged: the
        // earlier loop's access in tile t against the later loop's in tiles
        // two or more back (a conflict the other way round)
        int blo, bhi;
        touched(P, L, d, t, q.lp, B, &blo, &bhi);
        if (blo < bhi && t >= 2) {
          const int e2 = R[2 * ((t - 2) * L + q.l) + 1];
          const int a0 = R[2 * (0 * L + q.l)];
          const int as = A.reads ? A.slo[d] : 0, ae = A.reads ? A.shi[d] : 0;
          if (e2 > a0 && meet(blo, bhi, a0 + as, e2 + ae)) {
            *why = "an access of an earlier loop falls two or more tiles after a conflicting access of a later loop";
            out.bad_dim = d;
            return false;
          }
        }
      }
    }
  }
  // predecessor directions
  out.ndirs = (1 << nd) - 1;
  for (int m = 1; m <= out.ndirs; ++m)
    for (int d = 0; d < 3; ++d) out.dirs[m - 1][d] = d < nd ? (m >> d) & 1 : 0;
  // classes per dimension: tiles whose own ranges and the previous tile's,
  // relative to the tile's default start, are the same
  int Tn[3] = {1, 1, 1};
  std::vector<int> rep[3];
  for (int d = 0; d < 3; ++d) {
    Tn[d] = d < nd ? P.ntiles[d] : 1;
    out.cls[d].assign(Tn[d], 0);
    if (d >= nd) {
      rep[d].push_back(0);
      continue;
    }
    std::map<std::vector<int>, int> ids;
    const std::vector<int>& R = P.ranges[d];
    for (int t = 0; t < Tn[d]; ++t) {
      std::vector<int> key;
      key.reserve(4 * L + 1);
      const int base = t * P.tile[d];
      key.push_back(t == 0 ? 1 : 0);
      for (int u = t - 1; u <= t; ++u)
        for (int l = 0; l < L; ++l) {
          const int s0 = u < 0 ? 0 : R[2 * (u * L + l)], e0 = u < 0 ? 0 : R[2 * (u * L + l) + 1];
          if (e0 <= s0) {  // no tile, or an empty range: where it sits does not matter
            key.push_back(INT_MIN);
            key.push_back(u < 0 ? INT_MIN : INT_MIN + 1);
          } else {
            key.push_back(s0 - base);
            key.push_back(e0 - base);
          }
        }
      auto it = ids.find(key);
      if (it == ids.end()) {
        const int id = (int)ids.size();
        ids.emplace(std::move(key), id);
        rep[d].push_back(t);
        out.cls[d][t] = id;
      } else {
        out.cls[d][t] = it->second;
      }
    }
    out.ncls[d] = (int)ids.size();
  }
  // per dimension, class and step back (0 or 1): which pairs meet
  const size_t np = pairs.size();
  std::vector<std::vector<char>> meets[3];
  for (int d = 0; d < 3; ++d) {
    meets[d].assign((size_t)out.ncls[d] * 2, std::vector<char>(np, 0));
    for (int c = 0; c < out.ncls[d]; ++c) {
      const int t = rep[d][c];
      for (int s = 0; s < 2; ++s) {
        std::vector<char>& m = meets[d][(size_t)c * 2 + s];
        if (d >= nd) {
          std::fill(m.begin(), m.end(), s == 0 ? 1 : 0);
          continue;
        }
        if (t - s < 0) continue;
        for (size_t k = 0; k < np; ++k) {
          const APair& q = pairs[k];
          int alo, ahi, blo, bhi;
          touched(P, L, d, t, q.l, loops[q.l].args[q.a], &alo, &ahi);
          touched(P, L, d, t - s, q.lp, loops[q.lp].args[q.b], &blo, &bhi);
          m[k] = meet(alo, ahi, blo, bhi) ? 1 : 0;
        }
      }
    }
  }
  const int ncl = out.ncls[0] * out.ncls[1] * out.ncls[2];
  out.need.assign((size_t)ncl * out.ndirs * L, 0);
  for (int cz = 0; cz < out.ncls[2]; ++cz)
    for (int cy = 0; cy < out.ncls[1]; ++cy)
      for (int cx = 0; cx < out.ncls[0]; ++cx) {
        const int cc[3] = {cx, cy, cz};
        const int cl = (cz * out.ncls[1] + cy) * out.ncls[0] + cx;
        for (int di = 0; di < out.ndirs; ++di) {
          const char* m[3];
          for (int d = 0; d < 3; ++d) m[d] = meets[d][(size_t)cc[d] * 2 + out.dirs[di][d]].data();
          uint16_t* nv = &out.need[((size_t)cl * out.ndirs + di) * L];
          for (size_t k = 0; k < np; ++k)
            if (m[0][k] && m[1][k] && m[2][k]) {
              const APair& q = pairs[k];
              nv[q.l] = (uint16_t)std::max<int>(nv[q.l], q.lp + 1);
            }
        }
      }
  // steps: consecutive loops that share no dat with a write among them
  out.groups.clear();
  {
    auto clash = [&](const PLoop& a, const PLoop& b) {
      for (const PArg& x : a.args) {
        if (x.kind != OPS_ARG_DAT) continue;
        for (const PArg& y : b.args)
          if (y.kind == OPS_ARG_DAT && y.dat == x.dat && (x.writes || y.writes)) return true;
      }
      return false;
    };
    int g0 = 0;
    out.groups.push_back(0);
    for (int l = 1; l < L; ++l) {
      bool cut = l - g0 >= std::max(1, max_group);
      for (int m = g0; m < l && !cut; ++m) cut = clash(loops[m], loops[l]);
      if (cut) {
        out.groups.push_back(l);
        g0 = l;
      }
    }
    out.groups.push_back(L);
  }
  // tickets: strip by strip of `band` tiles along x, and inside a strip by
  // coordinate sum, then z, y, x
  out.order.clear();
  out.order.reserve((size_t)Tn[0] * Tn[1] * Tn[2]);
  const int bw = band > 0 ? std::min(band, Tn[0]) : Tn[0];
  for (int b0 = 0; b0 < Tn[0]; b0 += bw) {
    const int w = std::min(bw, Tn[0] - b0);
    for (int s = 0; s <= w + Tn[1] + Tn[2] - 3; ++s)
      for (int tz = 0; tz < Tn[2]; ++tz)
        for (int ty = 0; ty < Tn[1]; ++ty) {
          const int tl = s - tz - ty;
          if (tl < 0 || tl >= w) continue;
          out.order.push_back((tz * Tn[1] + ty) * Tn[0] + b0 + tl);
        }
  }
  return true;
}

}  // namespace opstile
