// Host runtime of opstile: context, declarations, delayed-execution queue
// (Sec. 4.A), flush into segments, plan cache (Sec. 4.B: plans are re-used
// when the same loop sequence comes back), tile-size choice (Sec. 4.C) and
// kernel launches.  Implements the C ABI of include/opstile.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <numeric>
#include <set>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"
#include "jit.h"
#include "opstile.h"
#include "plan.h"

using namespace opstile;

namespace {

struct Block {
  int dims;
  std::string name;
};

struct Dat {
  int block;
  int size[3], dm[3], dp[3], ext[3];
  double* alloc = nullptr;  // owned allocation (nullptr if borrowed)
  double* ptr0 = nullptr;   // grid point (0,0,0)
  double* alt = nullptr;    // second buffer for overlapped tiles (allocated on first use)
  double* alt_ptr0 = nullptr;
  int64_t pitch = 0, plane = 0;
  size_t bytes = 0;
  std::string name;
};

struct Stencil {
  int dims;
  std::vector<int> off;  // 3 per point
  int lo[3], hi[3];
  std::string name;
};

struct QLoop {
  int block, dims;
  int rng[6];
  std::vector<ops_arg> args;
  std::vector<int32_t> code;
  std::vector<double> K;
  std::string name;
};

struct CachedPlan {
  std::vector<int> key;
  SkewedPlan plan;
  Phase* d_phases = nullptr;
  // wavefront form: phase table, dependency lists and the ticket order on
  // the device (one allocation), per-phase completion counters + ticket
  WavePlan wave;
  int nlevels = 0;
  void* d_wave = nullptr;
  size_t wave_bytes = 0;
  int* d_wdone = nullptr;
  // tile-wavefront form: ranges | ticket order | tile classes | need table
  // (one allocation), per-tile progress + ticket, per-tile reduction partials
  TileWavePlan tw;
  void* d_tw = nullptr;
  size_t tw_bytes = 0;
  size_t tw_order = 0, tw_cls = 0, tw_need = 0, tw_grp = 0, tw_pf = 0;  // byte offsets inside d_tw
  int tw_roff[3] = {0, 0, 0}, tw_coff[3] = {0, 0, 0};
  int* d_twprog = nullptr;
  int tw_ntiles = 0;
  int tw_phases = 0;  // non-empty (tile, loop) pieces
  int tw_steps = 0;   // CTA-wide steps (block barriers between loop groups) over all tiles
  DD* d_twpart = nullptr;
  int tw_rows = 0;
};

// An overlapped-tile plan of one segment (Sec. 4.D per CTA tile).
struct OverlapPlan {
  int tile[3];
  int ntiles = 0, nloops = 0, ndats = 0;
  std::vector<int> seg_dats;                // context dat ids, in local order
  std::vector<int> written, spitch, splane, smem_off;
  int area_bytes = 0;
  int64_t redundant = 0;
  int* d_tab = nullptr;                     // own | boxes | foot
  size_t tab_ints = 0;
  int own_off = 0, box_off = 0, foot_off = 0;
  int first_loop = 0;
};

// Autotuning state of one segment signature.
struct TuneRec {
  std::vector<std::array<int, 5>> cand;  // (mode, tile x, tile y, tile z, loops per sub-segment; 0 = all)
  std::vector<double> ms;                // best device time of each candidate (-1: not yet run)
  std::vector<int> runs;                 // samples taken of each candidate
  int pending = -1;                      // candidate whose events are outstanding
  int best = -1;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
};

}  // namespace

struct ops_ctx_s {
  ops_config cfg;
  int es = 8;  // bytes per dat element: 8 (FP64) or 4 (FP32)
  bool host_only = false;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int num_sms = 0;
  int64_t l2_size = 0;
  std::vector<Block> blocks;
  std::vector<Dat> dats;
  std::vector<Stencil> stencils;
  std::vector<int> red_ops;
  std::vector<QLoop> queue;
  // device state
  double* d_scal = nullptr;
  int scal_cap = 0;
  DD* d_part = nullptr;
  int part_rows_cap = 0;
  int part_stride = 0;
  FoldRow* d_rows = nullptr;
  int rows_cap = 0;
  int* d_err = nullptr;
  unsigned* d_bar = nullptr;
  DLoop* d_loops = nullptr;
  int loops_cap = 0;
  // host copy of the descriptors d_loops holds (in stream order), so a flush
  // uploads only the descriptors that changed since the last one
  // dev_ok[i]: d_loops[i] holds the descriptor cache's entry i (stream order)
  std::vector<char> dev_ok;
  DLoop* mirror_of = nullptr;
  // descriptors of the last flush, kept with the loops they were filled
  // from: a flush that queues the same loop at the same position (same
  // block, range, arguments, body, partial row; constants may differ) at the
  // same buffer generation reuses the descriptor instead of refilling it
  std::vector<DLoop> hl_cache;
  std::vector<QLoop> hl_src;
  std::vector<char> hl_ok;
  uint64_t hl_gen = 0;
  uint64_t swap_gen = 0;  // bumped whenever overlapped tiles move dats to their other buffer
  int skewed_grid = 0;
  std::map<std::vector<int>, std::unique_ptr<CachedPlan>> plans;
  std::map<std::vector<int>, TuneRec> tune;
  std::map<std::vector<int>, std::unique_ptr<OverlapPlan>> oplans;
  DLoop* d_oloops = nullptr;  // overlapped segments: descriptors in shared-memory layout
  int oloops_cap = 0;
  OvDat* d_ovdat = nullptr;
  int ovdat_cap = 0;
  // compiled loop bodies per segment (by signature and IR); nullptr: interpret
  std::map<std::vector<int>, JitSegment*> jit;
  std::map<std::vector<int>, JitWave*> jitw;  // wavefront kernels, same keys
  std::map<std::vector<int>, JitTile*> jitt;  // tile-wavefront kernels, same keys
  std::map<std::vector<int>, JitSkew*> jitk;  // persistent skewed kernels, same keys
  std::string jit_why;
  int64_t allocated = 0;
  std::string err;
  ops_flush_stats stats;
  // timing=1: event pairs around the chain kernels of the last flush
  std::vector<cudaEvent_t> ev_pool;
  int ev_used = 0;
  // batches this context leads (ops_execute_batch): the batch kernel's
  // tables, and the autotuning state per segment signature and batch size
  void* d_batch = nullptr;
  size_t batch_cap = 0;
  std::map<std::vector<int>, TuneRec> btune;
  // recorded on this context's stream when another stream must wait for it
  cudaEvent_t ev_join = nullptr;
  // pinned staging of the flush's host-to-device copies (descriptors, fold
  // rows), so they queue without a synchronous pageable copy: two buffers
  // used by alternate flushes, each reused once the copies of the flush
  // before last have completed (ev_stage)
  char* h_stage[2] = {nullptr, nullptr};
  size_t stage_cap[2] = {0, 0};
  cudaEvent_t ev_stage[2] = {nullptr, nullptr};
  bool stage_live[2] = {false, false};
  int stage_slot = 0;
  size_t stage_used = 0;
  std::vector<FoldRow> rows_mirror;  // fold rows d_rows holds
  // pinned landing slots of ops_reduction_result: the value, the error word
  struct { double value; int err; int pad; }* h_small = nullptr;
};

namespace {

// red_ops entry of a handle made by ops_decl_scalar: a value SCALAR
// arguments read, which no loop reduces into
constexpr int kScalarHandle = 100;

int fail(ops_ctx c, int code, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return code;
}

int cuda_fail(ops_ctx c, cudaError_t e, const char* what) {
  return fail(c, OPS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CUDA_TRY(c, expr)                              \
  do {                                                 \
    cudaError_t e_ = (expr);                           \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, #expr); \
  } while (0)

// Address `n` elements of `es` bytes from p (dat pointers are kept as double*
// whatever the element type).
inline double* elem_at(double* p, int64_t n, int es) { return (double*)((char*)p + (int64_t)es * n); }

int dev_alloc(ops_ctx c, void** p, size_t bytes) {
  if (c->cfg.hbm_budget > 0 && c->allocated + (int64_t)bytes > c->cfg.hbm_budget)
    return fail(c, OPS_ERR_NOMEM, "allocation of %zu bytes exceeds the HBM budget (%lld of %lld used)", bytes,
                (long long)c->allocated, (long long)c->cfg.hbm_budget);
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, OPS_ERR_NOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
  }
  c->allocated += (int64_t)bytes;
  return OPS_OK;
}

void dev_free(ops_ctx c, void* p, size_t bytes) {
  if (p) {
    cudaFree(p);
    c->allocated -= (int64_t)bytes;
  }
}

// Grow a device array to hold at least n elements (contents discarded).
template <class T>
int ensure(ops_ctx c, T** p, int* cap, int n) {
  if (n <= *cap) return OPS_OK;
  int nc = std::max(n, *cap * 2);
  nc = std::max(nc, 16);
  if (*p) {
    cudaStreamSynchronize(c->stream);
    dev_free(c, *p, sizeof(T) * (size_t)*cap);
    *p = nullptr;
    *cap = 0;
  }
  int rc = dev_alloc(c, (void**)p, sizeof(T) * (size_t)nc);
  if (rc) return rc;
  *cap = nc;
  return OPS_OK;
}

bool valid_reg(int r) { return r >= 0 && r < kNReg; }

double red_identity(int op) {
  return op == OPS_RED_SUM ? 0.0 : (op == OPS_RED_MIN ? __builtin_inf() : -__builtin_inf());
}

LaunchEnv make_env(ops_ctx c) {
  LaunchEnv env;
  env.stream = c->stream;
  env.num_sms = c->num_sms;
  env.scal = c->d_scal;
  env.part = c->d_part;
  env.part_stride = c->part_stride;
  env.rows = c->d_rows;
  env.err = c->d_err;
  env.bar = c->d_bar;
  env.check = c->cfg.check;
  env.timeout_ns = (long long)(c->cfg.timeout_ms > 0 ? c->cfg.timeout_ms : 2000) * 1000000ll;
  env.skip_block = c->cfg.test_skip_barrier_block;
  return env;
}

// ---------------------------------------------------------------------------
// validation of one queued loop
// ---------------------------------------------------------------------------
int validate_loop(ops_ctx c, const QLoop& q) {
  const int nargs = (int)q.args.size();
  const int nK = (int)q.K.size();
  int nreds = 0;
  std::vector<int> seen_dat, seen_red;
  for (int i = 0; i < nargs; ++i) {
    const ops_arg& a = q.args[i];
    if (a.kind == OPS_ARG_DAT) {
      if (a.handle < 0 || a.handle >= (int)c->dats.size())
        return fail(c, OPS_ERR_INVALID_ARG, "loop '%s' arg %d: bad dat handle %d", q.name.c_str(), i, a.handle);
      if (c->dats[a.handle].block != q.block)
        return fail(c, OPS_ERR_INVALID_ARG, "loop '%s' arg %d: dat on another block", q.name.c_str(), i);
      if (a.stencil < 0 || a.stencil >= (int)c->stencils.size())
        return fail(c, OPS_ERR_INVALID_ARG, "loop '%s' arg %d: bad stencil %d", q.name.c_str(), i, a.stencil);
      if (a.access < OPS_READ || a.access > OPS_INC)
        return fail(c, OPS_ERR_INVALID_ARG, "loop '%s' arg %d: bad access mode", q.name.c_str(), i);
      if (std::find(seen_dat.begin(), seen_dat.end(), a.handle) != seen_dat.end())
        return fail(c, OPS_ERR_INVALID_ARG, "loop '%s': dat %d appears twice", q.name.c_str(), a.handle);
      seen_dat.push_back(a.handle);
      const Stencil& s = c->stencils[a.stencil];
      const int npts = (int)s.off.size() / 3;
      if (a.access != OPS_READ) {
        if (npts != 1 || s.off[0] || s.off[1] || s.off[2])
          return fail(c, OPS_ERR_INVALID_ARG, "loop '%s' arg %d: a written dat must use the point stencil {0}",
                      q.name.c_str(), i);
      }
      const Dat& D = c->dats[a.handle];
      for (int d = 0; d < q.dims; ++d) {
        if (q.rng[2 * d + 1] <= q.rng[2 * d]) continue;
        const int lo = q.rng[2 * d] + s.lo[d], hi = q.rng[2 * d + 1] - 1 + s.hi[d];
        if (lo < -D.dm[d] || hi >= D.size[d] + D.dp[d])
          return fail(c, OPS_ERR_BOUNDS,
                      "loop '%s' arg %d (dat '%s'): access [%d, %d] in dim %d outside [%d, %d)", q.name.c_str(), i,
                      D.name.c_str(), lo, hi, d, -D.dm[d], D.size[d] + D.dp[d]);
      }
    } else if (a.kind == OPS_ARG_SCALAR || a.kind == OPS_ARG_RED) {
      if (a.handle < 0 || a.handle >= (int)c->red_ops.size())
        return fail(c, OPS_ERR_INVALID_ARG, "loop '%s' arg %d: bad reduction handle %d", q.name.c_str(), i, a.handle);
      if (a.kind == OPS_ARG_RED) {
        if (c->red_ops[a.handle] == kScalarHandle)
          return fail(c, OPS_ERR_INVALID_ARG, "loop '%s' arg %d: handle %d is a scalar, not a reduction", q.name.c_str(),
                      i, a.handle);
        if (std::find(seen_red.begin(), seen_red.end(), a.handle) != seen_red.end())
          return fail(c, OPS_ERR_INVALID_ARG, "loop '%s': reduction %d appears twice", q.name.c_str(), a.handle);
        seen_red.push_back(a.handle);
        ++nreds;
      }
    } else {
      return fail(c, OPS_ERR_INVALID_ARG, "loop '%s' arg %d: bad kind %d", q.name.c_str(), i, a.kind);
    }
  }
  if (nreds > OPS_MAX_REDS_PER_LOOP)
    return fail(c, OPS_ERR_INVALID_ARG, "loop '%s': more than %d reductions", q.name.c_str(), OPS_MAX_REDS_PER_LOOP);
  int64_t npts = 1;
  for (int d = 0; d < 3; ++d) npts *= (int64_t)(q.rng[2 * d + 1] - q.rng[2 * d]);
  if (npts > (int64_t)kMaxLoopPoints)
    return fail(c, OPS_ERR_INVALID_ARG, "loop '%s': %lld points, at most %d per loop", q.name.c_str(),
                (long long)npts, kMaxLoopPoints);
  const int nins = (int)q.code.size() / 6;
  auto is_dat = [&](int a) { return a >= 0 && a < nargs && q.args[a].kind == OPS_ARG_DAT; };
  for (int pc = 0; pc < nins; ++pc) {
    const int32_t* I = &q.code[6 * pc];
    const int op = I[0], d = I[1], a = I[2], b = I[3], cc = I[4], e = I[5];
    bool ok = true;
    switch (op) {
      case OPS_IR_LD:
        ok = valid_reg(d) && a >= 0 && a < nargs;
        if (ok && q.args[a].kind == OPS_ARG_DAT) {
          const int acc = q.args[a].access;
          ok = (acc == OPS_READ || acc == OPS_RW) && b >= 0 && b < (int)c->stencils[q.args[a].stencil].off.size() / 3;
        } else if (ok) {
          ok = q.args[a].kind == OPS_ARG_SCALAR && b == 0;
        }
        break;
      case OPS_IR_CST: ok = valid_reg(d) && a >= 0 && a < nK; break;
      case OPS_IR_ADD: case OPS_IR_SUB: case OPS_IR_MUL: case OPS_IR_DIV: case OPS_IR_MIN: case OPS_IR_MAX:
        ok = valid_reg(d) && valid_reg(a) && valid_reg(b);
        break;
      case OPS_IR_FMA: ok = valid_reg(d) && valid_reg(a) && valid_reg(b) && valid_reg(cc); break;
      case OPS_IR_SGT: ok = valid_reg(d) && valid_reg(a) && valid_reg(b) && valid_reg(cc) && valid_reg(e); break;
      case OPS_IR_WSUM: case OPS_IR_WACC:
        ok = valid_reg(d) && is_dat(a) && (q.args[a].access == OPS_READ || q.args[a].access == OPS_RW) && b >= 0 &&
             b + (int)c->stencils[q.args[a].stencil].off.size() / 3 <= nK;
        break;
      case OPS_IR_POLY: ok = valid_reg(d) && valid_reg(a) && b >= 0 && cc >= 0 && b + cc < nK; break;
      case OPS_IR_ST: ok = is_dat(d) && q.args[d].access != OPS_READ && valid_reg(a); break;
      case OPS_IR_RED: ok = d >= 0 && d < nargs && q.args[d].kind == OPS_ARG_RED && valid_reg(a); break;
      default: ok = false;
    }
    if (!ok)
      return fail(c, OPS_ERR_INVALID_ARG, "loop '%s': malformed IR instruction %d (op %d %d %d %d %d %d)",
                  q.name.c_str(), pc, op, d, a, b, cc, e);
  }
  return OPS_OK;
}

// ---------------------------------------------------------------------------
// flush
// ---------------------------------------------------------------------------
void fill_dloop(ops_ctx c, const QLoop& q, DLoop& L, int part_row, std::vector<FoldRow>& rows) {
  std::memset(&L, 0, sizeof L);
  L.nargs = (int)q.args.size();
  L.nins = (int)q.code.size() / 6;
  for (int i = 0; i < 6; ++i) L.rng[i] = q.rng[i];
  for (int d = q.dims; d < 3; ++d) {
    L.rng[2 * d] = 0;
    L.rng[2 * d + 1] = 1;
  }
  std::memcpy(L.ins, q.code.data(), sizeof(int32_t) * q.code.size());
  std::memcpy(L.K, q.K.data(), sizeof(double) * q.K.size());
  L.part_row = part_row;
  int k = 0;
  for (int i = 0; i < L.nargs; ++i) {
    const ops_arg& a = q.args[i];
    DArg& A = L.args[i];
    A.kind = a.kind;
    A.access = a.access;
    if (a.kind == OPS_ARG_DAT) {
      const Dat& D = c->dats[a.handle];
      const Stencil& s = c->stencils[a.stencil];
      A.ptr0 = D.ptr0;
      A.pitch = D.pitch;
      A.plane = D.plane;
      A.npts = (int)s.off.size() / 3;
      for (int p = 0; p < A.npts; ++p)
        A.off[p] = (int32_t)(s.off[3 * p] + s.off[3 * p + 1] * D.pitch + s.off[3 * p + 2] * D.plane);
      for (int d = 0; d < 3; ++d) {
        A.alo[d] = -D.dm[d];
        A.ahi[d] = D.size[d] + D.dp[d];
        A.slo[d] = s.lo[d];
        A.shi[d] = s.hi[d];
      }
    } else if (a.kind == OPS_ARG_SCALAR) {
      A.slot = a.handle;
    } else {
      A.slot = k;
      L.red_op[k] = c->red_ops[a.handle];
      rows.push_back(FoldRow{a.handle, c->red_ops[a.handle]});
      ++k;
    }
  }
  L.nreds = k;
  finish_dloop(L);
}

PLoop plan_loop(ops_ctx c, const QLoop& q) {
  PLoop p;
  for (int i = 0; i < 6; ++i) p.rng[i] = q.rng[i];
  for (int d = q.dims; d < 3; ++d) {
    p.rng[2 * d] = 0;
    p.rng[2 * d + 1] = 1;
  }
  for (const ops_arg& a : q.args) {
    PArg pa;
    pa.kind = a.kind;
    pa.dat = a.kind == OPS_ARG_DAT ? a.handle : -1;
    pa.reads = a.kind == OPS_ARG_DAT && (a.access == OPS_READ || a.access == OPS_RW || a.access == OPS_INC);
    pa.writes = a.kind == OPS_ARG_DAT && a.access != OPS_READ;
    for (int d = 0; d < 3; ++d) {
      pa.slo[d] = a.kind == OPS_ARG_DAT ? c->stencils[a.stencil].lo[d] : 0;
      pa.shi[d] = a.kind == OPS_ARG_DAT ? c->stencils[a.stencil].hi[d] : 0;
    }
    p.args.push_back(pa);
  }
  return p;
}

// Automatic tile size (Sec. 4.C, adapted): bytes per grid point = element size x the
// number of distinct dats of the segment; rows stay whole (x untiled, so
// every access is a long coalesced row) and the outermost tiled dimension
// gets as many points as fit the L2 budget.
void auto_tile(ops_ctx c, const std::vector<PLoop>& pl, int ndim, int tile[3]) {
  std::vector<char> used(c->dats.size(), 0);
  int ndat = 0;
  int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {-(1 << 30), -(1 << 30), -(1 << 30)};
  for (const PLoop& p : pl) {
    for (const PArg& a : p.args)
      if (a.kind == OPS_ARG_DAT && !used[a.dat]) {
        used[a.dat] = 1;
        ++ndat;
      }
    for (int d = 0; d < 3; ++d) {
      lo[d] = std::min(lo[d], p.rng[2 * d]);
      hi[d] = std::max(hi[d], p.rng[2 * d + 1]);
    }
  }
  const int64_t budget = c->cfg.l2_bytes > 0 ? c->cfg.l2_bytes : (c->l2_size > 0 ? c->l2_size * 3 / 4 : 96ll << 20);
  const int64_t bpp = (int64_t)c->es * std::max(1, ndat);
  int64_t pts = std::max<int64_t>(1, budget / bpp);
  for (int d = 0; d < 3; ++d) tile[d] = std::max(1, hi[d] - lo[d]);
  // shrink the outermost dimensions first until a tile fits the budget
  for (int d = ndim - 1; d >= 0; --d) {
    int64_t inner = 1;
    for (int e = 0; e < d; ++e) inner *= tile[e];
    if (inner * tile[d] <= pts) break;
    if (d == 0) {
      tile[0] = (int)std::max<int64_t>(1, pts);
    } else {
      tile[d] = (int)std::max<int64_t>(1, pts / inner);
      if (inner <= pts) break;
    }
  }
}

// Record a timing event on the context's stream (timing=1 only).
int record_event(ops_ctx c) {
  if (!c->cfg.timing) return OPS_OK;
  if (c->ev_used == (int)c->ev_pool.size()) {
    cudaEvent_t e;
    CUDA_TRY(c, cudaEventCreate(&e));
    c->ev_pool.push_back(e);
  }
  CUDA_TRY(c, cudaEventRecord(c->ev_pool[c->ev_used++], c->stream));
  return OPS_OK;
}

std::vector<int> segment_signature(ops_ctx c, int first, int count);

// Make room for `bytes` of staged copies in this flush: waits for the
// previous flush's staged copies, then grows the pinned buffer if needed.
int stage_begin(ops_ctx c, size_t bytes) {
  const int k = c->stage_slot ^= 1;
  if (c->stage_live[k]) {
    CUDA_TRY(c, cudaEventSynchronize(c->ev_stage[k]));
    c->stage_live[k] = false;
  }
  c->stage_used = 0;
  if (bytes > c->stage_cap[k]) {
    if (c->h_stage[k]) cudaFreeHost(c->h_stage[k]);
    c->h_stage[k] = nullptr;
    c->stage_cap[k] = 0;
    // slack for the batch tables a batched flush stages after the descriptors
    const size_t want = std::max<size_t>(bytes + (64 << 10), 128 << 10);
    CUDA_TRY(c, cudaHostAlloc((void**)&c->h_stage[k], want, cudaHostAllocDefault));
    c->stage_cap[k] = want;
  }
  if (!c->ev_stage[k]) CUDA_TRY(c, cudaEventCreateWithFlags(&c->ev_stage[k], cudaEventDisableTiming));
  return OPS_OK;
}

// Host-to-device copy on the context's stream through the pinned staging
// (a plain pageable copy when the staging is full).
int stage_copy(ops_ctx c, void* dst, const void* src, size_t bytes) {
  const int k = c->stage_slot;
  const size_t at = (c->stage_used + 15) / 16 * 16;
  if (!c->h_stage[k] || at + bytes > c->stage_cap[k]) {
    CUDA_TRY(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream));
    return OPS_OK;
  }
  std::memcpy(c->h_stage[k] + at, src, bytes);
  CUDA_TRY(c, cudaMemcpyAsync(dst, c->h_stage[k] + at, bytes, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaEventRecord(c->ev_stage[k], c->stream));
  c->stage_live[k] = true;
  c->stage_used = at + bytes;
  return OPS_OK;
}

// Bring d_loops[first, first + count) up to date with hl (the context's
// descriptor cache), copying the runs of entries changed since the device
// last received them.
int upload_loops(ops_ctx c, const std::vector<DLoop>& hl, int first, int count) {
  if (c->mirror_of != c->d_loops) {
    c->dev_ok.clear();
    c->mirror_of = c->d_loops;
  }
  if ((int)c->dev_ok.size() < first + count) c->dev_ok.resize(first + count, 0);
  int i = first;
  const int end = first + count;
  while (i < end) {
    if (c->dev_ok[i]) {
      ++i;
      continue;
    }
    int j = i + 1;
    while (j < end && !c->dev_ok[j]) ++j;
    int rc = stage_copy(c, c->d_loops + i, hl.data() + i, sizeof(DLoop) * (j - i));
    if (rc) return rc;
    std::fill(c->dev_ok.begin() + i, c->dev_ok.begin() + j, 1);
    i = j;
  }
  return OPS_OK;
}

// Overlapped tiles (Sec. 4.D, CTA tiles in place of MPI ranks).  The tiles
// partition the dats' allocation box; in each tile the loops run on the boxes
// of build_overlap_tile and each dat lives in a shared-memory footprint that
// holds what the tile reads, computes and owns.  A run of loops is eligible
// when every dat it touches is library-owned with one common size and halo.
// Halos grow with every loop of a run, so a run is cut into sub-runs short
// enough that, for tiles of at least kOvMinX points in x, the footprints fit
// one CTA's shared memory and the points computed stay within
// kOvMaxRedundancy times the points the loops own.
constexpr double kOvMaxRedundancy = 2.0;
constexpr int kOvMinX = 32;

// Plan loops [first, first + n) for tile T (shrunk while needed); nullptr
// when no tile makes them fit.  Plans, and failures, are cached by the loops'
// signature and the requested tile.
int overlap_plan(ops_ctx c, int first, int n, const int* tile_in, OverlapPlan** out) {
  *out = nullptr;
  const int ndim = c->queue[first].dims;
  std::vector<int> seg;
  std::map<int, int> local;
  for (int i = 0; i < n; ++i)
    for (const ops_arg& a : c->queue[first + i].args)
      if (a.kind == OPS_ARG_DAT && !local.count(a.handle)) {
        local[a.handle] = (int)seg.size();
        seg.push_back(a.handle);
      }
  if (seg.empty()) return OPS_OK;
  const Dat& D0 = c->dats[seg[0]];
  for (int h : seg) {
    const Dat& D = c->dats[h];
    if (!D.alloc || D.pitch != D0.pitch || D.plane != D0.plane) return OPS_OK;
    for (int d = 0; d < 3; ++d)
      if (D.size[d] != D0.size[d] || D.dm[d] != D0.dm[d] || D.dp[d] != D0.dp[d]) return OPS_OK;
  }
  int alo[3], ahi[3];
  for (int d = 0; d < 3; ++d) {
    alo[d] = -D0.dm[d];
    ahi[d] = D0.size[d] + D0.dp[d];
  }
  int T[3];
  const int def[3][3] = {{2048, 1, 1}, {64, 32, 1}, {32, 16, 8}};
  for (int d = 0; d < 3; ++d) {
    T[d] = d < ndim ? (tile_in[d] > 0 ? tile_in[d] : def[ndim - 1][d]) : 1;
    T[d] = std::max(1, std::min(T[d], ahi[d] - alo[d]));
  }
  std::vector<int> key = segment_signature(c, first, n);
  key.push_back(-7);  // overlapped
  for (int d = 0; d < 3; ++d) key.push_back(T[d]);
  auto it = c->oplans.find(key);
  if (it != c->oplans.end()) {
    *out = it->second.get();
    if (*out) ++c->stats.plan_cache_hits;
    return OPS_OK;
  }
  auto t0 = std::chrono::steady_clock::now();
  std::vector<PLoop> pl;
  for (int i = 0; i < n; ++i) pl.push_back(plan_loop(c, c->queue[first + i]));
  const int nd = (int)seg.size();
  std::vector<int> written(nd, 0);
  for (int i = 0; i < n; ++i)
    for (const PArg& a : pl[i].args)
      if (a.kind == OPS_ARG_DAT && a.writes) written[local[a.dat]] = 1;
  const int area_cap = overlap_smem_area_bytes();
  // points of each loop's range, for the redundancy of a tile
  OverlapTile ot;
  // Geometry of the tile with corner index tt: owned box, loop boxes, footprints.
  auto eval_tile = [&](const int tt[3], int* own6, int* box6n, int* foot6d, int64_t* computed, int64_t* useful) {
    int ob[6];
    for (int d = 0; d < 3; ++d) {
      ob[2 * d] = alo[d] + tt[d] * T[d];
      ob[2 * d + 1] = std::min(ahi[d], ob[2 * d] + T[d]);
    }
    build_overlap_tile(pl, (int)c->dats.size(), ndim, ob, ot);
    std::memcpy(own6, ob, sizeof ob);
    *computed = *useful = 0;
    for (int l = 0; l < n; ++l) {
      int64_t pts = 1, upts = 1;
      for (int d = 0; d < 3; ++d) {
        box6n[6 * l + 2 * d] = ot.box[(size_t)6 * l + 2 * d];
        box6n[6 * l + 2 * d + 1] = ot.box[(size_t)6 * l + 2 * d + 1];
        pts *= std::max(0, ot.box[(size_t)6 * l + 2 * d + 1] - ot.box[(size_t)6 * l + 2 * d]);
        upts *= std::max(0, std::min(ob[2 * d + 1], pl[l].rng[2 * d + 1]) - std::max(ob[2 * d], pl[l].rng[2 * d]));
      }
      *computed += pts;
      *useful += upts;
    }
    for (int k = 0; k < nd; ++k) {
      const int h = seg[k];
      int F[6];
      for (int d = 0; d < 3; ++d) {
        F[2 * d] = 1 << 30;
        F[2 * d + 1] = -(1 << 30);
      }
      auto hull = [&](const int* b) {
        for (int d = 0; d < 3; ++d)
          if (b[2 * d + 1] <= b[2 * d]) return;
        for (int d = 0; d < 3; ++d) {
          F[2 * d] = std::min(F[2 * d], b[2 * d]);
          F[2 * d + 1] = std::max(F[2 * d + 1], b[2 * d + 1]);
        }
      };
      hull(&ot.foot[(size_t)6 * h]);
      for (int l = 0; l < n; ++l)
        for (const PArg& a : pl[l].args)
          if (a.kind == OPS_ARG_DAT && a.writes && a.dat == h) hull(&ot.box[(size_t)6 * l]);
      if (written[k]) hull(ob);
      bool empty = false;
      for (int d = 0; d < 3; ++d) {
        F[2 * d] = std::max(F[2 * d], alo[d]);
        F[2 * d + 1] = std::min(F[2 * d + 1], ahi[d]);
        if (F[2 * d + 1] <= F[2 * d]) empty = true;
      }
      if (empty) {
        for (int d = 0; d < 6; ++d) F[d] = 0;
      } else {
        // x widened to multiples of v = 16 bytes / element: grid x = 0
        // starts a 128-byte line and pitch and plane are whole lines, so
        // footprint rows then move as whole 16-byte bulk copies.  The
        // widening stays inside the row's 128-byte lines, which the
        // library's layout always holds (x = 0 sits at the line-rounded
        // front halo; the pitch rounds the row up to whole lines).
        const int v = 16 / c->es;
        F[0] -= ((F[0] % v) + v) % v;
        F[1] += (v - ((F[1] % v) + v) % v) % v;
      }
      std::memcpy(&foot6d[6 * k], F, sizeof F);
    }
  };
  // shared-memory doubles of footprints with extents m (3 per dat), 16-byte aligned regions
  auto area_of = [&](const std::vector<int>& m, std::vector<int>* sp, std::vector<int>* sq, std::vector<int>* so) {
    int64_t off = 0;
    for (int k = 0; k < nd; ++k) {
      const int p = std::max(1, m[3 * k]), q = p * std::max(1, m[3 * k + 1]);
      if (sp) {
        (*sp)[k] = p;
        (*sq)[k] = q;
        (*so)[k] = (int)off;
      }
      const int64_t v = 16 / c->es;  // regions start on 16-byte boundaries
      off += ((int64_t)q * std::max(1, m[3 * k + 2]) + v - 1) / v * v;
    }
    return off * c->es;
  };
  std::unique_ptr<OverlapPlan> np;
  std::vector<int> one_box((size_t)6 * n), one_foot((size_t)6 * nd), own6(6);
  for (int attempt = 0; attempt < 32 && !np; ++attempt) {
    int nt[3];
    for (int d = 0; d < 3; ++d) nt[d] = (ahi[d] - alo[d] + T[d] - 1) / T[d];
    // the centre tile first: most halo, no boundary clipping
    const int tc[3] = {nt[0] / 2, nt[1] / 2, nt[2] / 2};
    int64_t comp = 0, use = 0;
    eval_tile(tc, own6.data(), one_box.data(), one_foot.data(), &comp, &use);
    std::vector<int> m(3 * nd);
    for (int k = 0; k < nd; ++k)
      for (int d = 0; d < 3; ++d) m[3 * k + d] = one_foot[6 * k + 2 * d + 1] - one_foot[6 * k + 2 * d];
    bool ok = area_of(m, nullptr, nullptr, nullptr) <= area_cap && comp <= kOvMaxRedundancy * (double)std::max<int64_t>(1, use);
    if (ok) {
      const int ntiles = nt[0] * nt[1] * nt[2];
      std::vector<int> own((size_t)6 * ntiles), boxes((size_t)6 * ntiles * n), foot((size_t)6 * ntiles * nd);
      std::fill(m.begin(), m.end(), 0);
      int64_t computed = 0, useful = 0;
      for (int tz = 0, t = 0; tz < nt[2]; ++tz)
        for (int ty = 0; ty < nt[1]; ++ty)
          for (int tx = 0; tx < nt[0]; ++tx, ++t) {
            const int tt[3] = {tx, ty, tz};
            int64_t cp = 0, us = 0;
            eval_tile(tt, &own[(size_t)6 * t], &boxes[(size_t)6 * t * n], &foot[(size_t)6 * t * nd], &cp, &us);
            computed += cp;
            useful += us;
            for (int k = 0; k < nd; ++k)
              for (int d = 0; d < 3; ++d)
                m[3 * k + d] = std::max(m[3 * k + d], foot[(size_t)6 * (t * nd + k) + 2 * d + 1] -
                                                          foot[(size_t)6 * (t * nd + k) + 2 * d]);
          }
      np.reset(new OverlapPlan);
      np->spitch.assign(nd, 0);
      np->splane.assign(nd, 0);
      np->smem_off.assign(nd, 0);
      const int64_t area = area_of(m, &np->spitch, &np->splane, &np->smem_off);
      if (area > area_cap) {
        np.reset();  // a boundary tile is larger than the centre one
      } else {
        np->ntiles = ntiles;
        np->area_bytes = (int)area;
        np->redundant = computed - useful;
        np->own_off = 0;
        np->box_off = (int)own.size();
        np->foot_off = (int)(own.size() + boxes.size());
        std::vector<int> tab(own);
        tab.insert(tab.end(), boxes.begin(), boxes.end());
        tab.insert(tab.end(), foot.begin(), foot.end());
        np->tab_ints = tab.size();
        int rc = dev_alloc(c, (void**)&np->d_tab, sizeof(int) * tab.size());
        if (rc) return rc;
        CUDA_TRY(c, cudaMemcpyAsync(np->d_tab, tab.data(), sizeof(int) * tab.size(), cudaMemcpyHostToDevice,
                                    c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        break;
      }
    }
    // halve the largest tile dimension that may shrink (x stays >= kOvMinX in 2D / 3D)
    int big = -1;
    for (int d = 0; d < ndim; ++d) {
      const int floor_d = (d == 0 && ndim > 1) ? kOvMinX : 1;
      if (T[d] > floor_d && (big < 0 || T[d] > T[big])) big = d;
    }
    if (big < 0) break;
    T[big] = std::max((big == 0 && ndim > 1) ? kOvMinX : 1, (T[big] + 1) / 2);
  }
  c->stats.plan_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (!np) {
    c->oplans[key] = nullptr;
    return OPS_OK;
  }
  for (int d = 0; d < 3; ++d) np->tile[d] = T[d];
  np->first_loop = first;
  np->nloops = n;
  np->ndats = nd;
  np->seg_dats = seg;
  np->written = written;
  *out = np.get();
  c->oplans[key] = std::move(np);
  return OPS_OK;
}

// Launch one overlapped plan over loops [first, first + op->nloops).
// The run's descriptors in shared-memory layout: DAT args get the
// footprint strides, stencil offsets in those strides, slot = run dat index.
std::vector<DLoop> overlap_descriptors(ops_ctx c, int first, const std::vector<DLoop>& hl, const OverlapPlan* op) {
  const int n = op->nloops;
  std::map<int, int> local;
  for (int k = 0; k < op->ndats; ++k) local[op->seg_dats[k]] = k;
  std::vector<DLoop> ol(hl.begin() + first, hl.begin() + first + n);
  for (int i = 0; i < n; ++i) {
    const QLoop& q = c->queue[first + i];
    for (int a = 0; a < (int)q.args.size(); ++a) {
      if (q.args[a].kind != OPS_ARG_DAT) continue;
      const int k = local[q.args[a].handle];
      DArg& A = ol[i].args[a];
      const Stencil& s = c->stencils[q.args[a].stencil];
      A.ptr0 = nullptr;
      A.pitch = op->spitch[k];
      A.plane = op->splane[k];
      A.slot = k;
      for (int p = 0; p < A.npts; ++p)
        A.off[p] = (int32_t)(s.off[3 * p] + (int64_t)s.off[3 * p + 1] * A.pitch + (int64_t)s.off[3 * p + 2] * A.plane);
    }
  }
  return ol;
}

OvLayout overlap_layout(const OverlapPlan* op, int es) {
  OvLayout lay;
  lay.es = es;
  lay.ndats = op->ndats;
  lay.smem_off = op->smem_off;
  lay.spitch = op->spitch;
  lay.splane = op->splane;
  lay.written = op->written;
  return lay;
}

// Launch one overlapped run: jo = its compiled kernel, or nullptr for the interpreter kernel.
int run_overlap_plan(ops_ctx c, int first, const std::vector<DLoop>& hl, const OverlapPlan* op,
                     const std::vector<DLoop>& ol, JitOverlap* jo) {
  const int n = op->nloops;
  int rc = ensure(c, &c->d_oloops, &c->oloops_cap, n);
  if (rc) return rc;
  CUDA_TRY(c, cudaMemcpyAsync(c->d_oloops, ol.data(), sizeof(DLoop) * n, cudaMemcpyHostToDevice, c->stream));
  std::vector<OvDat> ov(op->ndats);
  for (int k = 0; k < op->ndats; ++k) {
    Dat& D = c->dats[op->seg_dats[k]];
    if (op->written[k] && !D.alt) {
      rc = dev_alloc(c, (void**)&D.alt, D.bytes);
      if (rc) return rc;
      D.alt_ptr0 = (double*)((char*)D.alt + ((char*)D.ptr0 - (char*)D.alloc));
    }
    ov[k].src = D.ptr0;
    ov[k].dst = op->written[k] ? D.alt_ptr0 : nullptr;
    ov[k].gpitch = D.pitch;
    ov[k].gplane = D.plane;
    ov[k].written = op->written[k];
    ov[k].smem_off = op->smem_off[k];
    ov[k].spitch = op->spitch[k];
    ov[k].splane = op->splane[k];
  }
  rc = ensure(c, &c->d_ovdat, &c->ovdat_cap, op->ndats);
  if (rc) return rc;
  CUDA_TRY(c, cudaMemcpyAsync(c->d_ovdat, ov.data(), sizeof(OvDat) * op->ndats, cudaMemcpyHostToDevice, c->stream));
  LaunchEnv env = make_env(c);
  int row0 = -1, nrows = 0;
  for (int i = 0; i < n; ++i) {
    const DLoop& L = hl[first + i];
    if (L.nreds) {
      if (row0 < 0) row0 = L.part_row;
      nrows = L.part_row + L.nreds - row0;
    }
  }
  int grid = 0;
  if (jo) grid = std::min({op->ntiles, jit_overlap_max_grid(jo, c->num_sms, op->area_bytes), c->part_stride});
  if (grid <= 0) jo = nullptr;
  if (!jo && c->es == 4) return fail(c, OPS_ERR_INVALID_ARG, "FP32 overlapped tiles run compiled bodies only");
  if (!jo) grid = std::max(1, std::min({op->ntiles, overlap_max_grid(c->num_sms, op->area_bytes), c->part_stride}));
  c->stats.compiled = jo ? 1 : 0;
  if (nrows) {
    CUDA_TRY(c, launch_part_init(env, row0, nrows));
    ++c->stats.launches;
  }
  rc = record_event(c);
  if (rc) return rc;
  if (jo)
    CUDA_TRY(c, jit_launch_overlap(jo, env, c->d_oloops, c->d_ovdat, op->d_tab + op->own_off, op->d_tab + op->box_off,
                                   op->d_tab + op->foot_off, op->ntiles, grid, op->area_bytes));
  else
    CUDA_TRY(c, launch_overlap(env, c->d_oloops, n, c->d_ovdat, op->ndats, op->d_tab + op->own_off,
                               op->d_tab + op->box_off, op->d_tab + op->foot_off, op->ntiles, grid, op->area_bytes));
  rc = record_event(c);
  if (rc) return rc;
  ++c->stats.launches;
  ++c->stats.kernel_launches;
  if (nrows) {
    CUDA_TRY(c, launch_fold(env, row0, nrows, grid));
    ++c->stats.launches;
  }
  // the other buffers now hold every written dat
  for (int k = 0; k < op->ndats; ++k)
    if (op->written[k]) {
      Dat& D = c->dats[op->seg_dats[k]];
      std::swap(D.alloc, D.alt);
      std::swap(D.ptr0, D.alt_ptr0);
      ++c->swap_gen;
    }
  ++c->stats.segments;
  c->stats.loops += n;
  c->stats.tiles = op->ntiles;
  for (int d = 0; d < 3; ++d) c->stats.tile[d] = op->tile[d];
  c->stats.redundant_points += op->redundant;
  for (int i = 0; i < n; ++i) {
    int64_t p = 1;
    for (int d = 0; d < 3; ++d) p *= std::max(0, hl[first + i].rng[2 * d + 1] - hl[first + i].rng[2 * d]);
    c->stats.points += p;
  }
  return OPS_OK;
}

// Longest leading run of loops [first, first + count) that has an overlapped
// plan (halving the run until one fits); *used = 0 when not even one loop does.
int overlap_prefix(ops_ctx c, int first, int count, const int* tile_in, OverlapPlan** out, int* used) {
  *used = 0;
  for (int n = count; n >= 1; n = n / 2) {
    int rc = overlap_plan(c, first, n, tile_in, out);
    if (rc) return rc;
    if (*out) {
      *used = n;
      return OPS_OK;
    }
  }
  return OPS_OK;
}

// Compiled kernels of a segment, generated from its loops' IR at its first
// flush; *out = nullptr (interpreter kernels) in checked mode, with
// interpret = 1, or when run-time compilation is unavailable.
std::vector<int> code_key(ops_ctx c, int first, int count) {
  std::vector<int> key = segment_signature(c, first, count);
  for (int i = 0; i < count; ++i) {
    const QLoop& q = c->queue[first + i];
    key.push_back(-1);
    key.insert(key.end(), q.code.begin(), q.code.end());
  }
  return key;
}

// dats no loop of the segment writes are read through the read-only path
std::vector<std::vector<char>> read_only_args(ops_ctx c, int first, int count) {
  std::set<int> written;
  for (int i = 0; i < count; ++i)
    for (const ops_arg& a : c->queue[first + i].args)
      if (a.kind == OPS_ARG_DAT && a.access != OPS_READ) written.insert(a.handle);
  std::vector<std::vector<char>> ro(count);
  for (int i = 0; i < count; ++i) {
    const QLoop& q = c->queue[first + i];
    ro[i].assign(q.args.size(), 0);
    for (size_t a = 0; a < q.args.size(); ++a)
      ro[i][a] = q.args[a].kind == OPS_ARG_DAT && !written.count(q.args[a].handle);
  }
  return ro;
}

int segment_code(ops_ctx c, int first, int count, const std::vector<DLoop>& hl, JitSegment** out) {
  *out = nullptr;
  if (c->cfg.interpret || c->cfg.check) return OPS_OK;
  std::vector<int> key = code_key(c, first, count);
  auto it = c->jit.find(key);
  if (it != c->jit.end()) {
    *out = it->second;
    return OPS_OK;
  }
  std::vector<std::vector<char>> ro = read_only_args(c, first, count);
  JitSegment* s = nullptr;
  std::string why;
  double ms = 0.0;
  const int rc = jit_segment(c->cfg.device, hl.data() + first, count, ro, c->es, &s, &why, &ms);
  c->stats.compile_ms += ms;
  if (rc) return fail(c, rc, "compiling loop bodies: %s", why.c_str());
  if (!s) c->jit_why = why;
  c->jit[key] = s;
  *out = s;
  return OPS_OK;
}

// Wavefront kernel of a segment (every loop body in one module), compiled
// at the segment's first wavefront flush; nullptr when run-time compilation
// is unavailable (reason in jit_why).
int wave_code(ops_ctx c, int first, int count, const std::vector<DLoop>& hl, JitWave** out) {
  *out = nullptr;
  std::vector<int> key = code_key(c, first, count);
  auto it = c->jitw.find(key);
  if (it != c->jitw.end()) {
    *out = it->second;
    return OPS_OK;
  }
  std::vector<std::vector<char>> ro = read_only_args(c, first, count);
  JitWave* w = nullptr;
  std::string why;
  double ms = 0.0;
  const int rc = jit_wavefront(c->cfg.device, hl.data() + first, count, ro, c->es, &w, &why, &ms);
  c->stats.compile_ms += ms;
  if (rc) return fail(c, rc, "compiling the wavefront kernel: %s", why.c_str());
  if (!w) c->jit_why = why;
  c->jitw[key] = w;
  *out = w;
  return OPS_OK;
}

// Points of one wavefront tile along the outermost dimension when the tile
// size is automatic: about 64 full 4096-point rows (the fastest of 4-64 rows
// on the 3840^2 CloverLeaf-shaped chain, FP32 and FP64).
constexpr int64_t kWavePoints = 64 * 4096;

// The plan of a wavefront segment (cached like the skewed plans): Algorithm
// 1's ranges for thin tiles along the outermost dimension (the others
// untiled unless a tile size is given), Algorithm 2's phase order, and the
// dependency lists and work units of build_wavefront, uploaded once.
int wave_plan(ops_ctx c, int first, int count, const int* tile_in, CachedPlan** out) {
  const int ndim = c->queue[first].dims;
  std::vector<PLoop> pl;
  pl.reserve(count);
  for (int i = 0; i < count; ++i) pl.push_back(plan_loop(c, c->queue[first + i]));
  int ext[3] = {1, 1, 1};
  for (int d = 0; d < ndim; ++d) {
    int lo = 1 << 30, hi = -(1 << 30);
    for (const PLoop& p : pl) {
      lo = std::min(lo, p.rng[2 * d]);
      hi = std::max(hi, p.rng[2 * d + 1]);
    }
    ext[d] = std::max(1, hi - lo);
  }
  int tile[3] = {1, 1, 1};
  int64_t inner = 1;
  for (int d = 0; d + 1 < ndim; ++d) {
    tile[d] = tile_in[d] > 0 ? tile_in[d] : ext[d];
    inner *= tile[d];
  }
  tile[ndim - 1] =
      tile_in[ndim - 1] > 0 ? tile_in[ndim - 1] : (int)std::max<int64_t>(1, kWavePoints / std::max<int64_t>(1, inner));
  const int P = jit_rows_per_unit(c->es), upc = jit_wave_units_per_chunk(), slope = jit_wave_slope();
  std::vector<int> key = {-OPS_MODE_WAVEFRONT, ndim, tile[0], tile[1], tile[2], P, upc, slope, jit_wave_threads()};
  for (int i = 0; i < count; ++i) {
    const QLoop& q = c->queue[first + i];
    for (int k = 0; k < 6; ++k) key.push_back(q.rng[k]);
    key.push_back((int)q.args.size());
    for (const ops_arg& a : q.args) {
      key.push_back(a.kind);
      key.push_back(a.handle);
      key.push_back(a.kind == OPS_ARG_DAT ? a.stencil : -1);
      key.push_back(a.access);
    }
  }
  auto it = c->plans.find(key);
  if (it != c->plans.end()) {
    ++c->stats.plan_cache_hits;
    *out = it->second.get();
    return OPS_OK;
  }
  auto t0 = std::chrono::steady_clock::now();
  std::unique_ptr<CachedPlan> np(new CachedPlan);
  np->key = key;
  build_skewed_ranges(pl, (int)c->dats.size(), ndim, tile, np->plan);
  build_phases(pl, np->plan);
  WavePlan& W = np->wave;
  build_wavefront(pl, (int)c->dats.size(), np->plan, ndim - 1, P, jit_wave_threads(), upc, slope, W);
  c->stats.plan_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  const size_t nph = np->plan.phases.size();
  if (W.nunits >= (1ll << 31) || W.deps.size() >= (1ull << 31))
    return fail(c, OPS_ERR_INVALID_ARG, "wavefront plan too large (%lld work units)", (long long)W.nunits);
  if (nph) {
    std::vector<WfPhase> tab(nph);
    for (size_t q = 0; q < nph; ++q) {
      WfPhase& f = tab[q];
      f.loop = np->plan.phases[q].loop;
      f.nchunk = W.nchunk[q];
      f.ustart = W.ustart[q];
      f.dep0 = W.dep_off[q];
      f.ndep = W.dep_off[q + 1] - W.dep_off[q];
      f.pad = W.level[q];
      for (int k = 0; k < 6; ++k) f.box[k] = np->plan.phases[q].box[k];
    }
    const size_t b0 = sizeof(WfPhase) * nph, b1 = sizeof(int) * W.deps.size(), b2 = sizeof(int) * W.uphase.size();
    np->wave_bytes = b0 + b1 + b2 + 16;
    int rc = dev_alloc(c, &np->d_wave, np->wave_bytes);
    if (!rc) rc = dev_alloc(c, (void**)&np->d_wdone, sizeof(int) * (nph + 1));
    if (rc) return rc;
    char* d = (char*)np->d_wave;
    CUDA_TRY(c, cudaMemcpyAsync(d, tab.data(), b0, cudaMemcpyHostToDevice, c->stream));
    if (b1) CUDA_TRY(c, cudaMemcpyAsync(d + b0, W.deps.data(), b1, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(d + b0 + b1, W.uphase.data(), b2, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));  // the host tables are temporaries
  }
  np->nlevels = W.nlevels;
  *out = np.get();
  c->plans[key] = std::move(np);
  return OPS_OK;
}

// Wavefront execution of a segment (OPS_MODE_WAVEFRONT): one persistent
// kernel takes the plan's work units in level order and waits, per unit,
// only on the phases it conflicts with.
int run_wavefront(ops_ctx c, int first, int count, int dl_base, std::vector<DLoop>& hl, const int* tile_in,
                  JitWave* w) {
  CachedPlan* cp = nullptr;
  int rc = wave_plan(c, first, count, tile_in, &cp);
  if (rc) return rc;
  const SkewedPlan& P = cp->plan;
  LaunchEnv env = make_env(c);
  c->stats.mode = OPS_MODE_WAVEFRONT;
  c->stats.compiled = 1;
  ++c->stats.segments;
  c->stats.loops += count;
  int ntiles = 1;
  for (int d = 0; d < 3; ++d) {
    ntiles *= P.ntiles[d];
    c->stats.tile[d] = P.tile[d];
    c->stats.skew[d] = P.skew[d];
  }
  c->stats.tiles = ntiles;
  c->stats.phases += (int)P.phases.size();
  c->stats.points += P.points;
  if (P.phases.empty()) return OPS_OK;
  const size_t nph = P.phases.size();
  int row0 = -1, nrows = 0;
  for (int i = 0; i < count; ++i) {
    const DLoop& L = hl[dl_base + i];
    if (L.nreds) {
      if (row0 < 0) row0 = L.part_row;
      nrows = L.part_row + L.nreds - row0;
    }
  }
  const int grid = std::min(std::max(1, jit_wavefront_max_grid(w, c->num_sms)), c->part_stride);
  if (nrows) {
    CUDA_TRY(c, launch_part_init(env, row0, nrows));
    ++c->stats.launches;
  }
  CUDA_TRY(c, cudaMemsetAsync(cp->d_wdone, 0, sizeof(int) * (nph + 1), c->stream));
  rc = record_event(c);
  if (rc) return rc;
  const char* d = (const char*)cp->d_wave;
  const WfPhase* d_ph = (const WfPhase*)d;
  const int* d_deps = (const int*)(d + sizeof(WfPhase) * nph);
  const int* d_uphase = d_deps + cp->wave.deps.size();
  CUDA_TRY(c, jit_launch_wavefront(w, env, c->d_loops + dl_base, d_ph, d_deps, d_uphase, (int)cp->wave.nunits,
                                   cp->d_wdone, cp->d_wdone + nph, grid));
  ++c->stats.launches;
  ++c->stats.kernel_launches;
  rc = record_event(c);
  if (rc) return rc;
  if (nrows) {
    CUDA_TRY(c, launch_fold(env, row0, nrows, grid));
    ++c->stats.launches;
  }
  return OPS_OK;
}

// Tile-wavefront kernel of a segment (every loop body in one module),
// compiled at the segment's first such flush; nullptr when run-time
// compilation is unavailable (reason in jit_why).
int tile_code(ops_ctx c, int first, int count, const std::vector<DLoop>& hl, JitTile** out, bool warp = false) {
  *out = nullptr;
  std::vector<int> key = code_key(c, first, count);
  if (warp) key.push_back(-OPS_MODE_TILEWARP);  // the tile-per-warp form
  auto it = c->jitt.find(key);
  if (it != c->jitt.end()) {
    *out = it->second;
    return OPS_OK;
  }
  std::vector<std::vector<char>> ro = read_only_args(c, first, count);
  JitTile* t = nullptr;
  std::string why;
  double ms = 0.0;
  const int rc = warp ? jit_tilewarp(c->cfg.device, hl.data() + first, count, ro, c->es, c->queue[first].dims, &t,
                                     &why, &ms)
                      : jit_tilewave(c->cfg.device, hl.data() + first, count, ro, c->es, c->queue[first].dims, &t,
                                     &why, &ms);
  c->stats.compile_ms += ms;
  if (rc) return fail(c, rc, "compiling the tile-wavefront kernel: %s", why.c_str());
  if (!t) c->jit_why = why;
  c->jitt[key] = t;
  *out = t;
  return OPS_OK;
}

// The persistent skewed kernel of a segment (compiled once per code).
int skew_code(ops_ctx c, int first, int count, const std::vector<DLoop>& hl, JitSkew** out) {
  *out = nullptr;
  std::vector<int> key = code_key(c, first, count);
  auto it = c->jitk.find(key);
  if (it != c->jitk.end()) {
    *out = it->second;
    return OPS_OK;
  }
  std::vector<std::vector<char>> ro = read_only_args(c, first, count);
  JitSkew* k = nullptr;
  std::string why;
  double ms = 0.0;
  const int rc = jit_skewed(c->cfg.device, hl.data() + first, count, ro, c->es, &k, &why, &ms);
  c->stats.compile_ms += ms;
  if (rc) return fail(c, rc, "compiling the persistent skewed kernel: %s", why.c_str());
  if (!k) c->jit_why = why;
  c->jitk[key] = k;
  *out = k;
  return OPS_OK;
}

// Automatic tile of the tile wavefront: 128 x 64 points in FP32 and 64 x 64
// in FP64 (2D), 64 x 16 x 16 (3D) -- the fastest shapes measured on GB300
// for the CloverLeaf- and PPCG-shaped chains; smaller, L2-sized tiles made
// more, shorter steps and ran slower.  Dimensions are capped by the extent,
// and tiles the chain's skew reaches across are grown by the planner.
void auto_tile_wave(ops_ctx c, const std::vector<PLoop>& pl, int ndim, int tile[3], bool warp = false) {
  int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {-(1 << 30), -(1 << 30), -(1 << 30)};
  for (const PLoop& p : pl)
    for (int d = 0; d < 3; ++d) {
      lo[d] = std::min(lo[d], p.rng[2 * d]);
      hi[d] = std::max(hi[d], p.rng[2 * d + 1]);
    }
  // a warp's tile is a quarter to an eighth of a CTA's: 64 x 32 FP32, 32 x 32 FP64, 32 x 8 x 8 in 3D
  const int shape2[2] = {warp ? (c->es == 4 ? 64 : 32) : (c->es == 4 ? 128 : 64), warp ? 32 : 64};
  const int shape3[3] = {warp ? 32 : 64, warp ? 8 : 16, warp ? 8 : 16};
  for (int d = 0; d < 3; ++d) {
    const int ext = std::max(1, hi[d] - lo[d]);
    int want = 1;
    if (d < ndim) want = ndim == 1 ? 8192 : (ndim == 2 ? shape2[d] : shape3[d]);
    tile[d] = std::min(ext, want);
  }
}

// The tile-wavefront plan of a segment (cached like the other plans).  A
// tile size the chain's skew reaches across is doubled in that dimension
// until the plan is valid; *out = nullptr (and jit_why says why) if no size
// up to the whole extent is.
int tile_plan(ops_ctx c, int first, int count, const std::vector<DLoop>& hl, int dl_base, const int* tile_in,
              CachedPlan** out, bool warp = false) {
  *out = nullptr;
  const int ndim = c->queue[first].dims;
  std::vector<PLoop> pl;
  pl.reserve(count);
  for (int i = 0; i < count; ++i) pl.push_back(plan_loop(c, c->queue[first + i]));
  int tile[3] = {tile_in[0], tile_in[1], tile_in[2]};
  bool autod = false;
  for (int d = 0; d < ndim; ++d) autod = autod || tile[d] <= 0;
  if (autod) {
    int at[3];
    auto_tile_wave(c, pl, ndim, at, warp);
    for (int d = 0; d < 3; ++d)
      if (tile[d] <= 0) tile[d] = at[d];
  }
  for (int d = ndim; d < 3; ++d) tile[d] = 1;
  std::vector<int> key = {-OPS_MODE_TILEWAVE, ndim, tile[0], tile[1], tile[2],
                          jit_tile_group(), jit_tile_prefetch(), jit_tile_band()};
  for (int i = 0; i < count; ++i) {
    const QLoop& q = c->queue[first + i];
    for (int k = 0; k < 6; ++k) key.push_back(q.rng[k]);
    key.push_back((int)q.args.size());
    for (const ops_arg& a : q.args) {
      key.push_back(a.kind);
      key.push_back(a.handle);
      key.push_back(a.kind == OPS_ARG_DAT ? a.stencil : -1);
      key.push_back(a.access);
    }
  }
  auto it = c->plans.find(key);
  if (it != c->plans.end()) {
    ++c->stats.plan_cache_hits;
    *out = it->second.get();
    return OPS_OK;
  }
  auto t0 = std::chrono::steady_clock::now();
  std::unique_ptr<CachedPlan> np(new CachedPlan);
  np->key = key;
  std::string why;
  bool ok = false;
  for (int attempt = 0; attempt < 24; ++attempt) {
    build_skewed_ranges(pl, (int)c->dats.size(), ndim, tile, np->plan);
    if (build_tile_wave(pl, np->plan, np->tw, &why, jit_tile_group(), jit_tile_band())) {
      ok = true;
      break;
    }
    const int d = np->tw.bad_dim;
    if (d < 0 || d >= ndim || np->plan.ntiles[d] <= 1) break;
    tile[d] *= 2;
  }
  c->stats.plan_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (!ok) {
    c->jit_why = "no tile size gives a valid tile wavefront: " + why;
    c->plans[key] = nullptr;
    return OPS_OK;
  }
  const SkewedPlan& P = np->plan;
  const TileWavePlan& W = np->tw;
  const int ntiles = P.ntiles[0] * P.ntiles[1] * P.ntiles[2];
  // ranges of every dimension (dimensions beyond the loops': each loop's (0, 1))
  std::vector<int> rng;
  for (int d = 0; d < 3; ++d) {
    np->tw_roff[d] = (int)rng.size();
    if (d < ndim) {
      rng.insert(rng.end(), P.ranges[d].begin(), P.ranges[d].end());
    } else {
      for (int l = 0; l < count; ++l) {
        rng.push_back(pl[l].rng[2 * d]);
        rng.push_back(pl[l].rng[2 * d + 1]);
      }
    }
  }
  std::vector<int> cls;
  for (int d = 0; d < 3; ++d) {
    np->tw_coff[d] = (int)cls.size();
    cls.insert(cls.end(), W.cls[d].begin(), W.cls[d].end());
  }
  // L2 prefetch masks per loop: its reading arguments whose dat no earlier
  // loop of the segment touched (mode 1), or all its reading arguments (2)
  std::vector<unsigned char> pf(count, 0);
  {
    const int pmode = jit_tile_prefetch();
    std::vector<char> seen(c->dats.size(), 0);
    for (int l = 0; l < count; ++l) {
      const QLoop& q = c->queue[first + l];
      for (size_t a = 0; a < q.args.size(); ++a) {
        const ops_arg& g = q.args[a];
        if (g.kind != OPS_ARG_DAT) continue;
        if (g.access != OPS_WRITE && (pmode == 2 || (pmode == 1 && !seen[g.handle]))) pf[l] |= (unsigned char)(1u << a);
      }
      for (const ops_arg& g : q.args)
        if (g.kind == OPS_ARG_DAT) seen[g.handle] = 1;
    }
  }
  const size_t b_rng = sizeof(int) * rng.size(), b_order = sizeof(int) * W.order.size(),
               b_cls = sizeof(int) * cls.size(), b_need = sizeof(uint16_t) * W.need.size(), b_pf = pf.size(),
               b_grp = sizeof(int) * W.groups.size();
  np->tw_order = (b_rng + 15) / 16 * 16;
  np->tw_cls = np->tw_order + (b_order + 15) / 16 * 16;
  np->tw_need = np->tw_cls + (b_cls + 15) / 16 * 16;
  np->tw_grp = np->tw_need + (b_need + 15) / 16 * 16;
  np->tw_pf = np->tw_grp + (b_grp + 15) / 16 * 16;
  np->tw_bytes = np->tw_pf + b_pf + 16;
  np->tw_ntiles = ntiles;
  int rows = 0;
  {
    int row0 = -1;
    for (int i = 0; i < count; ++i) {
      const DLoop& L = hl[dl_base + i];
      if (L.nreds) {
        if (row0 < 0) row0 = L.part_row;
        rows = L.part_row + L.nreds - row0;
      }
    }
  }
  np->tw_rows = rows;
  {
    // phases: per loop, the product over dimensions of the tiles its range meets;
    // steps: per tile, the loop groups with at least one non-empty loop
    int64_t ph = 0, st = 0;
    for (int l = 0; l < count; ++l) {
      int64_t k = 1;
      for (int d = 0; d < ndim; ++d) {
        int m = 0;
        for (int t = 0; t < P.ntiles[d]; ++t)
          m += P.ranges[d][2 * (t * count + l) + 1] > P.ranges[d][2 * (t * count + l)];
        k *= m;
      }
      ph += k;
    }
    st = (int64_t)ntiles * ((int64_t)W.groups.size() - 1);
    np->tw_phases = (int)std::min<int64_t>(ph, 1 << 30);
    np->tw_steps = (int)std::min<int64_t>(st, 1 << 30);
  }
  int rc = dev_alloc(c, &np->d_tw, np->tw_bytes);
  if (!rc) rc = dev_alloc(c, (void**)&np->d_twprog, sizeof(int) * (ntiles + 1));
  if (!rc && rows) rc = dev_alloc(c, (void**)&np->d_twpart, sizeof(DD) * (size_t)rows * ntiles);
  if (rc) return rc;
  char* d = (char*)np->d_tw;
  CUDA_TRY(c, cudaMemcpyAsync(d, rng.data(), b_rng, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(d + np->tw_order, W.order.data(), b_order, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(d + np->tw_cls, cls.data(), b_cls, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(d + np->tw_need, W.need.data(), b_need, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(d + np->tw_pf, pf.data(), b_pf, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(d + np->tw_grp, W.groups.data(), b_grp, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));  // the host tables are temporaries
  *out = np.get();
  c->plans[key] = std::move(np);
  return OPS_OK;
}

// Tile-wavefront execution of a segment (OPS_MODE_TILEWAVE).  *ran = false
// when no valid plan exists (the caller then runs the segment skewed).
int run_tilewave(ops_ctx c, int first, int count, int dl_base, std::vector<DLoop>& hl, const int* tile_in,
                 JitTile* t, bool* ran, bool warp = false) {
  *ran = false;
  CachedPlan* cp = nullptr;
  int rc = tile_plan(c, first, count, hl, dl_base, tile_in, &cp, warp);
  if (rc) return rc;
  if (!cp) return OPS_OK;
  *ran = true;
  const SkewedPlan& P = cp->plan;
  LaunchEnv env = make_env(c);
  c->stats.mode = warp ? OPS_MODE_TILEWARP : OPS_MODE_TILEWAVE;
  c->stats.compiled = 1;
  ++c->stats.segments;
  c->stats.loops += count;
  for (int d = 0; d < 3; ++d) {
    c->stats.tile[d] = P.tile[d];
    c->stats.skew[d] = P.skew[d];
  }
  c->stats.tiles = cp->tw_ntiles;
  c->stats.phases += cp->tw_phases;
  c->stats.barriers += cp->tw_steps;
  int64_t pts = 0;
  for (int l = 0; l < count; ++l) {
    int64_t n = 1;
    for (int d = 0; d < 3; ++d) {
      const QLoop& q = c->queue[first + l];
      const int a = d < q.dims ? q.rng[2 * d] : 0, b = d < q.dims ? q.rng[2 * d + 1] : 1;
      n *= std::max(0, b - a);
    }
    pts += n;
  }
  c->stats.points += pts;
  int row0 = -1, nrows = 0;
  for (int i = 0; i < count; ++i) {
    const DLoop& L = hl[dl_base + i];
    if (L.nreds) {
      if (row0 < 0) row0 = L.part_row;
      nrows = L.part_row + L.nreds - row0;
    }
  }
  if (nrows > cp->tw_rows) return fail(c, OPS_ERR_STATE, "tile-wavefront partial rows changed under a cached plan");
  const int grid = std::max(1, std::min(cp->tw_ntiles, jit_tilewave_max_grid(t, c->num_sms)));
  CUDA_TRY(c, cudaMemsetAsync(cp->d_twprog, 0, sizeof(int) * (cp->tw_ntiles + 1), c->stream));
  rc = record_event(c);
  if (rc) return rc;
  const char* d = (const char*)cp->d_tw;
  TwArgs a;
  std::memset(&a, 0, sizeof a);
  a.loops = c->d_loops + dl_base;
  a.rng = (const int*)d;
  a.order = (const int*)(d + cp->tw_order);
  a.cls = (const int*)(d + cp->tw_cls);
  a.need = (const unsigned short*)(d + cp->tw_need);
  a.prog = cp->d_twprog;
  a.ticket = cp->d_twprog + cp->tw_ntiles;
  a.scal = env.scal;
  a.part = cp->d_twpart;
  a.err = env.err;
  a.timeout_ns = env.timeout_ns;
  for (int k = 0; k < 3; ++k) {
    a.nt[k] = P.ntiles[k];
    a.ncls[k] = cp->tw.ncls[k];
    a.roff[k] = cp->tw_roff[k];
    a.coff[k] = cp->tw_coff[k];
  }
  a.ntiles = cp->tw_ntiles;
  a.stride = cp->tw_ntiles;
  a.row0 = row0 < 0 ? 0 : row0;
  a.skip_tile = env.skip_block;
  a.pf = (const unsigned char*)(d + cp->tw_pf);
  a.ahead = jit_tile_ahead();
  a.groups = (const int*)(d + cp->tw_grp);
  a.ngroups = (int)cp->tw.groups.size() - 1;
  CUDA_TRY(c, jit_launch_tilewave(t, a, c->stream, grid));
  ++c->stats.launches;
  ++c->stats.kernel_launches;
  rc = record_event(c);
  if (rc) return rc;
  if (nrows) {
    CUDA_TRY(c, launch_fold_rows(env, cp->d_twpart, cp->tw_ntiles, row0, nrows, cp->tw_ntiles));
    ++c->stats.launches;
  }
  return OPS_OK;
}

// Grid of a compiled per-loop kernel over a box: by default one wave of the
// CTAs that stay resident (the kernel's occupancy x SMs), each striding over
// the box's units, so no partly filled last wave of CTAs idles SMs;
// OPSTILE_JIT_GRID = k caps the grid at k CTAs per SM instead.
int compiled_grid(ops_ctx c, JitSegment* js, int i, const LaunchEnv& env, const int* box) {
  const int units = untiled_grid(env, box);  // enumeration units, capped at 8 CTAs per SM
  const int k = jit_grid_policy();
  const int cap = k > 0 ? k * c->num_sms : jit_resident(js, i) * c->num_sms;
  int g = std::max(1, std::min(units, std::min(cap, c->part_stride)));
  const int64_t nx = box[1] - box[0];
  if (k == 0 && g < units && nx >= 128) {
    // a stride that shares a factor with the row's x-chunk count hands each
    // CTA the same chunks of every row (unequal when nx is not a multiple of
    // the chunk width): keep the stride coprime to it
    const int xch = (int)((nx + kThreads - 1) / kThreads);
    while (g > 1 && std::gcd(g, xch) != 1) --g;
  }
  return g;
}

// Execute a segment in a given mode; tile_in entries <= 0 are chosen automatically.
int run_segment_mode(ops_ctx c, int first, int count, int dl_base, std::vector<DLoop>& hl, int mode,
                     const int* tile_in) {
  const QLoop& q0 = c->queue[first];
  const int ndim = q0.dims;
  if (mode == OPS_MODE_OVERLAPPED) {
    // consecutive overlapped runs; what no run covers goes to the skewed path
    const int dl_first = first;
    std::vector<std::pair<int, OverlapPlan*>> runs;
    std::vector<std::vector<DLoop>> ols;
    while (count > 0) {
      OverlapPlan* op = nullptr;
      int used = 0;
      int rc = overlap_prefix(c, first, count, tile_in, &op, &used);
      if (rc) return rc;
      if (!used) break;
      runs.emplace_back(first, op);
      ols.push_back(overlap_descriptors(c, first, hl, op));
      first += used;
      dl_base += used;
      count -= used;
    }
    // compiled kernels of every run (compiled together, in parallel), else the interpreter's
    std::vector<JitOverlap*> jos(runs.size(), nullptr);
    if (!runs.empty() && !c->cfg.interpret && !c->cfg.check) {
      std::vector<OvRequest> reqs;
      for (size_t r = 0; r < runs.size(); ++r)
        reqs.push_back(OvRequest{ols[r].data(), runs[r].second->nloops, overlap_layout(runs[r].second, c->es)});
      std::string why;
      double ms = 0.0;
      int rc = jit_overlap_many(c->cfg.device, reqs, &jos, &why, &ms);
      c->stats.compile_ms += ms;
      if (rc) return fail(c, rc, "compiling overlapped tiles: %s", why.c_str());
    }
    for (size_t r = 0; r < runs.size(); ++r) {
      c->stats.mode = mode;
      int rc = run_overlap_plan(c, runs[r].first, hl, runs[r].second, ols[r], jos[r]);
      if (rc) return rc;
    }
    if (count == 0) return OPS_OK;
    if (first != dl_first) {
      // earlier runs moved written dats to their other buffers
      std::vector<FoldRow> unused;
      for (int k = first; k < first + count; ++k) {
        fill_dloop(c, c->queue[k], hl[k], hl[k].part_row, unused);
        if (k < (int)c->dev_ok.size()) c->dev_ok[k] = 0;
      }
      int rc = upload_loops(c, hl, first, count);
      if (rc) return rc;
    }
    mode = OPS_MODE_SKEWED;
    tile_in = c->cfg.tile;
  }
  if (mode == OPS_MODE_TILEWAVE || mode == OPS_MODE_TILEWARP) {
    // one loop has no dependencies to schedule; checked and interpreted runs,
    // runs without run-time compilation and chains no tile size suits go
    // through the skewed path
    const bool warp = mode == OPS_MODE_TILEWARP;
    if (count > 1 && !c->cfg.interpret && !c->cfg.check) {
      JitTile* t = nullptr;
      int rc = tile_code(c, first, count, hl, &t, warp);
      if (rc) return rc;
      if (t) {
        bool ran = false;
        rc = run_tilewave(c, first, count, dl_base, hl, tile_in, t, &ran, warp);
        if (rc || ran) return rc;
        tile_in = c->cfg.tile;
      }
    }
    mode = count > 1 ? OPS_MODE_SKEWED : OPS_MODE_UNTILED;
  }
  if (mode == OPS_MODE_WAVEFRONT) {
    // one loop has no dependencies to schedule; checked and interpreted
    // runs, and runs without run-time compilation, go through the skewed path
    if (count > 1 && !c->cfg.interpret && !c->cfg.check) {
      JitWave* w = nullptr;
      int rc = wave_code(c, first, count, hl, &w);
      if (rc) return rc;
      if (w) return run_wavefront(c, first, count, dl_base, hl, tile_in, w);
    }
    mode = count > 1 ? OPS_MODE_SKEWED : OPS_MODE_UNTILED;
  }
  LaunchEnv env = make_env(c);
  c->stats.mode = mode;
  ++c->stats.segments;
  c->stats.loops += count;
  JitSegment* js = nullptr;
  int rcj = segment_code(c, first, count, hl, &js);
  if (rcj) return rcj;
  c->stats.compiled = js ? 1 : 0;
  if (!js && c->es == 4)
    return fail(c, OPS_ERR_INVALID_ARG, "FP32 loops run compiled bodies only (no checked or interpreted mode%s%s)",
                c->jit_why.empty() ? "" : "; ", c->jit_why.c_str());
  if (mode == OPS_MODE_UNTILED || count == 1) {
    for (int i = 0; i < count; ++i) {
      const QLoop& q = c->queue[first + i];
      int box[6];
      for (int k = 0; k < 6; ++k) box[k] = q.rng[k];
      for (int d = q.dims; d < 3; ++d) {
        box[2 * d] = 0;
        box[2 * d + 1] = 1;
      }
      bool empty = false;
      int64_t n = 1;
      for (int d = 0; d < 3; ++d) {
        if (box[2 * d + 1] <= box[2 * d]) empty = true;
        n *= (int64_t)(box[2 * d + 1] - box[2 * d]);
      }
      const DLoop& L = hl[dl_base + i];
      if (empty) continue;
      c->stats.points += n;
      const int grid = js ? compiled_grid(c, js, i, env, box) : untiled_grid(env, box);
      int rc = record_event(c);
      if (rc) return rc;
      if (js)
        CUDA_TRY(c, jit_launch(js, i, env, c->d_loops + dl_base + i, box, grid, 1));
      else
        CUDA_TRY(c, launch_untiled(env, c->d_loops + dl_base + i, box, grid));
      rc = record_event(c);
      if (rc) return rc;
      ++c->stats.launches;
      ++c->stats.kernel_launches;
      if (L.nreds) {
        CUDA_TRY(c, launch_fold(env, L.part_row, L.nreds, grid));
        ++c->stats.launches;
      }
    }
    return OPS_OK;
  }
  // skewed: plan lookup by the loop sequence (ranges, dats, stencils, access)
  std::vector<PLoop> pl;
  pl.reserve(count);
  for (int i = 0; i < count; ++i) pl.push_back(plan_loop(c, c->queue[first + i]));
  int tile[3] = {tile_in[0], tile_in[1], tile_in[2]};
  if (tile[0] <= 0 || (ndim > 1 && tile[1] <= 0) || (ndim > 2 && tile[2] <= 0)) {
    int at[3];
    auto_tile(c, pl, ndim, at);
    for (int d = 0; d < 3; ++d)
      if (tile[d] <= 0) tile[d] = at[d];
  }
  std::vector<int> key;
  key.push_back(ndim);
  for (int d = 0; d < 3; ++d) key.push_back(tile[d]);
  for (int i = 0; i < count; ++i) {
    const QLoop& q = c->queue[first + i];
    for (int k = 0; k < 6; ++k) key.push_back(q.rng[k]);
    key.push_back((int)q.args.size());
    for (const ops_arg& a : q.args) {
      key.push_back(a.kind);
      key.push_back(a.handle);
      key.push_back(a.kind == OPS_ARG_DAT ? a.stencil : -1);
      key.push_back(a.access);
    }
  }
  CachedPlan* cp = nullptr;
  auto it = c->plans.find(key);
  if (it != c->plans.end()) {
    cp = it->second.get();
    ++c->stats.plan_cache_hits;
  } else {
    auto t0 = std::chrono::steady_clock::now();
    std::unique_ptr<CachedPlan> np(new CachedPlan);
    np->key = key;
    build_skewed_ranges(pl, (int)c->dats.size(), ndim, tile, np->plan);
    build_phases(pl, np->plan);
    auto t1 = std::chrono::steady_clock::now();
    c->stats.plan_ms += std::chrono::duration<double, std::milli>(t1 - t0).count();
    if (!np->plan.phases.empty()) {
      int rc = dev_alloc(c, (void**)&np->d_phases, sizeof(Phase) * np->plan.phases.size());
      if (rc) return rc;
      CUDA_TRY(c, cudaMemcpyAsync(np->d_phases, np->plan.phases.data(), sizeof(Phase) * np->plan.phases.size(),
                                  cudaMemcpyHostToDevice, c->stream));
      CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    }
    cp = np.get();
    c->plans[key] = std::move(np);
  }
  const SkewedPlan& P = cp->plan;
  int ntiles = 1;
  for (int d = 0; d < 3; ++d) {
    ntiles *= P.ntiles[d];
    c->stats.tile[d] = P.tile[d];
    c->stats.skew[d] = P.skew[d];
  }
  c->stats.tiles = ntiles;
  c->stats.phases += (int)P.phases.size();
  c->stats.barriers += P.nbarriers;
  c->stats.points += P.points;
  if (P.phases.empty()) return OPS_OK;
  int row0 = -1, nrows = 0;
  for (int i = 0; i < count; ++i) {
    const DLoop& L = hl[dl_base + i];
    if (L.nreds) {
      if (row0 < 0) row0 = L.part_row;
      nrows = L.part_row + L.nreds - row0;
    }
  }
  if (nrows) {
    CUDA_TRY(c, launch_part_init(env, row0, nrows));
    ++c->stats.launches;
  }
  int rc = record_event(c);
  if (rc) return rc;
  int sgrid = c->skewed_grid;
  JitSkew* sk = nullptr;
  if (js && count > 1 && c->cfg.skewed_persistent) {
    rc = skew_code(c, first, count, hl, &sk);
    if (rc) return rc;
  }
  if (sk) {
    // compiled bodies in one cooperative launch: grid barriers only where
    // the plan keeps them
    sgrid = std::max(1, std::min(jit_skewed_max_grid(sk, c->num_sms), c->part_stride));
    CUDA_TRY(c, jit_launch_skewed(sk, env, c->d_loops + dl_base, cp->d_phases, (int)P.phases.size(), sgrid));
    ++c->stats.launches;
    ++c->stats.kernel_launches;
  } else if (js) {
    // compiled bodies: one launch per phase in plan order; the stream
    // orders the phases as the persistent kernel's barriers do
    sgrid = 1;
    for (const Phase& ph : P.phases) {
      const int g = std::min(compiled_grid(c, js, ph.loop, env, ph.box), c->part_stride);
      sgrid = std::max(sgrid, g);
      CUDA_TRY(c, jit_launch(js, ph.loop, env, c->d_loops + dl_base + ph.loop, ph.box, g, 0));
      ++c->stats.launches;
      ++c->stats.kernel_launches;
    }
  } else {
    CUDA_TRY(c, launch_skewed(env, c->d_loops + dl_base, cp->d_phases, (int)P.phases.size(), sgrid));
    ++c->stats.launches;
    ++c->stats.kernel_launches;
  }
  rc = record_event(c);
  if (rc) return rc;
  if (nrows) {
    CUDA_TRY(c, launch_fold(env, row0, nrows, sgrid));
    ++c->stats.launches;
  }
  return OPS_OK;
}

// Signature of a segment: its loops' ranges and arguments (what a plan depends on).
std::vector<int> segment_signature(ops_ctx c, int first, int count) {
  std::vector<int> sig;
  sig.push_back(c->queue[first].dims);
  for (int i = 0; i < count; ++i) {
    const QLoop& q = c->queue[first + i];
    for (int k = 0; k < 6; ++k) sig.push_back(q.rng[k]);
    sig.push_back((int)q.args.size());
    for (const ops_arg& a : q.args) {
      sig.push_back(a.kind);
      sig.push_back(a.handle);
      sig.push_back(a.kind == OPS_ARG_DAT ? a.stencil : -1);
      sig.push_back(a.access);
    }
  }
  return sig;
}

// Autotuner (the paper picks tile sizes by a cache heuristic, Sec. 4.C; here
// the heuristic only seeds the search): every schedule of a segment gives
// bit-identical dats, so successive flushes of the same segment each run one
// candidate -- untiled, the tile wavefront at three tile shapes, skewed at
// the cache-fitting outer tile size and 4 times it, skewed on quarter-length
// sub-segments -- timed with CUDA events; afterwards the fastest candidate
// (mode, tile and segment length) is used for that segment.
int run_segment_auto(ops_ctx c, int first, int count, int dl_base, std::vector<DLoop>& hl) {
  const int ndim = c->queue[first].dims;
  TuneRec& T = c->tune[segment_signature(c, first, count)];
  if (T.cand.empty()) {
    std::vector<PLoop> pl;
    for (int i = 0; i < count; ++i) pl.push_back(plan_loop(c, c->queue[first + i]));
    int at[3];
    auto_tile(c, pl, ndim, at);
    int ext[3] = {1, 1, 1};
    for (int d = 0; d < 3; ++d) {
      int lo = 1 << 30, hi = -(1 << 30);
      for (const PLoop& p : pl) {
        lo = std::min(lo, p.rng[2 * d]);
        hi = std::max(hi, p.rng[2 * d + 1]);
      }
      ext[d] = std::max(1, hi - lo);
    }
    int od = 0;  // outermost dimension the seed tile cuts
    for (int d = ndim - 1; d >= 0; --d)
      if (at[d] < ext[d]) {
        od = d;
        break;
      }
    T.cand.push_back({OPS_MODE_UNTILED, 0, 0, 0, 0});
    // the tile wavefront with its automatic tiles and two other shapes
    // (run-time compiled, so only where NVRTC is there)
    if (count > 1 && !c->cfg.interpret && !c->cfg.check && jit_available()) {
      T.cand.push_back({OPS_MODE_TILEWAVE, 0, 0, 0, 0});
      if (ndim == 2) {
        // square tiles suit chains of few dats (the heat equation's Jacobi steps
        // ran fastest at 128 x 128 in FP32), wide ones chains of many
        T.cand.push_back({OPS_MODE_TILEWAVE, 128, 128, 0, 0});
        T.cand.push_back({OPS_MODE_TILEWAVE, 256, 64, 0, 0});
      } else if (ndim == 3) {
        T.cand.push_back({OPS_MODE_TILEWAVE, 64, 32, 32, 0});
      }
    }
    // Algorithm 2 with every CTA on one L2-sized tile, at the seed tile and 4x taller
    for (int f = 1; f <= 4; f *= 4) {
      std::array<int, 5> cd = {OPS_MODE_SKEWED, at[0], at[1], at[2], 0};
      cd[1 + od] = (int)std::min<int64_t>((int64_t)at[od] * f, ext[od]);
      T.cand.push_back(cd);
      if (cd[1 + od] >= ext[od]) break;
    }
    // the segment length too: long segments cut into quarters (at least 8
    // loops each), whose smaller skew keeps the seed tiles valid
    if (count >= 16) T.cand.push_back({OPS_MODE_SKEWED, at[0], at[1], at[2], std::max(8, count / 4)});
    // Overlapped tiles are not a candidate: on GB300 their redundant halo
    // work and one-CTA-per-SM footprints made them 4-10x slower than
    // untiled on every chain measured; OPS_MODE_OVERLAPPED still runs them.
    T.ms.assign(T.cand.size(), -1.0);
    T.runs.assign(T.cand.size(), 0);
    CUDA_TRY(c, cudaEventCreate(&T.e0));
    CUDA_TRY(c, cudaEventCreate(&T.e1));
  }
  if (T.pending >= 0) {
    float t = 0.f;
    CUDA_TRY(c, cudaEventSynchronize(T.e1));
    CUDA_TRY(c, cudaEventElapsedTime(&t, T.e0, T.e1));
    T.ms[T.pending] = T.ms[T.pending] < 0 ? t : std::min<double>(T.ms[T.pending], t);
    ++T.runs[T.pending];
    T.pending = -1;
  }
  int pick = T.best;
  if (pick < 0) {
    // round robin until every candidate has kTuneSamples samples; keep the best of each
    constexpr int kTuneSamples = 2;
    for (size_t i = 0; i < T.cand.size(); ++i)
      if (T.runs[i] < kTuneSamples && (pick < 0 || T.runs[i] < T.runs[pick])) pick = (int)i;
    if (pick < 0) {
      pick = 0;
      for (size_t i = 1; i < T.cand.size(); ++i)
        if (T.ms[i] < T.ms[pick]) pick = (int)i;
      T.best = pick;
    }
  }
  const bool tuning = T.best < 0;
  c->stats.tuning |= tuning ? 1 : 0;
  if (tuning) CUDA_TRY(c, cudaEventRecord(T.e0, c->stream));
  const std::array<int, 5>& cd = T.cand[pick];
  int rc = OPS_OK;
  const int part = cd[4] > 0 ? cd[4] : count;
  for (int f = 0; f < count && !rc; f += part)
    rc = run_segment_mode(c, first + f, std::min(part, count - f), dl_base + f, hl, cd[0], &cd[1]);
  if (rc) return rc;
  if (tuning) {
    CUDA_TRY(c, cudaEventRecord(T.e1, c->stream));
    T.pending = pick;
  }
  return OPS_OK;
}

int run_segment(ops_ctx c, int first, int count, int dl_base, std::vector<DLoop>& hl) {
  int mode = c->cfg.mode;
  if (mode == OPS_MODE_AUTO && count >= 2) return run_segment_auto(c, first, count, dl_base, hl);
  if (mode == OPS_MODE_AUTO) mode = OPS_MODE_UNTILED;
  return run_segment_mode(c, first, count, dl_base, hl, mode, c->cfg.tile);
}

// The first half of a flush: every queued loop's descriptor and partial
// rows, the device buffers they need, and the cuts into segments.
struct FlushPrep {
  explicit FlushPrep(ops_ctx c) : hl(c->hl_cache) {}
  std::vector<DLoop>& hl;  // the context's descriptor cache, filled for this flush
  std::vector<int> prow;
  std::vector<std::pair<int, int>> segs;  // (first loop, loop count)
  uint64_t filled_gen = 0;
};

// Two queued loops give the same descriptor up to its constants.
bool same_loop_shape(const QLoop& a, const QLoop& b) {
  return a.block == b.block && a.dims == b.dims && std::memcmp(a.rng, b.rng, sizeof a.rng) == 0 &&
         a.args.size() == b.args.size() &&
         (a.args.empty() || std::memcmp(a.args.data(), b.args.data(), sizeof(ops_arg) * a.args.size()) == 0) &&
         a.code == b.code && a.K.size() == b.K.size();
}

int flush_prepare(ops_ctx c, FlushPrep& F) {
  std::memset(&c->stats, 0, sizeof c->stats);
  c->ev_used = 0;
  if (c->host_only) return fail(c, OPS_ERR_NO_DEVICE, "host-only context cannot execute loops");
  const int n = (int)c->queue.size();
  if ((int)F.hl.size() < n) {
    F.hl.resize(n);
    c->hl_src.resize(n);
    c->hl_ok.resize(n, 0);
  }
  if (c->hl_gen != c->swap_gen) std::fill(c->hl_ok.begin(), c->hl_ok.end(), 0);
  F.prow.assign(n, 0);
  F.segs.clear();
  std::vector<FoldRow> rows;
  for (int i = 0; i < n; ++i) {
    F.prow[i] = (int)rows.size();
    const QLoop& q = c->queue[i];
    QLoop& src = c->hl_src[i];
    DLoop& L = F.hl[i];
    if (c->hl_ok[i] && L.part_row == F.prow[i] && same_loop_shape(src, q)) {
      if (src.K != q.K) {
        std::memcpy(L.K, q.K.data(), sizeof(double) * q.K.size());
        src.K = q.K;
        if (i < (int)c->dev_ok.size()) c->dev_ok[i] = 0;
      }
      for (const ops_arg& a : q.args)
        if (a.kind == OPS_ARG_RED) rows.push_back(FoldRow{a.handle, c->red_ops[a.handle]});
    } else {
      fill_dloop(c, q, L, F.prow[i], rows);
      src = q;
      c->hl_ok[i] = 1;
      if (i < (int)c->dev_ok.size()) c->dev_ok[i] = 0;
    }
  }
  c->hl_gen = c->swap_gen;
  F.filled_gen = c->swap_gen;
  const int cap0 = c->loops_cap;
  int rc = ensure(c, &c->d_loops, &c->loops_cap, n);
  if (rc) return rc;
  if (c->loops_cap != cap0) c->dev_ok.clear();  // new allocation: contents unknown
  // every descriptor at most once per segment and the fold rows
  rc = stage_begin(c, sizeof(DLoop) * (size_t)n + sizeof(FoldRow) * rows.size() + 64);
  if (rc) return rc;
  if (!rows.empty()) {
    const int rcap0 = c->rows_cap;
    rc = ensure(c, &c->d_rows, &c->rows_cap, (int)rows.size());
    if (rc) return rc;
    if (c->rows_cap != rcap0) c->rows_mirror.clear();
    if (c->rows_mirror.size() < rows.size() ||
        std::memcmp(c->rows_mirror.data(), rows.data(), sizeof(FoldRow) * rows.size()) != 0) {
      rc = stage_copy(c, c->d_rows, rows.data(), sizeof(FoldRow) * rows.size());
      if (rc) return rc;
      c->rows_mirror = rows;
    }
    int cap = c->part_rows_cap;
    if ((int)rows.size() > cap) {
      int want = std::max((int)rows.size(), 8);
      if (c->d_part) {
        cudaStreamSynchronize(c->stream);
        dev_free(c, c->d_part, sizeof(DD) * (size_t)c->part_rows_cap * c->part_stride);
        c->d_part = nullptr;
      }
      rc = dev_alloc(c, (void**)&c->d_part, sizeof(DD) * (size_t)want * c->part_stride);
      if (rc) return rc;
      c->part_rows_cap = want;
    }
  }
  // segments end where a loop reads (SCALAR) a reduction that an earlier loop
  // of the same segment reduces into: that is a dependency on every point
  int first = 0;
  const int seglim = c->cfg.segment > 0 ? c->cfg.segment : (1 << 30);
  std::vector<int> reduced;
  for (int i = 0; i <= n; ++i) {
    bool cut = i == n || i - first >= seglim;
    if (!cut) {
      for (const ops_arg& a : c->queue[i].args)
        if (a.kind == OPS_ARG_SCALAR && std::find(reduced.begin(), reduced.end(), a.handle) != reduced.end())
          cut = true;
      if (!cut && c->queue[i].dims != c->queue[first].dims) cut = true;
      if (!cut && c->queue[i].block != c->queue[first].block) cut = true;
    }
    if (cut && i > first) {
      F.segs.emplace_back(first, i - first);
      first = i;
      reduced.clear();
    }
    if (i < n)
      for (const ops_arg& a : c->queue[i].args)
        if (a.kind == OPS_ARG_RED) reduced.push_back(a.handle);
  }
  return OPS_OK;
}

// Descriptors of segment (first, count) on the device, refilled first if an
// earlier overlapped segment of this flush moved dats to their other buffers.
int segment_descriptors(ops_ctx c, FlushPrep& F, int first, int count) {
  if (c->swap_gen != F.filled_gen) {
    std::vector<FoldRow> unused;
    for (int k = first; k < first + count; ++k) {
      fill_dloop(c, c->queue[k], F.hl[k], F.prow[k], unused);
      if (k < (int)c->dev_ok.size()) c->dev_ok[k] = 0;
    }
  }
  return upload_loops(c, F.hl, first, count);
}

// After a flush: descriptors refilled mid-flush (dats moved to their other
// buffers) leave the cache at mixed generations, so none of it is reused.
void flush_done(ops_ctx c, const FlushPrep& F) {
  if (c->swap_gen != F.filled_gen) std::fill(c->hl_ok.begin(), c->hl_ok.end(), 0);
  c->queue.clear();
}

int flush(ops_ctx c) {
  if (c->queue.empty()) return OPS_OK;
  FlushPrep F(c);
  int rc = flush_prepare(c, F);
  if (rc) return rc;
  for (size_t s = 0; s < F.segs.size() && !rc; ++s) {
    const int first = F.segs[s].first, count = F.segs[s].second;
    rc = segment_descriptors(c, F, first, count);
    if (!rc) rc = run_segment(c, first, count, first, F.hl);
  }
  flush_done(c, F);
  return rc;
}

// ---------------------------------------------------------------------------
// batched execution: several contexts' chains, one launch per segment
// ---------------------------------------------------------------------------

// Make dst's stream wait for the work queued so far on src's stream.
int stream_after(ops_ctx dst, ops_ctx src) {
  if (dst->stream == src->stream) return OPS_OK;
  if (!src->ev_join) CUDA_TRY(src, cudaEventCreateWithFlags(&src->ev_join, cudaEventDisableTiming));
  CUDA_TRY(src, cudaEventRecord(src->ev_join, src->stream));
  CUDA_TRY(dst, cudaStreamWaitEvent(dst->stream, src->ev_join, 0));
  return OPS_OK;
}

// Run f(i) for i in [lo, hi): split over up to 8 host threads (each with
// the device current) when there are 16 contexts or more and each brings
// enough loops that the work outweighs starting the threads (16 x 256
// loop descriptors at least: 64 grids of an 83-loop chain are split, 64
// grids of an 8-loop chain are not, which measured slower split); else on
// the calling thread.  The contexts of a batch share no host state, and
// CUDA runtime calls are thread-safe.
template <class F>
void for_contexts(int device, int lo, int hi, int loops, F f) {
  const int n = hi - lo;
  const int nt = n >= 16 && (int64_t)n * loops >= 4096
                     ? std::min(8, std::max(1, (int)std::thread::hardware_concurrency()))
                     : 1;
  if (nt <= 1) {
    for (int i = lo; i < hi; ++i) f(i);
    return;
  }
  std::vector<std::thread> th;
  const int per = (n + nt - 1) / nt;
  for (int t = 0; t < nt; ++t) {
    const int a = lo + t * per, b = std::min(hi, a + per);
    if (a >= b) break;
    th.emplace_back([=, &f] {
      cudaSetDevice(device);
      for (int i = a; i < b; ++i) f(i);
    });
  }
  for (std::thread& t : th) t.join();
}

// The batch kernel of a segment (compiled once per code, like tile_code).
int tile_code_batch(ops_ctx c, int first, int count, const std::vector<DLoop>& hl, JitTile** out) {
  *out = nullptr;
  std::vector<int> key = code_key(c, first, count);
  key.push_back(-OPS_MODE_TILEWAVE);  // the batch form
  auto it = c->jitt.find(key);
  if (it != c->jitt.end()) {
    *out = it->second;
    return OPS_OK;
  }
  std::vector<std::vector<char>> ro = read_only_args(c, first, count);
  JitTile* t = nullptr;
  std::string why;
  double ms = 0.0;
  const int rc = jit_tilewave(c->cfg.device, hl.data() + first, count, ro, c->es, c->queue[first].dims, &t, &why,
                              &ms, true);
  c->stats.compile_ms += ms;
  if (rc) return fail(c, rc, "compiling the batch tile-wavefront kernel: %s", why.c_str());
  if (!t) c->jit_why = why;
  c->jitt[key] = t;
  *out = t;
  return OPS_OK;
}

// Segment (first, count) of every context of the batch in one launch of the
// tile-wavefront batch kernel, on cs[0]'s stream (which the caller has made
// wait for the others).  Tickets interleave the instances: the k-th tile in
// plan order of every instance comes before the (k+1)-th of any, so the
// instances advance together and each instance's tiles keep its plan order
// (what the waits of the tile wavefront rely on).  *ran = false when an
// instance has no valid plan or run-time compilation is unavailable.
int run_batch_tilewave(ops_ctx* cs, int n, std::vector<FlushPrep>& F, int first, int count, const int* tile_in,
                       bool* ran) {
  *ran = false;
  ops_ctx c0 = cs[0];
  // The instances' loops match in ranges, stencils, accesses and dats, so
  // the first context's plan is every instance's plan; only the progress
  // counters and the reduction partials are per instance.
  CachedPlan* p = nullptr;
  int rc = tile_plan(c0, first, count, F[0].hl, first, tile_in, &p);
  if (rc) return rc;
  if (!p) return OPS_OK;
  JitTile* t = nullptr;
  rc = tile_code_batch(c0, first, count, F[0].hl, &t);
  if (rc) return rc;
  if (!t) return OPS_OK;
  *ran = true;
  int row0 = -1, nrows = 0;
  for (int l = 0; l < count; ++l) {
    const DLoop& L = F[0].hl[first + l];
    if (L.nreds) {
      if (row0 < 0) row0 = L.part_row;
      nrows = L.part_row + L.nreds - row0;
    }
  }
  if (nrows > p->tw_rows) return fail(c0, OPS_ERR_STATE, "tile-wavefront partial rows changed under a cached plan");
  const int nt = p->tw_ntiles;
  const int64_t total64 = (int64_t)nt * n;
  if (total64 >= (1 << 30)) return fail(c0, OPS_ERR_INVALID_ARG, "a batch of %lld tiles is too large", (long long)total64);
  const int total = (int)total64;
  // device tables: arguments | fold instances | ticket map | partials | progress + ticket
  const size_t b_args = sizeof(TwArgs) * n, b_fold = sizeof(FoldInst) * n, b_map = sizeof(int) * 2 * (size_t)total,
               b_part = sizeof(DD) * (size_t)nrows * total, b_prog = sizeof(int) * ((size_t)total + 1);
  const size_t o_fold = (b_args + 15) / 16 * 16, o_map = o_fold + (b_fold + 15) / 16 * 16,
               o_part = o_map + (b_map + 15) / 16 * 16, o_prog = o_part + (b_part + 15) / 16 * 16,
               bytes = o_prog + b_prog;
  if (bytes > c0->batch_cap) {
    if (c0->d_batch) {
      CUDA_TRY(c0, cudaStreamSynchronize(c0->stream));
      dev_free(c0, c0->d_batch, c0->batch_cap);
      c0->d_batch = nullptr;
      c0->batch_cap = 0;
    }
    const size_t want = std::max<size_t>(bytes, 4096);
    rc = dev_alloc(c0, &c0->d_batch, want);
    if (rc) return rc;
    c0->batch_cap = want;
  }
  char* d = (char*)c0->d_batch;
  int* d_prog = (int*)(d + o_prog);
  DD* d_part = (DD*)(d + o_part);
  std::vector<char> host(o_part, 0);
  TwArgs* ha = (TwArgs*)host.data();
  FoldInst* hf = (FoldInst*)(host.data() + o_fold);
  int* hm = (int*)(host.data() + o_map);
  const LaunchEnv env0 = make_env(c0);
  const char* dt = (const char*)p->d_tw;
  for (int i = 0; i < n; ++i) {
    ops_ctx c = cs[i];
    TwArgs& a = ha[i];
    std::memset(&a, 0, sizeof a);
    a.loops = c->d_loops + first;
    a.rng = (const int*)dt;
    a.order = (const int*)(dt + p->tw_order);
    a.cls = (const int*)(dt + p->tw_cls);
    a.need = (const unsigned short*)(dt + p->tw_need);
    a.prog = d_prog + (size_t)i * nt;
    a.ticket = d_prog + total;
    a.scal = c->d_scal;
    a.part = d_part + (size_t)i * nrows * nt;
    a.err = env0.err;
    a.timeout_ns = env0.timeout_ns;
    for (int k = 0; k < 3; ++k) {
      a.nt[k] = p->plan.ntiles[k];
      a.ncls[k] = p->tw.ncls[k];
      a.roff[k] = p->tw_roff[k];
      a.coff[k] = p->tw_coff[k];
    }
    a.ntiles = nt;
    a.stride = nt;
    a.row0 = row0 < 0 ? 0 : row0;
    a.skip_tile = i == 0 ? env0.skip_block : -1;
    a.pf = (const unsigned char*)(dt + p->tw_pf);
    a.ahead = jit_tile_ahead();
    a.groups = (const int*)(dt + p->tw_grp);
    a.ngroups = (int)p->tw.groups.size() - 1;
    hf[i] = FoldInst{a.part, c->d_rows, c->d_scal, nt, nt};
  }
  for (int k = 0, q = 0; k < nt; ++k)
    for (int i = 0; i < n; ++i, ++q) {
      hm[2 * q] = i;
      hm[2 * q + 1] = p->tw.order[k];
    }
  rc = stage_copy(c0, d, host.data(), o_map + b_map);
  if (rc) return rc;
  CUDA_TRY(c0, cudaMemsetAsync(d_prog, 0, b_prog, c0->stream));
  const int grid = std::max(1, std::min(total, jit_tilewave_max_grid(t, c0->num_sms)));
  rc = record_event(c0);
  if (rc) return rc;
  CUDA_TRY(c0, jit_launch_tilewave_batch(t, (const TwArgs*)d, (const int*)(d + o_map), total, d_prog + total,
                                         c0->stream, grid));
  rc = record_event(c0);
  if (rc) return rc;
  if (nrows) CUDA_TRY(c0, launch_fold_batch(c0->stream, (const FoldInst*)(d + o_fold), n, row0, nrows, row0, 0));
  for (int i = 0; i < n; ++i) {
    ops_ctx c = cs[i];
    c->stats.mode = OPS_MODE_TILEWAVE;
    c->stats.compiled = 1;
    c->stats.batched = n;
    ++c->stats.segments;
    c->stats.loops += count;
    for (int k = 0; k < 3; ++k) {
      c->stats.tile[k] = p->plan.tile[k];
      c->stats.skew[k] = p->plan.skew[k];
    }
    c->stats.tiles = p->tw_ntiles;
    c->stats.phases += p->tw_phases;
    c->stats.barriers += p->tw_steps;
  }
  ++c0->stats.launches;
  ++c0->stats.kernel_launches;
  if (nrows) ++c0->stats.launches;
  return OPS_OK;
}

// The batch form of a segment's per-loop kernels (compiled once per code).
int segment_code_batch(ops_ctx c, int first, int count, const std::vector<DLoop>& hl, JitSegment** out) {
  *out = nullptr;
  if (c->cfg.interpret || c->cfg.check) return OPS_OK;
  std::vector<int> key = code_key(c, first, count);
  key.push_back(-OPS_MODE_UNTILED - 100);  // the batch form
  auto it = c->jit.find(key);
  if (it != c->jit.end()) {
    *out = it->second;
    return OPS_OK;
  }
  std::vector<std::vector<char>> ro = read_only_args(c, first, count);
  JitSegment* js = nullptr;
  std::string why;
  double ms = 0.0;
  const int rc = jit_segment(c->cfg.device, hl.data() + first, count, ro, c->es, &js, &why, &ms, true);
  c->stats.compile_ms += ms;
  if (rc) return fail(c, rc, "compiling the batch loop kernels: %s", why.c_str());
  if (!js) c->jit_why = why;
  c->jit[key] = js;
  *out = js;
  return OPS_OK;
}

// Segment (first, count) of every context of the batch untiled, one launch
// per loop for all instances (blockIdx.y = instance), on cs[0]'s stream:
// the loops run in program order as in the untiled form, each instance's
// reductions fold from its own partials, all instances' in one launch.
// *ran = false without run-time compilation.
int run_batch_untiled(ops_ctx* cs, int n, std::vector<FlushPrep>& F, int first, int count, bool* ran) {
  *ran = false;
  ops_ctx c0 = cs[0];
  JitSegment* js = nullptr;
  int rc = segment_code_batch(c0, first, count, F[0].hl, &js);
  if (rc) return rc;
  if (!js) return OPS_OK;
  *ran = true;
  const LaunchEnv env0 = make_env(c0);
  // per loop: its box and the CTAs per instance (one wave of the resident
  // CTAs shared by the instances, at most one CTA per enumeration unit)
  std::vector<std::array<int, 6>> boxes(count);
  std::vector<int> grid(count, 0);
  int stride = 1, rows = 0;
  for (int i = 0; i < count; ++i) {
    const QLoop& q = c0->queue[first + i];
    std::array<int, 6>& box = boxes[i];
    for (int k = 0; k < 6; ++k) box[k] = q.rng[k];
    for (int d = q.dims; d < 3; ++d) {
      box[2 * d] = 0;
      box[2 * d + 1] = 1;
    }
    bool empty = false;
    for (int d = 0; d < 3; ++d) empty = empty || box[2 * d + 1] <= box[2 * d];
    if (empty) continue;
    const int units = untiled_grid(env0, box.data());
    const int cap = std::max(1, jit_resident(js, i) * c0->num_sms / n);
    grid[i] = std::max(1, std::min(units, cap));
    stride = std::max(stride, grid[i]);
    const DLoop& L = F[0].hl[first + i];
    if (L.nreds) rows = std::max(rows, L.part_row + L.nreds);
  }
  // device tables: instances | fold instances | partials
  const size_t b_inst = sizeof(BatchInst) * n, b_fold = sizeof(FoldInst) * n,
               b_part = sizeof(DD) * (size_t)rows * stride * n;
  const size_t o_fold = (b_inst + 15) / 16 * 16, o_part = o_fold + (b_fold + 15) / 16 * 16, bytes = o_part + b_part;
  if (bytes > c0->batch_cap) {
    if (c0->d_batch) {
      CUDA_TRY(c0, cudaStreamSynchronize(c0->stream));
      dev_free(c0, c0->d_batch, c0->batch_cap);
      c0->d_batch = nullptr;
      c0->batch_cap = 0;
    }
    const size_t want = std::max<size_t>(bytes, 4096);
    rc = dev_alloc(c0, &c0->d_batch, want);
    if (rc) return rc;
    c0->batch_cap = want;
  }
  char* d = (char*)c0->d_batch;
  DD* d_part = (DD*)(d + o_part);
  std::vector<char> host(o_part, 0);
  BatchInst* hb = (BatchInst*)host.data();
  FoldInst* hf = (FoldInst*)(host.data() + o_fold);
  for (int k = 0; k < n; ++k) {
    DD* part = d_part + (size_t)k * rows * stride;
    hb[k] = BatchInst{cs[k]->d_loops + first, cs[k]->d_scal, part};
    hf[k] = FoldInst{part, cs[k]->d_rows, cs[k]->d_scal, stride, 0};
  }
  rc = stage_copy(c0, d, host.data(), host.size());
  if (rc) return rc;
  int launches = 0, kernels = 0;
  int64_t pts = 0;
  for (int i = 0; i < count; ++i) {
    if (!grid[i]) continue;
    const std::array<int, 6>& box = boxes[i];
    pts += (int64_t)(box[1] - box[0]) * (box[3] - box[2]) * (box[5] - box[4]);
    rc = record_event(c0);
    if (rc) return rc;
    CUDA_TRY(c0, jit_launch_batch(js, i, c0->stream, (const BatchInst*)d, n, box.data(), grid[i], stride));
    rc = record_event(c0);
    if (rc) return rc;
    ++launches;
    ++kernels;
    const DLoop& L = F[0].hl[first + i];
    if (L.nreds) {
      CUDA_TRY(c0, launch_fold_batch(c0->stream, (const FoldInst*)(d + o_fold), n, L.part_row, L.nreds, 0,
                                     grid[i]));
      ++launches;
    }
  }
  for (int k = 0; k < n; ++k) {
    ops_ctx c = cs[k];
    c->stats.mode = OPS_MODE_UNTILED;
    c->stats.compiled = 1;
    c->stats.batched = n;
    c->stats.loops += count;
    c->stats.points += pts;
  }
  c0->stats.launches += launches;
  c0->stats.kernel_launches += kernels;
  return OPS_OK;
}

// Run segment (first, count) of every context of the batch, in the batch
// candidate cd (mode, tile): untiled or the tile wavefront in launches
// shared by all instances, or each context on its own stream in any other
// mode cd[0].  On return cs[0]'s stream has the whole segment queued.
int run_batch_candidate(ops_ctx* cs, int n, std::vector<FlushPrep>& F, int first, int count,
                        const std::array<int, 5>& cd) {
  ops_ctx c0 = cs[0];
  if (cd[0] == OPS_MODE_TILEWAVE && count > 1) {
    bool ran = false;
    int rc = run_batch_tilewave(cs, n, F, first, count, &cd[1], &ran);
    if (rc || ran) return rc;
  }
  if (cd[0] == OPS_MODE_TILEWAVE || cd[0] == OPS_MODE_UNTILED || cd[0] == OPS_MODE_AUTO) {
    bool ran = false;
    int rc = run_batch_untiled(cs, n, F, first, count, &ran);
    if (rc || ran) return rc;
  }
  const int mode = cd[0] == OPS_MODE_TILEWAVE || cd[0] == OPS_MODE_AUTO ? OPS_MODE_UNTILED : cd[0];
  for (int i = 1; i < n; ++i) {
    int rc = stream_after(cs[i], c0);
    if (rc) return rc;
  }
  for (int i = 0; i < n; ++i) {
    int rc = run_segment_mode(cs[i], first, count, first, F[i].hl, mode, &cd[1]);
    if (rc) return rc;
  }
  for (int i = 1; i < n; ++i) {
    int rc = stream_after(c0, cs[i]);
    if (rc) return rc;
  }
  return OPS_OK;
}

// Candidates of the batch autotuner: untiled with one launch per loop for
// all instances; the tile wavefront with its automatic tiles, with the
// whole grid as one tile (each CTA then runs a whole instance's chain, no
// waits), and with tiles of half the automatic size in y (more tiles per
// instance for few instances).
std::vector<std::array<int, 5>> batch_candidates(ops_ctx c, int first, int count) {
  std::vector<std::array<int, 5>> cand;
  cand.push_back({OPS_MODE_UNTILED, 0, 0, 0, 0});
  if (count < 2 || c->cfg.interpret || c->cfg.check || !jit_available()) return cand;
  const int ndim = c->queue[first].dims;
  std::vector<PLoop> pl;
  for (int i = 0; i < count; ++i) pl.push_back(plan_loop(c, c->queue[first + i]));
  int at[3];
  auto_tile_wave(c, pl, ndim, at);
  cand.push_back({OPS_MODE_TILEWAVE, 0, 0, 0, 0});
  cand.push_back({OPS_MODE_TILEWAVE, 1 << 20, ndim > 1 ? 1 << 20 : 1, ndim > 2 ? 1 << 20 : 1, 0});
  if (ndim >= 2 && at[1] >= 16) cand.push_back({OPS_MODE_TILEWAVE, at[0], at[1] / 2, ndim > 2 ? at[2] : 1, 0});
  return cand;
}

// One segment of the batch: the candidate of the context's mode, or under
// OPS_MODE_AUTO the autotuner's pick (each candidate timed on cs[0]'s
// stream twice, then the fastest kept for this signature and batch size).
int run_batch_segment(ops_ctx* cs, int n, std::vector<FlushPrep>& F, int first, int count) {
  ops_ctx c0 = cs[0];
  std::vector<int> drc(n, 0);
  for_contexts(c0->cfg.device, 1, n, count, [&](int i) { drc[i] = segment_descriptors(cs[i], F[i], first, count); });
  for (int i = 1; i < n; ++i) {
    int rc = drc[i] ? fail(c0, drc[i], "context %d of the batch: %s", i, cs[i]->err.c_str()) : stream_after(c0, cs[i]);
    if (rc) return rc;
  }
  int rc = segment_descriptors(c0, F[0], first, count);
  if (rc) return rc;
  const int mode = c0->cfg.mode;
  if (mode != OPS_MODE_AUTO) {
    std::array<int, 5> cd = {mode, c0->cfg.tile[0], c0->cfg.tile[1], c0->cfg.tile[2], 0};
    return run_batch_candidate(cs, n, F, first, count, cd);
  }
  std::vector<int> key = segment_signature(c0, first, count);
  key.push_back(-1);
  key.push_back(n);
  TuneRec& T = c0->btune[key];
  if (T.cand.empty()) {
    T.cand = batch_candidates(c0, first, count);
    T.ms.assign(T.cand.size(), -1.0);
    T.runs.assign(T.cand.size(), 0);
    CUDA_TRY(c0, cudaEventCreate(&T.e0));
    CUDA_TRY(c0, cudaEventCreate(&T.e1));
  }
  if (T.pending >= 0) {
    float t = 0.f;
    CUDA_TRY(c0, cudaEventSynchronize(T.e1));
    CUDA_TRY(c0, cudaEventElapsedTime(&t, T.e0, T.e1));
    T.ms[T.pending] = T.ms[T.pending] < 0 ? t : std::min<double>(T.ms[T.pending], t);
    ++T.runs[T.pending];
    T.pending = -1;
  }
  int pick = T.best;
  if (pick < 0) {
    constexpr int kTuneSamples = 2;
    for (size_t i = 0; i < T.cand.size(); ++i)
      if (T.runs[i] < kTuneSamples && (pick < 0 || T.runs[i] < T.runs[pick])) pick = (int)i;
    if (pick < 0) {
      pick = 0;
      for (size_t i = 1; i < T.cand.size(); ++i)
        if (T.ms[i] < T.ms[pick]) pick = (int)i;
      T.best = pick;
    }
  }
  const bool tuning = T.best < 0;
  if (tuning) CUDA_TRY(c0, cudaEventRecord(T.e0, c0->stream));
  rc = run_batch_candidate(cs, n, F, first, count, T.cand[pick]);
  if (rc) return rc;
  for (int i = 0; i < n; ++i) cs[i]->stats.tuning |= tuning ? 1 : 0;
  if (tuning) {
    CUDA_TRY(c0, cudaEventRecord(T.e1, c0->stream));
    T.pending = pick;
  }
  return OPS_OK;
}

// Two descriptors agree in everything the generated code depends on: all
// but the dats' addresses and the constants (which the kernels load).
bool same_descriptor(const DLoop& a, const DLoop& b) {
  if (std::memcmp(&a, &b, offsetof(DLoop, ins)) != 0) return false;
  if (std::memcmp(a.ins, b.ins, sizeof(a.ins[0]) * a.nins) != 0) return false;
  for (int k = 0; k < a.nargs; ++k) {
    const DArg &x = a.args[k], &y = b.args[k];
    const size_t from = offsetof(DArg, pitch), to = offsetof(DArg, off) + sizeof(int32_t) * x.npts;
    if (x.npts != y.npts || std::memcmp((const char*)&x + from, (const char*)&y + from, to - from) != 0) return false;
  }
  return true;
}

// 0 when loop by loop ctx c's queued chain matches the first context's in
// everything but the dats' addresses and the loops' constants, else the
// index of the first loop that does not, plus one.
int batch_mismatch(ops_ctx c0, const FlushPrep& F0, ops_ctx c, const FlushPrep& F) {
  const int nloops = (int)c0->queue.size();
  if (F.segs != F0.segs) return 1;
  for (int l = 0; l < nloops; ++l) {
    const QLoop &q0 = c0->queue[l], &qi = c->queue[l];
    bool same = same_descriptor(F0.hl[l], F.hl[l]) && q0.dims == qi.dims && q0.code == qi.code &&
                q0.args.size() == qi.args.size();
    for (size_t k = 0; same && k < q0.args.size(); ++k)
      same = q0.args[k].kind == qi.args[k].kind && q0.args[k].handle == qi.args[k].handle &&
             q0.args[k].stencil == qi.args[k].stencil && q0.args[k].access == qi.args[k].access;
    if (!same) return l + 1;
  }
  return 0;
}

int execute_batch(ops_ctx* cs, int n) {
  ops_ctx c0 = cs[0];
  const int nloops = (int)c0->queue.size();
  for (int i = 0; i < n; ++i) {
    ops_ctx c = cs[i];
    if (c->host_only) return fail(c0, OPS_ERR_NO_DEVICE, "host-only context %d in the batch", i);
    if (c->cfg.device != c0->cfg.device || c->es != c0->es)
      return fail(c0, OPS_ERR_INVALID_ARG, "context %d of the batch has another device or precision", i);
    if ((int)c->queue.size() != nloops)
      return fail(c0, OPS_ERR_INVALID_ARG, "context %d queued %d loops, the first %d", i, (int)c->queue.size(),
                  nloops);
    for (int j = 0; j < i; ++j)
      if (cs[j] == c) return fail(c0, OPS_ERR_INVALID_ARG, "context %d appears twice in the batch", i);
  }
  if (nloops == 0) return OPS_OK;
  std::vector<FlushPrep> F;
  F.reserve(n);
  for (int i = 0; i < n; ++i) F.emplace_back(cs[i]);
  int rc = flush_prepare(c0, F[0]);
  if (rc) return rc;
  // The other contexts' descriptors (in parallel for large batches), each
  // checked against the first context's: the chains must match loop for
  // loop in everything but the dats' addresses, so the same code serves
  // every instance.  Nothing has run yet when they do not, and every queue
  // is kept.
  std::vector<int> prc(n, 0), mism(n, 0);
  for_contexts(c0->cfg.device, 1, n, nloops, [&](int i) {
    prc[i] = flush_prepare(cs[i], F[i]);
    if (!prc[i]) mism[i] = batch_mismatch(c0, F[0], cs[i], F[i]);
  });
  for (int i = 1; i < n; ++i) {
    if (prc[i]) return fail(c0, prc[i], "context %d of the batch: %s", i, cs[i]->err.c_str());
    if (mism[i])
      return fail(c0, OPS_ERR_INVALID_ARG,
                  "loop %d of context %d differs from the first context's in more than its dats' addresses "
                  "and constants (or the chain is cut into other segments)", mism[i] - 1, i);
  }
  for (size_t s = 0; s < F[0].segs.size() && !rc; ++s)
    rc = run_batch_segment(cs, n, F, F[0].segs[s].first, F[0].segs[s].second);
  // the other contexts' later work follows the batch
  for (int i = 1; i < n && !rc; ++i) rc = stream_after(cs[i], c0);
  for (int i = 0; i < n; ++i) flush_done(cs[i], F[i]);
  return rc;
}

int check_device_error(ops_ctx c) {
  int h = 0;
  CUDA_TRY(c, cudaMemcpyAsync(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (h) {
    CUDA_TRY(c, cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
    if (h == kDevErrTimeout)
      return fail(c, OPS_ERR_TIMEOUT, "a device-side wait exceeded %d ms", c->cfg.timeout_ms > 0 ? c->cfg.timeout_ms : 2000);
    return fail(c, OPS_ERR_DEVICE_BOUNDS, "a kernel caught an out-of-range access (checked mode)");
  }
  return OPS_OK;
}

}  // namespace

// ===========================================================================
// context services for cg.cu and serve.cpp
// ===========================================================================
namespace opstile {
cudaStream_t ctx_stream(ops_ctx c) { return c->stream; }
int ctx_num_sms(ops_ctx c) { return c->num_sms; }
bool ctx_host_only(ops_ctx c) { return c->host_only; }
int ctx_alloc(ops_ctx c, void** p, size_t bytes) { return dev_alloc(c, p, bytes); }
void ctx_free(ops_ctx c, void* p, size_t bytes) { dev_free(c, p, bytes); }
int ctx_fail(ops_ctx c, int code, const char* msg) { return fail(c, code, "%s", msg); }
}  // namespace opstile

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void ops_config_default(ops_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof *cfg);
  cfg->device = 0;
  cfg->mode = OPS_MODE_AUTO;
  cfg->timeout_ms = 2000;
  cfg->test_skip_barrier_block = -1;
}

int ops_init(ops_ctx* out, const ops_config* cfg) {
  if (!out) return OPS_ERR_INVALID_ARG;
  *out = nullptr;
  std::unique_ptr<ops_ctx_s> c(new ops_ctx_s);
  if (cfg) c->cfg = *cfg;
  else ops_config_default(&c->cfg);
  if (c->cfg.real != OPS_REAL_F64 && c->cfg.real != OPS_REAL_F32) return OPS_ERR_INVALID_ARG;
  c->es = c->cfg.real == OPS_REAL_F32 ? 4 : 8;
  std::memset(&c->stats, 0, sizeof c->stats);
  if (c->cfg.device < 0) {  // host-only: declarations, validation and planning
    c->host_only = true;
    *out = c.release();
    return OPS_OK;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || c->cfg.device >= ndev) {
    cudaGetLastError();
    return OPS_ERR_NO_DEVICE;
  }
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, c->cfg.device) != cudaSuccess) return OPS_ERR_NO_DEVICE;
  if (prop.major != 10 || prop.minor != 3) return OPS_ERR_NO_DEVICE;
  if (cudaSetDevice(c->cfg.device) != cudaSuccess) return OPS_ERR_NO_DEVICE;
  c->num_sms = prop.multiProcessorCount;
  c->l2_size = prop.l2CacheSize;
  ops_ctx cp = c.get();
  if (c->cfg.stream) {
    c->stream = (cudaStream_t)c->cfg.stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) return OPS_ERR_CUDA;
    c->own_stream = true;
  }
  int rc = dev_alloc(cp, (void**)&c->d_err, sizeof(int));
  if (!rc) rc = dev_alloc(cp, (void**)&c->d_bar, 4 * sizeof(unsigned));
  if (rc) return rc;
  cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream);
  cudaMemsetAsync(c->d_bar, 0, 4 * sizeof(unsigned), c->stream);
  if (chain_kernels_setup() != cudaSuccess) return OPS_ERR_CUDA;
  c->skewed_grid = skewed_max_grid(c->num_sms, c->cfg.blocks_per_sm);
  c->part_stride = std::max(c->skewed_grid, c->num_sms * 8);
  if (c->skewed_grid <= 0) return OPS_ERR_CUDA;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return OPS_ERR_CUDA;
  *out = c.release();
  return OPS_OK;
}

int ops_finalize(ops_ctx c) {
  if (!c) return OPS_ERR_INVALID_ARG;
  if (!c->host_only) {
    cudaStreamSynchronize(c->stream);
    for (Dat& d : c->dats) {
      dev_free(c, d.alloc, d.bytes);
      dev_free(c, d.alt, d.bytes);
    }
    for (auto& kv : c->plans) {
      if (!kv.second) continue;  // a tile-wavefront plan no tile size suits
      if (kv.second->d_phases) dev_free(c, kv.second->d_phases, sizeof(Phase) * kv.second->plan.phases.size());
      if (kv.second->d_wave) dev_free(c, kv.second->d_wave, kv.second->wave_bytes);
      if (kv.second->d_wdone) dev_free(c, kv.second->d_wdone, sizeof(int) * (kv.second->plan.phases.size() + 1));
      if (kv.second->d_tw) dev_free(c, kv.second->d_tw, kv.second->tw_bytes);
      if (kv.second->d_twprog) dev_free(c, kv.second->d_twprog, sizeof(int) * (kv.second->tw_ntiles + 1));
      if (kv.second->d_twpart)
        dev_free(c, kv.second->d_twpart, sizeof(DD) * (size_t)kv.second->tw_rows * kv.second->tw_ntiles);
    }
    for (auto& kv : c->oplans)
      if (kv.second && kv.second->d_tab) dev_free(c, kv.second->d_tab, sizeof(int) * kv.second->tab_ints);
    dev_free(c, c->d_oloops, sizeof(DLoop) * (size_t)c->oloops_cap);
    dev_free(c, c->d_ovdat, sizeof(OvDat) * (size_t)c->ovdat_cap);
    dev_free(c, c->d_scal, sizeof(double) * (size_t)c->scal_cap);
    dev_free(c, c->d_part, sizeof(DD) * (size_t)c->part_rows_cap * c->part_stride);
    dev_free(c, c->d_rows, sizeof(FoldRow) * (size_t)c->rows_cap);
    dev_free(c, c->d_loops, sizeof(DLoop) * (size_t)c->loops_cap);
    dev_free(c, c->d_err, sizeof(int));
    dev_free(c, c->d_bar, 4 * sizeof(unsigned));
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    for (auto* tm : {&c->tune, &c->btune})
      for (auto& kv : *tm) {
        if (kv.second.e0) cudaEventDestroy(kv.second.e0);
        if (kv.second.e1) cudaEventDestroy(kv.second.e1);
      }
    dev_free(c, c->d_batch, c->batch_cap);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    for (int k = 0; k < 2; ++k) {
      if (c->ev_stage[k]) cudaEventDestroy(c->ev_stage[k]);
      if (c->h_stage[k]) cudaFreeHost(c->h_stage[k]);
    }
    if (c->h_small) cudaFreeHost(c->h_small);
    if (c->own_stream) cudaStreamDestroy(c->stream);
  }
  delete c;
  return OPS_OK;
}

const char* ops_last_error(ops_ctx c) { return c ? c->err.c_str() : "null context"; }

int ops_set_timing(ops_ctx c, int timing) {
  if (!c) return OPS_ERR_INVALID_ARG;
  c->cfg.timing = timing ? 1 : 0;
  return OPS_OK;
}

int ops_set_mode(ops_ctx c, int mode, const int* tile, int segment) {
  if (!c) return OPS_ERR_INVALID_ARG;
  if (mode < OPS_MODE_UNTILED || mode > OPS_MODE_TILEWARP) return fail(c, OPS_ERR_INVALID_ARG, "bad mode %d", mode);
  c->cfg.mode = mode;
  if (tile)
    for (int d = 0; d < 3; ++d) c->cfg.tile[d] = tile[d];
  c->cfg.segment = segment;
  return OPS_OK;
}

int ops_decl_block(ops_ctx c, int dims, const char* name, int* out) {
  if (!c || !out) return OPS_ERR_INVALID_ARG;
  if (dims < 1 || dims > 3) return fail(c, OPS_ERR_INVALID_ARG, "block dims must be 1..3 (got %d)", dims);
  c->blocks.push_back(Block{dims, name ? name : ""});
  *out = (int)c->blocks.size() - 1;
  return OPS_OK;
}

int ops_decl_dat(ops_ctx c, int block, const int size[3], const int d_m[3], const int d_p[3], double* dev_ptr0,
                 int64_t pitch, int64_t plane, const char* name, int* out) {
  if (!c || !out || !size || !d_m || !d_p) return OPS_ERR_INVALID_ARG;
  if (block < 0 || block >= (int)c->blocks.size()) return fail(c, OPS_ERR_INVALID_ARG, "bad block %d", block);
  const int dims = c->blocks[block].dims;
  Dat D;
  D.block = block;
  D.name = name ? name : "";
  for (int d = 0; d < 3; ++d) {
    D.size[d] = d < dims ? size[d] : 1;
    D.dm[d] = d < dims ? d_m[d] : 0;
    D.dp[d] = d < dims ? d_p[d] : 0;
    if (D.size[d] < 1 || D.dm[d] < 0 || D.dp[d] < 0)
      return fail(c, OPS_ERR_INVALID_ARG, "dat '%s': bad size/halo in dim %d", D.name.c_str(), d);
    D.ext[d] = D.size[d] + D.dm[d] + D.dp[d];
  }
  if (dev_ptr0) {
    if (pitch < D.ext[0] || plane < pitch * (D.ext[1] > 1 ? 1 : 0))
      return fail(c, OPS_ERR_INVALID_ARG, "dat '%s': pitch/plane too small", D.name.c_str());
    D.ptr0 = dev_ptr0;
    D.pitch = pitch;
    D.plane = plane;
  } else {
    // point x = 0 starts a 128-byte line: pad the row front to a whole
    // number of lines, and the row to whole lines
    const int64_t line = 128 / c->es;
    const int64_t xo = (D.dm[0] + line - 1) / line * line;
    D.pitch = (xo + D.size[0] + D.dp[0] + line - 1) / line * line;
    D.plane = D.pitch * D.ext[1];
    D.bytes = (size_t)c->es * (size_t)(D.plane * D.ext[2]);
    if (!c->host_only) {
      int rc = dev_alloc(c, (void**)&D.alloc, D.bytes);
      if (rc) return rc;
      CUDA_TRY(c, cudaMemsetAsync(D.alloc, 0, D.bytes, c->stream));
      D.ptr0 = elem_at(D.alloc, xo + D.pitch * D.dm[1] + D.plane * D.dm[2], c->es);
    }
  }
  c->dats.push_back(D);
  *out = (int)c->dats.size() - 1;
  return OPS_OK;
}

int ops_decl_stencil(ops_ctx c, int dims, int npts, const int* offsets, const char* name, int* out) {
  if (!c || !out || !offsets) return OPS_ERR_INVALID_ARG;
  if (dims < 1 || dims > 3 || npts < 1 || npts > OPS_MAX_STENCIL_POINTS)
    return fail(c, OPS_ERR_INVALID_ARG, "stencil: dims 1..3 and 1..%d points", OPS_MAX_STENCIL_POINTS);
  Stencil s;
  s.dims = dims;
  s.name = name ? name : "";
  s.off.assign(offsets, offsets + 3 * npts);
  for (int d = 0; d < 3; ++d) {
    s.lo[d] = 0;
    s.hi[d] = 0;
  }
  for (int p = 0; p < npts; ++p)
    for (int d = 0; d < 3; ++d) {
      if (d >= dims && s.off[3 * p + d] != 0)
        return fail(c, OPS_ERR_INVALID_ARG, "stencil '%s': offset in unused dim %d", s.name.c_str(), d);
      s.lo[d] = std::min(s.lo[d], s.off[3 * p + d]);
      s.hi[d] = std::max(s.hi[d], s.off[3 * p + d]);
    }
  c->stencils.push_back(s);
  *out = (int)c->stencils.size() - 1;
  return OPS_OK;
}

namespace {
// a new slot of the device scalar array, holding init (reductions: their identity)
int new_slot(ops_ctx c, int op, double init, int* out);
}  // namespace

int ops_decl_reduction(ops_ctx c, int op, int* out) {
  if (!c || !out) return OPS_ERR_INVALID_ARG;
  if (op < OPS_RED_SUM || op > OPS_RED_MAX) return fail(c, OPS_ERR_INVALID_ARG, "bad reduction op %d", op);
  return new_slot(c, op, red_identity(op), out);
}

int ops_decl_scalar(ops_ctx c, double init, int* out) {
  if (!c || !out) return OPS_ERR_INVALID_ARG;
  return new_slot(c, kScalarHandle, init, out);
}

int ops_scalar_set(ops_ctx c, int h, double value) {
  if (!c) return OPS_ERR_INVALID_ARG;
  if (h < 0 || h >= (int)c->red_ops.size() || c->red_ops[h] != kScalarHandle)
    return fail(c, OPS_ERR_INVALID_ARG, "bad scalar %d", h);
  if (c->host_only) return fail(c, OPS_ERR_NO_DEVICE, "host-only context");
  int rc = flush(c);  // loops queued before the call read the old value
  if (rc) return rc;
  LaunchEnv env = make_env(c);
  CUDA_TRY(c, launch_set_scalar(env, h, value));
  return OPS_OK;
}

int ops_scalar_get(ops_ctx c, int h, double* host_out) {
  if (!c || !host_out) return OPS_ERR_INVALID_ARG;
  if (h < 0 || h >= (int)c->red_ops.size() || c->red_ops[h] != kScalarHandle)
    return fail(c, OPS_ERR_INVALID_ARG, "bad scalar %d", h);
  if (c->host_only) return fail(c, OPS_ERR_NO_DEVICE, "host-only context");
  int rc = flush(c);
  if (rc) return rc;
  CUDA_TRY(c, cudaMemcpyAsync(host_out, c->d_scal + h, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  return check_device_error(c);  // synchronises the stream
}

namespace {
int new_slot(ops_ctx c, int op, double init, int* out) {
  const int h = (int)c->red_ops.size();
  if (!c->host_only) {
    int rc = flush(c);  // the slot array may be reallocated
    if (rc) return rc;
    if (h >= c->scal_cap) {
      const int nc = std::max(16, 2 * c->scal_cap);
      double* nd = nullptr;
      rc = dev_alloc(c, (void**)&nd, sizeof(double) * nc);
      if (rc) return rc;
      if (c->d_scal) {
        CUDA_TRY(c, cudaMemcpyAsync(nd, c->d_scal, sizeof(double) * c->scal_cap, cudaMemcpyDeviceToDevice, c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        dev_free(c, c->d_scal, sizeof(double) * c->scal_cap);
      }
      c->d_scal = nd;
      c->scal_cap = nc;
    }
    LaunchEnv env = make_env(c);
    CUDA_TRY(c, launch_set_scalar(env, h, init));
  }
  c->red_ops.push_back(op);
  *out = h;
  return OPS_OK;
}
}  // namespace

int ops_par_loop(ops_ctx c, int block, int dims, const int* range, int nargs, const ops_arg* args, int nins,
                 const int32_t* code, int nconsts, const double* consts, const char* name) {
  if (!c || !range || (nargs > 0 && !args) || (nins > 0 && !code) || (nconsts > 0 && !consts))
    return OPS_ERR_INVALID_ARG;
  if (block < 0 || block >= (int)c->blocks.size()) return fail(c, OPS_ERR_INVALID_ARG, "bad block %d", block);
  if (dims != c->blocks[block].dims) return fail(c, OPS_ERR_INVALID_ARG, "loop dims %d != block dims", dims);
  if (nargs < 0 || nargs > OPS_MAX_ARGS || nins < 0 || nins > OPS_MAX_INS || nconsts < 0 || nconsts > OPS_MAX_CONSTS)
    return fail(c, OPS_ERR_INVALID_ARG, "loop '%s': limits are %d args, %d instructions, %d constants",
                name ? name : "", OPS_MAX_ARGS, OPS_MAX_INS, OPS_MAX_CONSTS);
  QLoop q;
  q.block = block;
  q.dims = dims;
  q.name = name ? name : "";
  for (int d = 0; d < 3; ++d) {
    q.rng[2 * d] = d < dims ? range[2 * d] : 0;
    q.rng[2 * d + 1] = d < dims ? range[2 * d + 1] : 1;
    if (q.rng[2 * d + 1] < q.rng[2 * d])
      return fail(c, OPS_ERR_INVALID_ARG, "loop '%s': range end < start in dim %d", q.name.c_str(), d);
  }
  q.args.assign(args, args + nargs);
  q.code.assign(code, code + 6 * nins);
  q.K.assign(consts, consts + nconsts);
  int rc = validate_loop(c, q);
  if (rc) return rc;
  c->queue.push_back(std::move(q));
  return OPS_OK;
}

int ops_execute(ops_ctx c) {
  if (!c) return OPS_ERR_INVALID_ARG;
  return flush(c);
}

int ops_execute_batch(ops_ctx* ctxs, int count) {
  if (!ctxs || count < 1) return OPS_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i)
    if (!ctxs[i]) return OPS_ERR_INVALID_ARG;
  return execute_batch(ctxs, count);
}

int ops_queue_clear(ops_ctx c) {
  if (!c) return OPS_ERR_INVALID_ARG;
  c->queue.clear();
  return OPS_OK;
}

int ops_sync(ops_ctx c) {
  if (!c) return OPS_ERR_INVALID_ARG;
  int rc = flush(c);
  if (rc) return rc;
  if (c->host_only) return OPS_OK;
  return check_device_error(c);
}

int ops_reduction_result(ops_ctx c, int red, double* host_out) {
  if (!c || !host_out) return OPS_ERR_INVALID_ARG;
  if (red < 0 || red >= (int)c->red_ops.size() || c->red_ops[red] == kScalarHandle)
    return fail(c, OPS_ERR_INVALID_ARG, "bad reduction %d", red);
  int rc = flush(c);
  if (rc) return rc;
  if (c->host_only) return fail(c, OPS_ERR_NO_DEVICE, "host-only context");
  if (!c->h_small) CUDA_TRY(c, cudaHostAlloc((void**)&c->h_small, sizeof *c->h_small, cudaHostAllocDefault));
  // the value and the error word land in pinned memory: one wait for both
  CUDA_TRY(c, cudaMemcpyAsync(&c->h_small->value, c->d_scal + red, sizeof(double), cudaMemcpyDeviceToHost,
                              c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(&c->h_small->err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (c->h_small->err) {
    rc = check_device_error(c);  // resets the word and reports it
    if (rc) return rc;
  }
  *host_out = c->h_small->value;
  LaunchEnv env = make_env(c);
  CUDA_TRY(c, launch_set_scalar(env, red, red_identity(c->red_ops[red])));
  ++c->stats.launches;
  return OPS_OK;
}

// Copy a dat between its device allocation box and a dense host array
// (x fastest), after flushing the queue; to_host selects the direction.
// wait = 0 leaves the copy queued on the context's stream.
int dat_copy(ops_ctx c, int dat, void* host, int64_t nelems, bool to_host, bool wait) {
  if (!c || !host) return OPS_ERR_INVALID_ARG;
  if (dat < 0 || dat >= (int)c->dats.size()) return fail(c, OPS_ERR_INVALID_ARG, "bad dat %d", dat);
  const Dat& D0 = c->dats[dat];
  if (nelems != (int64_t)D0.ext[0] * D0.ext[1] * D0.ext[2])
    return fail(c, OPS_ERR_INVALID_ARG, "dat '%s': %s needs %lld elements", D0.name.c_str(),
                to_host ? "fetch" : "upload", (long long)D0.ext[0] * D0.ext[1] * D0.ext[2]);
  if (c->host_only) return fail(c, OPS_ERR_NO_DEVICE, "host-only context");
  int rc = flush(c);
  if (rc) return rc;
  const Dat& D = c->dats[dat];  // the flush may have moved it to its other buffer
  char* base = (char*)elem_at(D.ptr0, -(D.dm[0] + D.pitch * D.dm[1] + D.plane * D.dm[2]), c->es);
  const size_t es = (size_t)c->es, hrow = es * D.ext[0], drow = es * D.pitch;
  for (int z = 0; z < D.ext[2]; ++z) {
    char* h = (char*)host + es * (size_t)z * D.ext[0] * D.ext[1];
    char* d = base + es * (size_t)z * D.plane;
    if (to_host)
      CUDA_TRY(c, cudaMemcpy2DAsync(h, hrow, d, drow, hrow, D.ext[1], cudaMemcpyDeviceToHost, c->stream));
    else
      CUDA_TRY(c, cudaMemcpy2DAsync(d, drow, h, hrow, hrow, D.ext[1], cudaMemcpyHostToDevice, c->stream));
  }
  return wait ? check_device_error(c) : OPS_OK;
}

int ops_dat_fetch(ops_ctx c, int dat, void* host_out, int64_t nelems) {
  return dat_copy(c, dat, host_out, nelems, true, true);
}

int ops_dat_upload(ops_ctx c, int dat, const void* host_in, int64_t nelems) {
  return dat_copy(c, dat, const_cast<void*>(host_in), nelems, false, true);
}

int ops_dat_fetch_async(ops_ctx c, int dat, void* host_out, int64_t nelems) {
  return dat_copy(c, dat, host_out, nelems, true, false);
}

int ops_dat_upload_async(ops_ctx c, int dat, const void* host_in, int64_t nelems) {
  return dat_copy(c, dat, const_cast<void*>(host_in), nelems, false, false);
}

int ops_dat_info(ops_ctx c, int dat, double** dev_ptr0, int64_t* pitch, int64_t* plane, int* ext) {
  if (!c) return OPS_ERR_INVALID_ARG;
  if (dat < 0 || dat >= (int)c->dats.size()) return fail(c, OPS_ERR_INVALID_ARG, "bad dat %d", dat);
  const Dat& D = c->dats[dat];
  if (dev_ptr0) *dev_ptr0 = D.ptr0;
  if (pitch) *pitch = D.pitch;
  if (plane) *plane = D.plane;
  if (ext)
    for (int d = 0; d < 3; ++d) ext[d] = D.ext[d];
  return OPS_OK;
}

int ops_last_stats(ops_ctx c, ops_flush_stats* out) {
  if (!c || !out) return OPS_ERR_INVALID_ARG;
  if (c->cfg.timing && c->ev_used >= 2) {
    double ms = 0.0;
    for (int i = 0; i + 1 < c->ev_used; i += 2) {
      CUDA_TRY(c, cudaEventSynchronize(c->ev_pool[i + 1]));
      float t = 0.f;
      CUDA_TRY(c, cudaEventElapsedTime(&t, c->ev_pool[i], c->ev_pool[i + 1]));
      ms += t;
    }
    c->stats.kernel_ms = ms;
  }
  *out = c->stats;
  return OPS_OK;
}

int ops_plan_skewed(ops_ctx c, const int* tile, int* out_ntiles, int* out_ranges, int64_t cap) {
  if (!c || !tile || !out_ntiles || !out_ranges) return OPS_ERR_INVALID_ARG;
  if (c->queue.empty()) return fail(c, OPS_ERR_STATE, "no queued loops");
  const int ndim = c->queue[0].dims;
  std::vector<PLoop> pl;
  for (const QLoop& q : c->queue) {
    if (q.dims != ndim) return fail(c, OPS_ERR_INVALID_ARG, "queued loops of different dimensionality");
    pl.push_back(plan_loop(c, q));
  }
  int t[3] = {1, 1, 1};
  for (int d = 0; d < ndim; ++d) {
    if (tile[d] < 1) return fail(c, OPS_ERR_INVALID_ARG, "tile sizes must be >= 1");
    t[d] = tile[d];
  }
  SkewedPlan P;
  build_skewed_ranges(pl, (int)c->dats.size(), ndim, t, P);
  int64_t need = 0;
  for (int d = 0; d < ndim; ++d) need += (int64_t)P.ranges[d].size();
  if (need > cap) return fail(c, OPS_ERR_INVALID_ARG, "out_ranges needs %lld ints", (long long)need);
  int64_t pos = 0;
  for (int d = 0; d < ndim; ++d) {
    out_ntiles[d] = P.ntiles[d];
    std::memcpy(out_ranges + pos, P.ranges[d].data(), sizeof(int) * P.ranges[d].size());
    pos += (int64_t)P.ranges[d].size();
  }
  return OPS_OK;
}

int ops_compile_queued_wavefront(ops_ctx c, char* src_out, int64_t cap, int64_t* src_len, double* compile_ms) {
  if (!c) return OPS_ERR_INVALID_ARG;
  if (c->queue.empty()) return fail(c, OPS_ERR_STATE, "no queued loops");
  const int n = (int)c->queue.size();
  std::vector<DLoop> hl(n);
  std::vector<FoldRow> rows;
  for (int i = 0; i < n; ++i) fill_dloop(c, c->queue[i], hl[i], (int)rows.size(), rows);
  std::string src, why;
  double ms = 0.0;
  const int rc = jit_compile_wavefront_only(hl.data(), n, read_only_args(c, 0, n), c->es, &src, &why, &ms);
  if (src_len) *src_len = (int64_t)src.size();
  if (src_out && cap > 0) {
    const size_t k = std::min<size_t>(src.size(), (size_t)cap - 1);
    std::memcpy(src_out, src.data(), k);
    src_out[k] = '\0';
  }
  if (compile_ms) *compile_ms = ms;
  if (rc) return fail(c, rc, "%s", why.c_str());
  return OPS_OK;
}

int compile_queued_tilewave(ops_ctx c, char* src_out, int64_t cap, int64_t* src_len, double* compile_ms,
                            bool batch);

int ops_compile_queued_tilewarp(ops_ctx c, char* src_out, int64_t cap, int64_t* src_len, double* compile_ms) {
  if (!c) return OPS_ERR_INVALID_ARG;
  if (c->queue.empty()) return fail(c, OPS_ERR_STATE, "no queued loops");
  const int n = (int)c->queue.size();
  std::vector<DLoop> hl(n);
  std::vector<FoldRow> rows;
  for (int i = 0; i < n; ++i) fill_dloop(c, c->queue[i], hl[i], (int)rows.size(), rows);
  std::string src, why;
  double ms = 0.0;
  const int rc = jit_compile_tilewarp_only(hl.data(), n, read_only_args(c, 0, n), c->es, c->queue[0].dims, &src,
                                           &why, &ms);
  if (src_len) *src_len = (int64_t)src.size();
  if (src_out && cap > 0) {
    const size_t k = std::min<size_t>(src.size(), (size_t)cap - 1);
    std::memcpy(src_out, src.data(), k);
    src_out[k] = '\0';
  }
  if (compile_ms) *compile_ms = ms;
  if (rc) return fail(c, rc, "%s", why.c_str());
  return OPS_OK;
}

int ops_compile_queued_skewed(ops_ctx c, char* src_out, int64_t cap, int64_t* src_len, double* compile_ms) {
  if (!c) return OPS_ERR_INVALID_ARG;
  if (c->queue.empty()) return fail(c, OPS_ERR_STATE, "no queued loops");
  const int n = (int)c->queue.size();
  std::vector<DLoop> hl(n);
  std::vector<FoldRow> rows;
  for (int i = 0; i < n; ++i) fill_dloop(c, c->queue[i], hl[i], (int)rows.size(), rows);
  std::string src, why;
  double ms = 0.0;
  const int rc = jit_compile_skewed_only(hl.data(), n, read_only_args(c, 0, n), c->es, &src, &why, &ms);
  if (src_len) *src_len = (int64_t)src.size();
  if (src_out && cap > 0) {
    const size_t k = std::min<size_t>(src.size(), (size_t)cap - 1);
    std::memcpy(src_out, src.data(), k);
    src_out[k] = '\0';
  }
  if (compile_ms) *compile_ms = ms;
  if (rc) return fail(c, rc, "%s", why.c_str());
  return OPS_OK;
}

int ops_compile_queued_tilewave(ops_ctx c, char* src_out, int64_t cap, int64_t* src_len, double* compile_ms) {
  return compile_queued_tilewave(c, src_out, cap, src_len, compile_ms, false);
}

int ops_compile_queued_tilewave_batch(ops_ctx c, char* src_out, int64_t cap, int64_t* src_len,
                                      double* compile_ms) {
  return compile_queued_tilewave(c, src_out, cap, src_len, compile_ms, true);
}

int compile_queued_tilewave(ops_ctx c, char* src_out, int64_t cap, int64_t* src_len, double* compile_ms,
                            bool batch) {
  if (!c) return OPS_ERR_INVALID_ARG;
  if (c->queue.empty()) return fail(c, OPS_ERR_STATE, "no queued loops");
  const int n = (int)c->queue.size();
  std::vector<DLoop> hl(n);
  std::vector<FoldRow> rows;
  for (int i = 0; i < n; ++i) fill_dloop(c, c->queue[i], hl[i], (int)rows.size(), rows);
  std::string src, why;
  double ms = 0.0;
  const int rc = jit_compile_tilewave_only(hl.data(), n, read_only_args(c, 0, n), c->es, c->queue[0].dims, &src,
                                           &why, &ms, batch);
  if (src_len) *src_len = (int64_t)src.size();
  if (src_out && cap > 0) {
    const size_t k = std::min<size_t>(src.size(), (size_t)cap - 1);
    std::memcpy(src_out, src.data(), k);
    src_out[k] = '\0';
  }
  if (compile_ms) *compile_ms = ms;
  if (rc) return fail(c, rc, "%s", why.c_str());
  return OPS_OK;
}

int ops_plan_tilewave(ops_ctx c, const int* tile, int64_t* counts, int* out_need, int64_t need_cap, int* out_class,
                      int* out_order, int64_t tile_cap, int* out_steps) {
  if (!c || !tile || !counts) return OPS_ERR_INVALID_ARG;
  if (c->queue.empty()) return fail(c, OPS_ERR_STATE, "no queued loops");
  const int ndim = c->queue[0].dims;
  std::vector<PLoop> pl;
  for (const QLoop& q : c->queue) {
    if (q.dims != ndim) return fail(c, OPS_ERR_INVALID_ARG, "queued loops of different dimensionality");
    pl.push_back(plan_loop(c, q));
  }
  int t[3] = {1, 1, 1};
  for (int d = 0; d < ndim; ++d) {
    if (tile[d] < 1) return fail(c, OPS_ERR_INVALID_ARG, "tile sizes must be >= 1");
    t[d] = tile[d];
  }
  SkewedPlan P;
  build_skewed_ranges(pl, (int)c->dats.size(), ndim, t, P);
  TileWavePlan W;
  std::string why;
  if (!build_tile_wave(pl, P, W, &why, jit_tile_group(), jit_tile_band()))
    return fail(c, OPS_ERR_INVALID_ARG, "%s", why.c_str());
  const int64_t ntiles = (int64_t)P.ntiles[0] * P.ntiles[1] * P.ntiles[2];
  const int64_t ncl = (int64_t)W.ncls[0] * W.ncls[1] * W.ncls[2];
  counts[0] = ntiles;
  counts[1] = ncl;
  counts[2] = W.ndirs;
  counts[3] = W.nloops;
  counts[4] = (int64_t)W.groups.size() - 1;
  if (out_steps) std::memcpy(out_steps, W.groups.data(), sizeof(int) * W.groups.size());
  if (out_need) {
    if ((int64_t)W.need.size() > need_cap)
      return fail(c, OPS_ERR_INVALID_ARG, "out_need needs %lld ints", (long long)W.need.size());
    for (size_t k = 0; k < W.need.size(); ++k) out_need[k] = W.need[k];
  }
  if ((out_class || out_order) && ntiles > tile_cap)
    return fail(c, OPS_ERR_INVALID_ARG, "tile outputs need %lld ints", (long long)ntiles);
  if (out_class)
    for (int tz = 0; tz < P.ntiles[2]; ++tz)
      for (int ty = 0; ty < P.ntiles[1]; ++ty)
        for (int tx = 0; tx < P.ntiles[0]; ++tx)
          out_class[((int64_t)tz * P.ntiles[1] + ty) * P.ntiles[0] + tx] =
              (W.cls[2][tz] * W.ncls[1] + W.cls[1][ty]) * W.ncls[0] + W.cls[0][tx];
  if (out_order) std::memcpy(out_order, W.order.data(), sizeof(int) * W.order.size());
  return OPS_OK;
}

int ops_plan_wavefront(ops_ctx c, const int* tile, int64_t* counts, int* out_phases, int64_t phase_cap,
                       int* out_deps, int64_t dep_cap) {
  if (!c || !tile || !counts) return OPS_ERR_INVALID_ARG;
  if (c->queue.empty()) return fail(c, OPS_ERR_STATE, "no queued loops");
  const int ndim = c->queue[0].dims;
  std::vector<PLoop> pl;
  for (const QLoop& q : c->queue) {
    if (q.dims != ndim) return fail(c, OPS_ERR_INVALID_ARG, "queued loops of different dimensionality");
    pl.push_back(plan_loop(c, q));
  }
  int t[3] = {1, 1, 1};
  for (int d = 0; d < ndim; ++d) {
    if (tile[d] < 1) return fail(c, OPS_ERR_INVALID_ARG, "tile sizes must be >= 1");
    t[d] = tile[d];
  }
  SkewedPlan P;
  build_skewed_ranges(pl, (int)c->dats.size(), ndim, t, P);
  build_phases(pl, P);
  WavePlan W;
  build_wavefront(pl, (int)c->dats.size(), P, ndim - 1, jit_rows_per_unit(c->es), jit_wave_threads(),
                  jit_wave_units_per_chunk(), jit_wave_slope(), W);
  const int64_t nph = (int64_t)P.phases.size();
  counts[0] = nph;
  counts[1] = (int64_t)W.deps.size();
  counts[2] = W.nunits;
  counts[3] = W.nlevels;
  if (out_phases) {
    if (12 * nph > phase_cap) return fail(c, OPS_ERR_INVALID_ARG, "out_phases needs %lld ints", (long long)(12 * nph));
    for (int64_t q = 0; q < nph; ++q) {
      int* o = out_phases + 12 * q;
      o[0] = P.phases[q].loop;
      o[1] = W.nchunk[q];
      o[2] = W.ustart[q];
      o[3] = W.dep_off[q];
      o[4] = W.dep_off[q + 1] - W.dep_off[q];
      o[5] = W.level[q];
      for (int k = 0; k < 6; ++k) o[6 + k] = P.phases[q].box[k];
    }
  }
  if (out_deps) {
    if ((int64_t)W.deps.size() > dep_cap)
      return fail(c, OPS_ERR_INVALID_ARG, "out_deps needs %lld ints", (long long)W.deps.size());
    if (!W.deps.empty()) std::memcpy(out_deps, W.deps.data(), sizeof(int) * W.deps.size());
  }
  return OPS_OK;
}

int ops_compile_queued(ops_ctx c, char* src_out, int64_t cap, int64_t* src_len, double* compile_ms) {
  if (!c) return OPS_ERR_INVALID_ARG;
  if (c->queue.empty()) return fail(c, OPS_ERR_STATE, "no queued loops");
  const int n = (int)c->queue.size();
  std::vector<DLoop> hl(n);
  std::vector<FoldRow> rows;
  std::set<int> written;
  for (int i = 0; i < n; ++i) {
    fill_dloop(c, c->queue[i], hl[i], (int)rows.size(), rows);
    for (const ops_arg& a : c->queue[i].args)
      if (a.kind == OPS_ARG_DAT && a.access != OPS_READ) written.insert(a.handle);
  }
  std::vector<std::vector<char>> ro(n);
  for (int i = 0; i < n; ++i) {
    const QLoop& q = c->queue[i];
    ro[i].assign(q.args.size(), 0);
    for (size_t a = 0; a < q.args.size(); ++a)
      ro[i][a] = q.args[a].kind == OPS_ARG_DAT && !written.count(q.args[a].handle);
  }
  std::string src, why;
  double ms = 0.0;
  int rc = jit_compile_only(hl.data(), n, ro, c->es, &src, &why, &ms);
  if (!rc) {
    // the overlapped-tile form of the same loops, with each dat's own strides as its footprint strides
    std::map<int, int> local;
    OvLayout lay;
    lay.es = c->es;
    std::vector<DLoop> ol(hl);
    for (int i = 0; i < n; ++i) {
      const QLoop& q = c->queue[i];
      for (size_t a = 0; a < q.args.size(); ++a) {
        if (q.args[a].kind != OPS_ARG_DAT) continue;
        auto it = local.find(q.args[a].handle);
        if (it == local.end()) {
          const Dat& D = c->dats[q.args[a].handle];
          it = local.emplace(q.args[a].handle, lay.ndats++).first;
          lay.smem_off.push_back(0);
          lay.spitch.push_back((int)D.pitch);
          lay.splane.push_back((int)D.plane);
          lay.written.push_back(0);
        }
        ol[i].args[a].slot = it->second;
        if (q.args[a].access != OPS_READ) lay.written[it->second] = 1;
      }
    }
    std::string osrc;
    rc = jit_compile_overlap_only(ol.data(), n, lay, &osrc, &why, &ms);
    src += osrc;
  }

  if (src_len) *src_len = (int64_t)src.size();
  if (src_out && cap > 0) {
    const size_t k = std::min<size_t>(src.size(), (size_t)cap - 1);
    std::memcpy(src_out, src.data(), k);
    src_out[k] = '\0';
  }
  if (compile_ms) *compile_ms = ms;
  if (rc) return fail(c, rc, "%s", why.c_str());
  return OPS_OK;
}

int ops_plan_overlapped(ops_ctx c, const int owned[6], int* out_boxes, int* out_foot) {
  if (!c || !owned || !out_boxes || !out_foot) return OPS_ERR_INVALID_ARG;
  if (c->queue.empty()) return fail(c, OPS_ERR_STATE, "no queued loops");
  const int ndim = c->queue[0].dims;
  std::vector<PLoop> pl;
  for (const QLoop& q : c->queue) {
    if (q.dims != ndim) return fail(c, OPS_ERR_INVALID_ARG, "queued loops of different dimensionality");
    pl.push_back(plan_loop(c, q));
  }
  OverlapTile ot;
  build_overlap_tile(pl, (int)c->dats.size(), ndim, owned, ot);
  std::memcpy(out_boxes, ot.box.data(), sizeof(int) * ot.box.size());
  std::memcpy(out_foot, ot.foot.data(), sizeof(int) * ot.foot.size());
  return OPS_OK;
}

}  // extern "C"
