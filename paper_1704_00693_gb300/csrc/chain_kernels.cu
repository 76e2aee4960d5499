// Device side of the loop-chain executor for GB300 (sm_103a).
//
// Every loop body is a short program in the register IR of opstile.h,
// interpreted per grid point.  All arithmetic uses the explicitly rounded
// intrinsics (__dadd_rn, __dmul_rn, __fma_rn, __ddiv_rn) and the library is
// built with -fmad=false, so a point's value is bit-identical whatever the
// schedule: untiled, skewed (Sec. 4.B, Algorithm 2) or overlapped (Sec. 4.D).
//
// Interpreter layout.  A thread owns a group of kPts points (consecutive
// rows of one x, or kPts flattened points of a thin box).  Each instruction
// is decoded once, warp-uniformly, from the shared-memory copy of the loop
// and applied to the whole group: decoding is amortised over kPts points
// and every stencil load comes with kPts independent siblings.  The eight IR
// registers of every point live in shared memory as R[reg][point][thread]
// (consecutive threads hit consecutive words: no bank conflicts, no local
// memory).  FP64 on GB300 issues about two DFMA per clock per SM, so a body
// with a handful of fma per point is bound by the FP64 pipe once the
// interpreter's own instructions stay well below ~60 per FP64 instruction.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace opstile {

#ifndef OPS_PTS
#define OPS_PTS 4
#endif
#ifndef OPS_MIN_CTAS
#define OPS_MIN_CTAS 2
#endif
constexpr int kPts = OPS_PTS;  // points per thread

// Shared memory of the chain kernels (dynamic, 16-byte aligned), for P
// points per thread.
template <int P>
struct ChainSmemT {
  DLoop L;
  DD sh[32];                                 // block reductions
  DD sred[OPS_MAX_REDS_PER_LOOP * kThreads]; // per-thread reduction accumulators
  int own[6];                                // overlapped tiles: only points in this box reduce
  int own_check;
  int pad_;
  double R[kNReg * P * kThreads];            // IR registers [reg][point][thread]
};
using ChainSmem = ChainSmemT<kPts>;
constexpr size_t kChainSmem = sizeof(ChainSmem);

#include "device_common.cuh"
static_assert(OPS_RED_SUM == 0 && OPS_RED_MIN == 1 && OPS_RED_MAX == 2, "device_common.cuh reduction codes");

template <int P>
__device__ __forceinline__ void red_init(ChainSmemT<P>& S) {
  for (int k = 0; k < S.L.nreds; ++k) S.sred[k * kThreads + threadIdx.x] = DD{red_identity(S.L.red_op[k]), 0.0};
}

// ----------------------------------------------------------------------------
// a group of points
// ----------------------------------------------------------------------------
template <int P>
struct GroupT {
  int x[P], y[P], z[P];
  unsigned mask;  // bit p: point p exists
};

__device__ __forceinline__ bool point_ok(const DLoop& L, int x, int y, int z) {
  if (x < L.rng[0] || x >= L.rng[1] || y < L.rng[2] || y >= L.rng[3] || z < L.rng[4] || z >= L.rng[5])
    return false;
  const int c[3] = {x, y, z};
  for (int a = 0; a < L.nargs; ++a) {
    const DArg& A = L.args[a];
    if (A.kind != OPS_ARG_DAT) continue;
    for (int d = 0; d < 3; ++d)
      if (c[d] + A.slo[d] < A.alo[d] || c[d] + A.shi[d] >= A.ahi[d]) return false;
  }
  return true;
}

// Address of the group's point p in the dat of argument A.
template <int P>
__device__ __forceinline__ const double* gptr(const DArg& A, const GroupT<P>& g, int p) {
  return A.ptr0 + ((int64_t)g.x[p] + (int64_t)g.y[p] * A.pitch + (int64_t)g.z[p] * A.plane);
}

template <int P>
__device__ __forceinline__ void run_group(ChainSmemT<P>& S, const GroupT<P>& g, const double* __restrict__ scal) {
  const DLoop& L = S.L;
  double* Rt = S.R + threadIdx.x;  // register r, point p at Rt[(r * P + p) * kThreads]
  constexpr int RS = P * kThreads;
  const unsigned m = g.mask;
  for (int r = 0; r < kNReg; ++r)
    if ((L.zmask >> r) & 1) {
#pragma unroll
      for (int p = 0; p < P; ++p) Rt[r * RS + p * kThreads] = 0.0;
    }
  const int nins = L.nins;
  for (int pc = 0; pc < nins; ++pc) {
    const int2 i01 = *reinterpret_cast<const int2*>(&L.ins[pc][0]);
    const int2 i23 = *reinterpret_cast<const int2*>(&L.ins[pc][2]);
    const int2 i45 = *reinterpret_cast<const int2*>(&L.ins[pc][4]);
    const int op = i01.x;
    double* Rd = Rt + i01.y * RS;
    const double* Ra = Rt + i23.x * RS;
    const double* Rb = Rt + i23.y * RS;
    switch (op) {
      case OPS_IR_LD: {
        const DArg& A = L.args[i23.x];
        if (A.kind == OPS_ARG_SCALAR) {
          const double v = scal[A.slot];
#pragma unroll
          for (int p = 0; p < P; ++p) Rd[p * kThreads] = v;
        } else {
          const int32_t o = A.off[i23.y];
          double v[P];
#pragma unroll
          for (int p = 0; p < P; ++p) v[p] = ((m >> p) & 1u) ? gptr(A, g, p)[o] : 0.0;
#pragma unroll
          for (int p = 0; p < P; ++p) Rd[p * kThreads] = v[p];
        }
        break;
      }
      case OPS_IR_CST: {
        const double v = L.K[i23.x];
#pragma unroll
        for (int p = 0; p < P; ++p) Rd[p * kThreads] = v;
        break;
      }
      case OPS_IR_ADD:
#pragma unroll
        for (int p = 0; p < P; ++p) Rd[p * kThreads] = __dadd_rn(Ra[p * kThreads], Rb[p * kThreads]);
        break;
      case OPS_IR_SUB:
#pragma unroll
        for (int p = 0; p < P; ++p) Rd[p * kThreads] = __dsub_rn(Ra[p * kThreads], Rb[p * kThreads]);
        break;
      case OPS_IR_MUL:
#pragma unroll
        for (int p = 0; p < P; ++p) Rd[p * kThreads] = __dmul_rn(Ra[p * kThreads], Rb[p * kThreads]);
        break;
      case OPS_IR_DIV:
#pragma unroll
        for (int p = 0; p < P; ++p) Rd[p * kThreads] = __ddiv_rn(Ra[p * kThreads], Rb[p * kThreads]);
        break;
      case OPS_IR_MIN:
#pragma unroll
        for (int p = 0; p < P; ++p) {
          const double a = Ra[p * kThreads], b = Rb[p * kThreads];
          Rd[p * kThreads] = (b < a) ? b : a;
        }
        break;
      case OPS_IR_MAX:
#pragma unroll
        for (int p = 0; p < P; ++p) {
          const double a = Ra[p * kThreads], b = Rb[p * kThreads];
          Rd[p * kThreads] = (b > a) ? b : a;
        }
        break;
      case OPS_IR_FMA: {
        const double* Rc = Rt + i45.x * RS;
#pragma unroll
        for (int p = 0; p < P; ++p)
          Rd[p * kThreads] = __fma_rn(Ra[p * kThreads], Rb[p * kThreads], Rc[p * kThreads]);
        break;
      }
      case OPS_IR_SGT: {
        const double* Rc = Rt + i45.x * RS;
        const double* Re = Rt + i45.y * RS;
#pragma unroll
        for (int p = 0; p < P; ++p)
          Rd[p * kThreads] = (Ra[p * kThreads] > Rb[p * kThreads]) ? Rc[p * kThreads] : Re[p * kThreads];
        break;
      }
      case OPS_IR_WSUM:
      case OPS_IR_WACC: {
        const DArg& A = L.args[i23.x];
        const double* Kb = L.K + i23.y;
        const int n = A.npts;
        const double* base[P];
        double t[P];
#pragma unroll
        for (int p = 0; p < P; ++p) base[p] = gptr(A, g, p);
        int q = 0;
        if (op == OPS_IR_WSUM) {
          const int32_t o = A.off[0];
          const double k = Kb[0];
#pragma unroll
          for (int p = 0; p < P; ++p) t[p] = __dmul_rn(k, ((m >> p) & 1u) ? base[p][o] : 0.0);
          q = 1;
        } else {
#pragma unroll
          for (int p = 0; p < P; ++p) t[p] = Rd[p * kThreads];
        }
        for (; q + 2 <= n; q += 2) {
          const int32_t o0 = A.off[q], o1 = A.off[q + 1];
          const double k0 = Kb[q], k1 = Kb[q + 1];
          double v0[P], v1[P];
#pragma unroll
          for (int p = 0; p < P; ++p) {
            const bool on = (m >> p) & 1u;
            v0[p] = on ? base[p][o0] : 0.0;
            v1[p] = on ? base[p][o1] : 0.0;
          }
#pragma unroll
          for (int p = 0; p < P; ++p) t[p] = __fma_rn(k1, v1[p], __fma_rn(k0, v0[p], t[p]));
        }
        if (q < n) {
          const int32_t o = A.off[q];
          const double k = Kb[q];
#pragma unroll
          for (int p = 0; p < P; ++p) t[p] = __fma_rn(k, ((m >> p) & 1u) ? base[p][o] : 0.0, t[p]);
        }
#pragma unroll
        for (int p = 0; p < P; ++p) Rd[p * kThreads] = t[p];
        break;
      }
      case OPS_IR_POLY: {
        const int c = i45.x;
        const double* Kb = L.K + i23.y;
        double x[P], t[P];
#pragma unroll
        for (int p = 0; p < P; ++p) {
          x[p] = Ra[p * kThreads];
          t[p] = Kb[c];
        }
        for (int i = c - 1; i >= 0; --i) {
          const double k = Kb[i];
#pragma unroll
          for (int p = 0; p < P; ++p) t[p] = __fma_rn(t[p], x[p], k);
        }
#pragma unroll
        for (int p = 0; p < P; ++p) Rd[p * kThreads] = t[p];
        break;
      }
      case OPS_IR_ST: {
        const DArg& A = L.args[i01.y];
        const bool inc = A.access == OPS_INC;
#pragma unroll
        for (int p = 0; p < P; ++p) {
          if ((m >> p) & 1u) {
            double* q = const_cast<double*>(gptr(A, g, p));
            const double v = Ra[p * kThreads];
            *q = inc ? __dadd_rn(*q, v) : v;
          }
        }
        break;
      }
      case OPS_IR_RED: {
        const int k = L.args[i01.y].slot;
        const int rop = L.red_op[k];
        DD* slot = S.sred + k * kThreads + threadIdx.x;
        DD acc = *slot;
#pragma unroll
        for (int p = 0; p < P; ++p) {
          if (!((m >> p) & 1u)) continue;
          if (S.own_check && (g.x[p] < S.own[0] || g.x[p] >= S.own[1] || g.y[p] < S.own[2] || g.y[p] >= S.own[3] ||
                              g.z[p] < S.own[4] || g.z[p] >= S.own[5]))
            continue;  // redundant point of an overlapped tile
          acc = red_add(rop, acc, Ra[p * kThreads]);
        }
        *slot = acc;
        break;
      }
      default:
        break;
    }
  }
}

// Copy a loop descriptor into shared memory (all threads participate).
__device__ __forceinline__ void stage_loop(DLoop* dst, const DLoop* src) {
  const int4* s = reinterpret_cast<const int4*>(src);
  int4* d = reinterpret_cast<int4*>(dst);
  constexpr int n = sizeof(DLoop) / sizeof(int4);
  for (int i = threadIdx.x; i < n; i += blockDim.x) d[i] = s[i];
}

// Drop points that fail the checked-mode test, flagging the error word.
template <int P>
__device__ __forceinline__ void check_group(const DLoop& L, GroupT<P>& g, int* err) {
#pragma unroll
  for (int p = 0; p < P; ++p)
    if (((g.mask >> p) & 1u) && !point_ok(L, g.x[p], g.y[p], g.z[p])) {
      g.mask &= ~(1u << p);
      atomicCAS(err, 0, kDevErrBounds);
    }
}

// Run this CTA's share of `box` for the staged loop.  Boxes with rows of at
// least 128 points are cut into units of 256 consecutive x by kPts
// consecutive rows (a thread takes one x and kPts rows: coalesced loads, and
// the rows share stencil neighbours in L1); thinner boxes are flattened into
// units of 256 * kPts points.  Units are enumerated as part, part + nparts,
// ... with coordinates advanced incrementally (no division in the loop).
template <int P>
__device__ __forceinline__ void run_box(ChainSmemT<P>& S, const int* box, const double* __restrict__ scal, int part,
                                        int nparts, int check, int* err) {
  const int x0 = box[0], nx = box[1] - box[0];
  const int y0 = box[2], ny = box[3] - box[2];
  const int z0 = box[4], nz = box[5] - box[4];
  if (nx <= 0 || ny <= 0 || nz <= 0) return;
  GroupT<P> g;
  if (nx >= 128) {
    const int xch = (nx + kThreads - 1) / kThreads;
    const int nrg = (ny + P - 1) / P;  // row groups per plane
    const int nunits = xch * nrg * nz;
    int u = part;
    int xc = u % xch, rg = (u / xch) % nrg, z = u / (xch * nrg);
    const int dxc = nparts % xch, drg = (nparts / xch) % nrg, dz = nparts / (xch * nrg);
    while (u < nunits) {
      const int x = x0 + xc * kThreads + (int)threadIdx.x;
      g.mask = 0;
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const int y = rg * P + p;
        g.x[p] = x;
        g.y[p] = y0 + y;
        g.z[p] = z0 + z;
        if (x < x0 + nx && y < ny) g.mask |= 1u << p;
      }
      if (check) check_group(S.L, g, err);
      if (g.mask) run_group(S, g, scal);
      u += nparts;
      xc += dxc;
      rg += drg;
      z += dz;
      if (xc >= xch) {
        xc -= xch;
        ++rg;
      }
      if (rg >= nrg) {
        rg -= nrg;
        ++z;
      }
    }
  } else {
    const int npts = nx * ny * nz;
    const int step = nparts * kThreads * P;
    // point p of the thread's group: linear index i + p * kThreads
    int i = part * kThreads * P + (int)threadIdx.x;
    int x = i % nx, row = i / nx;
    int y = row % ny, zz = row / ny;
    const int dx = step % nx, drow = step / nx;
    const int dy = drow % ny, dzz = drow / ny;
    const int px = kThreads % nx, prow = kThreads / nx;
    const int py = prow % ny, pz = prow / ny;
    while (i < npts) {
      g.mask = 0;
      int xp = x, yp = y, zp = zz;
#pragma unroll
      for (int p = 0; p < P; ++p) {
        g.x[p] = x0 + xp;
        g.y[p] = y0 + yp;
        g.z[p] = z0 + zp;
        if (i + p * kThreads < npts) g.mask |= 1u << p;
        xp += px;
        yp += py;
        zp += pz;
        if (xp >= nx) {
          xp -= nx;
          ++yp;
        }
        if (yp >= ny) {
          yp -= ny;
          ++zp;
        }
      }
      if (check) check_group(S.L, g, err);
      if (g.mask) run_group(S, g, scal);
      i += step;
      x += dx;
      y += dy;
      zz += dzz;
      if (x >= nx) {
        x -= nx;
        ++y;
      }
      if (y >= ny) {
        y -= ny;
        ++zz;
      }
    }
  }
}

// Fold this CTA's reduction accumulators into its partial column (assign or combine).
template <int P>
__device__ __forceinline__ void flush_partials(ChainSmemT<P>& S, DD* part, int stride, bool assign) {
  const DLoop& L = S.L;
  for (int k = 0; k < L.nreds; ++k) {
    const int op = L.red_op[k];
    DD v = block_combine(op, S.sred[k * kThreads + threadIdx.x], S.sh);
    if (threadIdx.x == 0) {
      DD* dst = part + (size_t)(L.part_row + k) * stride + blockIdx.x;
      *dst = assign ? v : red_combine(op, *dst, v);
    }
    __syncthreads();
  }
}

// ----------------------------------------------------------------------------
// untiled: one launch per loop over a box (the comparator form)
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads, OPS_MIN_CTAS) k_untiled(const DLoop* __restrict__ gL, int bx0, int bx1,
                                                                    int by0, int by1, int bz0, int bz1,
                                                                    const double* __restrict__ scal, DD* part,
                                                                    int stride, int check, int* err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ChainSmem& S = *reinterpret_cast<ChainSmem*>(smem_raw);
  stage_loop(&S.L, gL);
  if (threadIdx.x == 0) S.own_check = 0;
  __syncthreads();
  red_init(S);
  const int box[6] = {bx0, bx1, by0, by1, bz0, bz1};
  run_box(S, box, scal, blockIdx.x, gridDim.x, check, err);
  if (S.L.nreds) flush_partials(S, part, stride, true);
}

int untiled_grid(const LaunchEnv& env, const int* box) {
  const long long nx = box[1] - box[0], ny = box[3] - box[2], nz = box[5] - box[4];
  long long units = nx >= 128 ? ((nx + kThreads - 1) / kThreads) * ((ny + kPts - 1) / kPts) * nz
                              : (nx * ny * nz + (long long)kThreads * kPts - 1) / ((long long)kThreads * kPts);
  long long cap = (long long)env.num_sms * 8;
  if (units < 1) units = 1;
  return (int)(units < cap ? units : cap);
}

cudaError_t launch_untiled(const LaunchEnv& env, const DLoop* d_loop, const int* box, int grid) {
  k_untiled<<<grid, kThreads, kChainSmem, env.stream>>>(d_loop, box[0], box[1], box[2], box[3], box[4], box[5],
                                                        env.scal, env.part, env.part_stride, env.check, env.err);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// reduction partials: initialise rows, fold rows into scalar slots
// ----------------------------------------------------------------------------
__global__ void k_part_init(DD* part, int stride, const FoldRow* rows, int row0) {
  const int r = row0 + blockIdx.x;
  const double id = red_identity(rows[r].op);
  for (int i = threadIdx.x; i < stride; i += blockDim.x) part[(size_t)r * stride + i] = DD{id, 0.0};
}

cudaError_t launch_part_init(const LaunchEnv& env, int row0, int nrows) {
  if (nrows <= 0) return cudaSuccess;
  k_part_init<<<nrows, kThreads, 0, env.stream>>>(env.part, env.part_stride, env.rows, row0);
  return cudaGetLastError();
}

// Each row's partials are combined in a fixed order (strided per thread, then
// a fixed tree), so results depend only on the launch shape, never on timing.
// Fold row r of the partials (stored at row r - rbase) into its slot.
__device__ __forceinline__ void fold_row(const DD* __restrict__ part, int stride, const FoldRow* rows, int r,
                                         int rbase, int nused, double* scal) {
  __shared__ DD sh[32];
  const int op = rows[r].op;
  DD v{red_identity(op), 0.0};
  for (int i = threadIdx.x; i < nused; i += blockDim.x) v = red_combine(op, v, part[(size_t)(r - rbase) * stride + i]);
  v = block_combine(op, v, sh);
  if (threadIdx.x == 0) {
    const int s = rows[r].slot;
    const double cur = scal[s];
    if (op == OPS_RED_SUM) {
      DD t = dd_add(DD{cur, 0.0}, v.hi);
      scal[s] = __dadd_rn(t.hi, __dadd_rn(t.lo, v.lo));
    } else if (op == OPS_RED_MIN) {
      scal[s] = (v.hi < cur) ? v.hi : cur;
    } else {
      scal[s] = (v.hi > cur) ? v.hi : cur;
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_fold(const DD* __restrict__ part, int stride, const FoldRow* rows,
                                                   int row0, int nused, double* scal, int rbase) {
  fold_row(part, stride, rows, row0 + blockIdx.x, rbase, nused, scal);
}

// One launch folds the same rows of several instances (blockIdx.y).
__global__ void __launch_bounds__(kThreads) k_fold_batch(const FoldInst* __restrict__ fi, int row0, int rbase,
                                                         int nused) {
  const FoldInst& F = fi[blockIdx.y];
  fold_row(F.part, F.stride, F.rows, row0 + blockIdx.x, rbase, nused > 0 ? nused : F.nused, F.scal);
}

cudaError_t launch_fold(const LaunchEnv& env, int row0, int nrows, int grid_used) {
  if (nrows <= 0) return cudaSuccess;
  k_fold<<<nrows, kThreads, 0, env.stream>>>(env.part, env.part_stride, env.rows, row0, grid_used, env.scal, 0);
  return cudaGetLastError();
}

cudaError_t launch_fold_rows(const LaunchEnv& env, const DD* part, int stride, int row0, int nrows, int nused) {
  if (nrows <= 0) return cudaSuccess;
  k_fold<<<nrows, kThreads, 0, env.stream>>>(part, stride, env.rows, row0, nused, env.scal, row0);
  return cudaGetLastError();
}

cudaError_t launch_fold_batch(cudaStream_t stream, const FoldInst* d_fi, int ninst, int row0, int nrows, int rbase,
                              int nused) {
  if (nrows <= 0 || ninst <= 0) return cudaSuccess;
  k_fold_batch<<<dim3(nrows, ninst), kThreads, 0, stream>>>(d_fi, row0, rbase, nused);
  return cudaGetLastError();
}

__global__ void k_set_scalar(double* scal, int slot, double v) { scal[slot] = v; }

cudaError_t launch_set_scalar(const LaunchEnv& env, int slot, double value) {
  k_set_scalar<<<1, 1, 0, env.stream>>>(env.scal, slot, value);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// skewed tiling (Algorithm 2): one persistent cooperative kernel runs every
// (tile, loop) phase of a segment in plan order; phases that conflict are
// separated by a grid barrier, so a tile's intermediate dats are re-read from
// L2 by the next loop instead of from HBM.
// ----------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier by arrival counter and generation, with a wall-clock limit.
// On timeout the error word is set and every CTA leaves the kernel at its
// next barrier.
__device__ bool grid_barrier(unsigned* bar, int* err, long long timeout_ns, bool skip) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = bar + 1;
    volatile int* verr = err;
    const unsigned gen = *vgen;
    __threadfence();
    bool wait = true;
    if (!skip) {
      const unsigned arrived = atomicAdd(bar, 1u);
      if (arrived == gridDim.x - 1) {
        atomicExch(bar, 0u);
        __threadfence();
        atomicAdd(bar + 1, 1u);
        wait = false;
      }
    }
    if (wait) {
      const unsigned long long t0 = global_ns();
      unsigned spins = 0;
      while (*vgen == gen) {
        if (*verr) break;
        if ((++spins & 31u) == 0 && (long long)(global_ns() - t0) > timeout_ns) {
          atomicCAS(err, 0, kDevErrTimeout);
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile int*)err == 0;
}

__global__ void __launch_bounds__(kThreads, OPS_MIN_CTAS) k_skewed(const DLoop* __restrict__ loops,
                                                                   const Phase* __restrict__ phases, int nphases,
                                                                   const double* __restrict__ scal, DD* part,
                                                                   int stride, int check, int* err, unsigned* bar,
                                                                   long long timeout_ns, int skip_block) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ChainSmem& S = *reinterpret_cast<ChainSmem*>(smem_raw);
  const bool skip = (int)blockIdx.x == skip_block;
  if (threadIdx.x == 0) S.own_check = 0;
  int cur = -1;
  for (int ph = 0; ph < nphases; ++ph) {
    const Phase P = phases[ph];
    if (P.barrier && ph > 0) {
      if (!grid_barrier(bar, err, timeout_ns, skip)) return;
    }
    if (P.loop != cur) {
      __syncthreads();
      stage_loop(&S.L, loops + P.loop);
      __syncthreads();
      cur = P.loop;
    }
    red_init(S);
    run_box(S, P.box, scal, blockIdx.x, gridDim.x, check, err);
    if (S.L.nreds) flush_partials(S, part, stride, false);
  }
}

cudaError_t chain_kernels_setup() {
  cudaError_t e = cudaFuncSetAttribute(k_untiled, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kChainSmem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_skewed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kChainSmem);
}

int skewed_max_grid(int num_sms, int blocks_per_sm) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_skewed, kThreads, kChainSmem) != cudaSuccess) return 0;
  if (blocks_per_sm > 0 && blocks_per_sm < per_sm) per_sm = blocks_per_sm;
  return per_sm * num_sms;
}

cudaError_t launch_skewed(const LaunchEnv& env, const DLoop* d_loops, const Phase* d_phases, int nphases, int grid) {
  cudaError_t e = cudaMemsetAsync(env.bar, 0, 2 * sizeof(unsigned), env.stream);
  if (e != cudaSuccess) return e;
  const DLoop* a0 = d_loops;
  const Phase* a1 = d_phases;
  int a2 = nphases;
  const double* a3 = env.scal;
  DD* a4 = env.part;
  int a5 = env.part_stride;
  int a6 = env.check;
  int* a7 = env.err;
  unsigned* a8 = env.bar;
  long long a9 = env.timeout_ns;
  int a10 = env.skip_block;
  void* args[] = {&a0, &a1, &a2, &a3, &a4, &a5, &a6, &a7, &a8, &a9, &a10};
  return cudaLaunchCooperativeKernel((const void*)k_skewed, dim3(grid), dim3(kThreads), args, kChainSmem,
                                     env.stream);
}

// ----------------------------------------------------------------------------
// overlapped tiles (Sec. 4.D, with CTA tiles in place of MPI ranks): a CTA
// copies its tile's live-in footprint of every dat of the segment into
// shared memory, runs the segment's loops there on boxes grown by what later
// loops of the tile read (recomputing halo points other tiles also compute),
// and writes its owned box of every written dat to the dat's other buffer.
// Tiles never wait for one another.
// ----------------------------------------------------------------------------
using OvSmem = ChainSmemT<1>;
constexpr int kOvHeader = (int)((sizeof(OvSmem) + 15) / 16 * 16);
constexpr int kMaxSmemOptin = 232448;  // sm_103a: per-block opt-in shared memory

__global__ void __launch_bounds__(kThreads) k_overlap(const DLoop* __restrict__ loops, int nloops,
                                                      const OvDat* __restrict__ dats, int ndats,
                                                      const int* __restrict__ own, const int* __restrict__ boxes,
                                                      const int* __restrict__ foot, int ntiles,
                                                      const double* __restrict__ scal, DD* part, int stride,
                                                      int check, int* err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  OvSmem& S = *reinterpret_cast<OvSmem*>(smem_raw);
  double* area = reinterpret_cast<double*>(smem_raw + kOvHeader);
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    __syncthreads();
    for (int d = 0; d < ndats; ++d) {
      const OvDat D = dats[d];
      const int* fb = foot + ((size_t)t * ndats + d) * 6;
      copy_box<double>(fb, fb, area + D.smem_off, D.spitch, D.splane, D.src, nullptr, D.gpitch, D.gplane, true);
    }
    for (int l = 0; l < nloops; ++l) {
      const int* bx = boxes + ((size_t)t * nloops + l) * 6;
      if (bx[1] <= bx[0] || bx[3] <= bx[2] || bx[5] <= bx[4]) continue;
      __syncthreads();
      stage_loop(&S.L, loops + l);
      __syncthreads();
      if ((int)threadIdx.x < S.L.nargs) {
        DArg& A = S.L.args[threadIdx.x];
        if (A.kind == OPS_ARG_DAT) {
          const int d = A.slot;
          const int* fb = foot + ((size_t)t * ndats + d) * 6;
          A.ptr0 = area + dats[d].smem_off - (fb[0] + (int64_t)fb[2] * A.pitch + (int64_t)fb[4] * A.plane);
        }
      }
      if (threadIdx.x < 6) S.own[threadIdx.x] = own[(size_t)t * 6 + threadIdx.x];
      if (threadIdx.x == 0) S.own_check = 1;
      __syncthreads();
      red_init(S);
      run_box(S, bx, scal, 0, 1, check, err);
      __syncthreads();
      if (S.L.nreds) flush_partials(S, part, stride, false);
    }
    __syncthreads();
    const int* ob = own + (size_t)t * 6;
    for (int d = 0; d < ndats; ++d) {
      const OvDat D = dats[d];
      if (!D.written) continue;
      const int* fb = foot + ((size_t)t * ndats + d) * 6;
      copy_box<double>(ob, fb, area + D.smem_off, D.spitch, D.splane, nullptr, D.dst, D.gpitch, D.gplane, false);
    }
  }
}

int overlap_smem_area_bytes() { return (kMaxSmemOptin - kOvHeader) / 16 * 16; }

int overlap_max_grid(int num_sms, int area_bytes) {
  int per_sm = 0;
  if (cudaFuncSetAttribute(k_overlap, cudaFuncAttributeMaxDynamicSharedMemorySize, kOvHeader + area_bytes) !=
      cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_overlap, kThreads, kOvHeader + area_bytes) !=
      cudaSuccess)
    return 0;
  return per_sm * num_sms;
}

cudaError_t launch_overlap(const LaunchEnv& env, const DLoop* d_loops, int nloops, const OvDat* d_dats, int ndats,
                           const int* d_own, const int* d_boxes, const int* d_foot, int ntiles, int grid,
                           int area_bytes) {
  cudaError_t e =
      cudaFuncSetAttribute(k_overlap, cudaFuncAttributeMaxDynamicSharedMemorySize, kOvHeader + area_bytes);
  if (e != cudaSuccess) return e;
  k_overlap<<<grid, kThreads, kOvHeader + area_bytes, env.stream>>>(d_loops, nloops, d_dats, ndats, d_own, d_boxes,
                                                                    d_foot, ntiles, env.scal, env.part,
                                                                    env.part_stride, env.check, env.err);
  return cudaGetLastError();
}

}  // namespace opstile
