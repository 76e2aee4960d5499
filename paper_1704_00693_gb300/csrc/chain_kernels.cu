// Device side of the loop-chain executor for GB300 (sm_103a).
//
// Every loop body is a short program in the register IR of opstile.h,
// interpreted per grid point.  All arithmetic uses the explicitly rounded
// intrinsics (__dadd_rn, __dmul_rn, __fma_rn, __ddiv_rn) and the library is
// built with -fmad=false, so a point's value is bit-identical whatever the
// schedule: untiled, skewed (Sec. 4.B, Algorithm 2) or overlapped (Sec. 4.D).
//
// FP64 on GB300 issues about two DFMA per clock per SM, so the interpreter's
// integer work (dispatch, addressing) hides behind the FP64 pipe for any body
// with a few fma per point; light bodies (copies) are bound by HBM.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace opstile {

// ----------------------------------------------------------------------------
// compensated accumulation (Knuth's two-sum; order fixed by the launch shape)
// ----------------------------------------------------------------------------
__device__ __forceinline__ DD dd_add(DD a, double x) {
  double s = __dadd_rn(a.hi, x);
  double bp = __dsub_rn(s, a.hi);
  double e = __dadd_rn(__dsub_rn(a.hi, __dsub_rn(s, bp)), __dsub_rn(x, bp));
  return DD{s, __dadd_rn(a.lo, e)};
}
__device__ __forceinline__ DD dd_merge(DD a, DD b) {
  DD t = dd_add(a, b.hi);
  t.lo = __dadd_rn(t.lo, b.lo);
  return t;
}
__device__ __forceinline__ double red_identity(int op) {
  return op == OPS_RED_SUM ? 0.0 : (op == OPS_RED_MIN ? __longlong_as_double(0x7ff0000000000000ll)
                                                       : __longlong_as_double(0xfff0000000000000ll));
}
__device__ __forceinline__ DD red_combine(int op, DD a, DD b) {
  if (op == OPS_RED_SUM) return dd_merge(a, b);
  if (op == OPS_RED_MIN) return DD{(b.hi < a.hi) ? b.hi : a.hi, 0.0};
  return DD{(b.hi > a.hi) ? b.hi : a.hi, 0.0};
}
__device__ __forceinline__ DD shfl_down_dd(DD v, int o) {
  return DD{__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)};
}

// Block-wide combine in a fixed tree; result valid in thread 0.
__device__ DD block_combine(int op, DD v, DD* sh) {
  for (int o = 16; o > 0; o >>= 1) v = red_combine(op, v, shfl_down_dd(v, o));
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    v = lane < nw ? sh[lane] : DD{red_identity(op), 0.0};
    for (int o = 16; o > 0; o >>= 1) v = red_combine(op, v, shfl_down_dd(v, o));
  }
  return v;
}

// ----------------------------------------------------------------------------
// one grid point of one loop body
// ----------------------------------------------------------------------------
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

__device__ __forceinline__ void run_point(const DLoop& L, int x, int y, int z, const double* __restrict__ scal,
                                          DD* acc) {
  double r[kNReg];
#pragma unroll
  for (int i = 0; i < kNReg; ++i) r[i] = 0.0;
  const int nins = L.nins;
  for (int pc = 0; pc < nins; ++pc) {
    const int* I = L.ins[pc];
    const int op = I[0], d = I[1], a = I[2], b = I[3];
    switch (op) {
      case OPS_IR_LD: {
        const DArg& A = L.args[a];
        if (A.kind == OPS_ARG_SCALAR) {
          r[d] = scal[A.slot];
        } else {
          r[d] = A.ptr0[x + y * A.pitch + z * A.plane + A.off[b]];
        }
        break;
      }
      case OPS_IR_CST: r[d] = L.K[a]; break;
      case OPS_IR_ADD: r[d] = __dadd_rn(r[a], r[b]); break;
      case OPS_IR_SUB: r[d] = __dsub_rn(r[a], r[b]); break;
      case OPS_IR_MUL: r[d] = __dmul_rn(r[a], r[b]); break;
      case OPS_IR_FMA: r[d] = __fma_rn(r[a], r[b], r[I[4]]); break;
      case OPS_IR_DIV: r[d] = __ddiv_rn(r[a], r[b]); break;
      case OPS_IR_MIN: r[d] = (r[b] < r[a]) ? r[b] : r[a]; break;
      case OPS_IR_MAX: r[d] = (r[b] > r[a]) ? r[b] : r[a]; break;
      case OPS_IR_SGT: r[d] = (r[a] > r[b]) ? r[I[4]] : r[I[5]]; break;
      case OPS_IR_WSUM:
      case OPS_IR_WACC: {
        const DArg& A = L.args[a];
        const double* p = A.ptr0 + (x + y * A.pitch + z * A.plane);
        const double* Kb = L.K + b;
        const int n = A.npts;
        double t = r[d];
        int q = 0;
        if (op == OPS_IR_WSUM) {
          t = __dmul_rn(Kb[0], p[A.off[0]]);
          q = 1;
        }
        for (; q + 4 <= n; q += 4) {
          const double v0 = p[A.off[q]], v1 = p[A.off[q + 1]], v2 = p[A.off[q + 2]], v3 = p[A.off[q + 3]];
          t = __fma_rn(Kb[q], v0, t);
          t = __fma_rn(Kb[q + 1], v1, t);
          t = __fma_rn(Kb[q + 2], v2, t);
          t = __fma_rn(Kb[q + 3], v3, t);
        }
        for (; q < n; ++q) t = __fma_rn(Kb[q], p[A.off[q]], t);
        r[d] = t;
        break;
      }
      case OPS_IR_POLY: {
        const int c = I[4];
        double t = L.K[b + c];
        for (int i = c - 1; i >= 0; --i) t = __fma_rn(t, r[a], L.K[b + i]);
        r[d] = t;
        break;
      }
      case OPS_IR_ST: {
        const DArg& A = L.args[d];
        double* q = A.ptr0 + (x + y * A.pitch + z * A.plane);
        if (A.access == OPS_INC)
          *q = __dadd_rn(*q, r[a]);
        else
          *q = r[a];
        break;
      }
      case OPS_IR_RED: {
        const int k = L.args[d].slot;
        const int rop = L.red_op[k];
        if (rop == OPS_RED_SUM)
          acc[k] = dd_add(acc[k], r[a]);
        else if (rop == OPS_RED_MIN)
          acc[k].hi = (r[a] < acc[k].hi) ? r[a] : acc[k].hi;
        else
          acc[k].hi = (r[a] > acc[k].hi) ? r[a] : acc[k].hi;
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
static_assert(sizeof(DLoop) % sizeof(int4) == 0, "DLoop must be a multiple of 16 bytes");

// Run this CTA's share of `box` for the staged loop L.  Rows of at least 128
// points are split into 256-wide x chunks (coalesced); thinner boxes are
// flattened.  `part` is this CTA's unit index and `nparts` the number of CTAs.
__device__ __forceinline__ void run_box(const DLoop& L, const int* box, const double* __restrict__ scal, DD* acc,
                                        int part, int nparts, int check, int* err) {
  const int x0 = box[0], nx = box[1] - box[0];
  const int y0 = box[2], ny = box[3] - box[2];
  const int z0 = box[4], nz = box[5] - box[4];
  if (nx <= 0 || ny <= 0 || nz <= 0) return;
  if (nx >= 128) {
    const int xch = (nx + kThreads - 1) / kThreads;
    const long long units = (long long)xch * ny * nz;
    for (long long u = part; u < units; u += nparts) {
      const int xc = (int)(u % xch);
      const long long row = u / xch;
      const int y = y0 + (int)(row % ny);
      const int z = z0 + (int)(row / ny);
      const int x = x0 + xc * kThreads + (int)threadIdx.x;
      if (x < x0 + nx) {
        if (check && !point_ok(L, x, y, z)) {
          atomicCAS(err, 0, kDevErrBounds);
          continue;
        }
        run_point(L, x, y, z, scal, acc);
      }
    }
  } else {
    const long long npts = (long long)nx * ny * nz;
    for (long long p = (long long)part * kThreads + threadIdx.x; p < npts; p += (long long)nparts * kThreads) {
      const int x = x0 + (int)(p % nx);
      const long long row = p / nx;
      const int y = y0 + (int)(row % ny);
      const int z = z0 + (int)(row / ny);
      if (check && !point_ok(L, x, y, z)) {
        atomicCAS(err, 0, kDevErrBounds);
        continue;
      }
      run_point(L, x, y, z, scal, acc);
    }
  }
}

// Fold this CTA's reduction accumulators into its partial column (assign or combine).
__device__ __forceinline__ void flush_partials(const DLoop& L, DD* acc, DD* part, int stride, DD* sh, bool assign) {
  for (int k = 0; k < L.nreds; ++k) {
    const int op = L.red_op[k];
    DD v = block_combine(op, acc[k], sh);
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
__global__ void __launch_bounds__(kThreads) k_untiled(const DLoop* __restrict__ gL, int bx0, int bx1, int by0,
                                                      int by1, int bz0, int bz1, const double* __restrict__ scal,
                                                      DD* part, int stride, int check, int* err) {
  __shared__ __align__(16) DLoop L;
  __shared__ DD sh[32];
  stage_loop(&L, gL);
  __syncthreads();
  DD acc[OPS_MAX_REDS_PER_LOOP];
  for (int k = 0; k < OPS_MAX_REDS_PER_LOOP; ++k) acc[k] = DD{red_identity(k < L.nreds ? L.red_op[k] : 0), 0.0};
  const int box[6] = {bx0, bx1, by0, by1, bz0, bz1};
  run_box(L, box, scal, acc, blockIdx.x, gridDim.x, check, err);
  if (L.nreds) flush_partials(L, acc, part, stride, sh, true);
}

int untiled_grid(const LaunchEnv& env, const int* box) {
  const long long nx = box[1] - box[0], ny = box[3] - box[2], nz = box[5] - box[4];
  long long units = nx >= 128 ? ((nx + kThreads - 1) / kThreads) * ny * nz : (nx * ny * nz + kThreads - 1) / kThreads;
  long long cap = (long long)env.num_sms * 8;
  if (units < 1) units = 1;
  return (int)(units < cap ? units : cap);
}

cudaError_t launch_untiled(const LaunchEnv& env, const DLoop* d_loop, const int* box, int grid) {
  k_untiled<<<grid, kThreads, 0, env.stream>>>(d_loop, box[0], box[1], box[2], box[3], box[4], box[5], env.scal,
                                               env.part, env.part_stride, env.check, env.err);
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
__global__ void __launch_bounds__(kThreads) k_fold(const DD* __restrict__ part, int stride, const FoldRow* rows,
                                                   int row0, int nused, double* scal) {
  __shared__ DD sh[32];
  const int r = row0 + blockIdx.x;
  const int op = rows[r].op;
  DD v{red_identity(op), 0.0};
  for (int i = threadIdx.x; i < nused; i += blockDim.x) v = red_combine(op, v, part[(size_t)r * stride + i]);
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

cudaError_t launch_fold(const LaunchEnv& env, int row0, int nrows, int grid_used) {
  if (nrows <= 0) return cudaSuccess;
  k_fold<<<nrows, kThreads, 0, env.stream>>>(env.part, env.part_stride, env.rows, row0, grid_used, env.scal);
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

// Sense-by-generation grid barrier with a wall-clock limit.  On timeout the
// error word is set and every CTA leaves the kernel at its next barrier.
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

__global__ void __launch_bounds__(kThreads) k_skewed(const DLoop* __restrict__ loops, const Phase* __restrict__ phases,
                                                     int nphases, const double* __restrict__ scal, DD* part,
                                                     int stride, int check, int* err, unsigned* bar,
                                                     long long timeout_ns, int skip_block) {
  __shared__ __align__(16) DLoop L;
  __shared__ DD sh[32];
  const bool skip = (int)blockIdx.x == skip_block;
  int cur = -1;
  DD acc[OPS_MAX_REDS_PER_LOOP];
  for (int ph = 0; ph < nphases; ++ph) {
    const Phase P = phases[ph];
    if (P.barrier && ph > 0) {
      if (!grid_barrier(bar, err, timeout_ns, skip)) return;
    }
    if (P.loop != cur) {
      __syncthreads();
      stage_loop(&L, loops + P.loop);
      __syncthreads();
      cur = P.loop;
    }
    for (int k = 0; k < OPS_MAX_REDS_PER_LOOP; ++k) acc[k] = DD{red_identity(k < L.nreds ? L.red_op[k] : 0), 0.0};
    run_box(L, P.box, scal, acc, blockIdx.x, gridDim.x, check, err);
    if (L.nreds) flush_partials(L, acc, part, stride, sh, false);
  }
}

int skewed_max_grid(int num_sms, int blocks_per_sm) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_skewed, kThreads, 0) != cudaSuccess) return 0;
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
  return cudaLaunchCooperativeKernel((const void*)k_skewed, dim3(grid), dim3(kThreads), args, 0, env.stream);
}

}  // namespace opstile
