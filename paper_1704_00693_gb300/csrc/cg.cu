// Batched CG for the 5-point heat-conduction operator (TeaLeaf-shaped solves,
// Sec. 5 and Sec. 6.D), GB300 design:
//   - the operator is (A u)_c = d_c u_c - sum_f k_f u_nb over the four faces,
//     k_f the harmonic mean of the two cells' conductivity (a boundary face
//     takes the cell's own), d_c = 1 + sum_f k_f, neighbours outside are 0;
//   - mixed precision: the bandwidth-bound sweeps (matvec, axpy) run in FP32
//     with FP32 copies of the face coefficients; dot products accumulate the
//     (exact) FP64 products of FP32 values with one FP64 fma per term per
//     thread, then fixed-order FP64 trees over threads, units and problems
//     (compensated two-sums per term, or long dependent chains of them, would
//     make the solver FP64-latency-bound on GB300); the residual
//     r = b - A x, its norm and the correction x += |r| d are FP64
//     (iterative refinement);
//   - in the FP32 inner iterations the direction update p = r + beta p is
//     fused into the next matvec: each thread recomputes it at the five
//     stencil points from r and the previous direction (double-buffered), so
//     an inner iteration is two sweeps (FP64 iterations keep a third sweep:
//     the recomputation would cost FP64 fma on GB300's narrow FP64 pipe);
//   - every problem is a state machine advanced by one CG iteration per
//     "tick" of five kernels (sweep, scalars, sweep, scalars, and a third
//     sweep that only applies the refinement correction), so many
//     grids of different sizes share every launch; a problem's reductions use
//     only its own work units in a fixed order, so its result does not depend
//     on what else is in the batch.
#include <cuda_runtime.h>

#include <array>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "cg.h"

namespace opstile {

constexpr int kCgThreads = 256;

// Work-unit size in points (whole rows where they fit) and the sweep grid:
// CTAs per SM, 0 = as many as are resident at once.  OPSTILE_CG_UNIT and
// OPSTILE_CG_GRID override the defaults, 4096 points and 16 CTAs per SM:
// more CTAs than fit at once let the block scheduler even out the last wave
// (measured on GB300 for one 4000^2 solve and for the served mix).
static int cg_env(const char* name, int def, int lo, int hi) {
  const char* e = getenv(name);
  if (!e || !*e) return def;
  const int v = atoi(e);
  return v < lo ? lo : (v > hi ? hi : v);
}
static int cg_unit_pts() {
  static const int v = cg_env("OPSTILE_CG_UNIT", 4096, 256, 1 << 20);
  return v;
}
static int cg_grid_per_sm() {
  static const int v = cg_env("OPSTILE_CG_GRID", 16, 0, 64);
  return v;
}

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------
// block sum of doubles in a fixed tree (plain FP64: short dependent chains,
// which matter on GB300's slow FP64 pipe), valid in thread 0
__device__ double cg_block_sum_d(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_down_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    v = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_down_sync(0xffffffffu, v, o));
  }
  __syncthreads();
  return v;
}
// ---------------------------------------------------------------------------
// the operator at one cell, in the fixed term order
// ---------------------------------------------------------------------------
template <class T>
struct OpView {
  const T *kx, *ky, *dg;
  int n;
};
__device__ __forceinline__ double av64(const OpView<double>& A, const double* u, int j, int i) {
  const int n = A.n;
  const int64_t c = (int64_t)j * n + i;
  const double uW = i > 0 ? u[c - 1] : 0.0;
  const double uE = i < n - 1 ? u[c + 1] : 0.0;
  const double uS = j > 0 ? u[c - n] : 0.0;
  const double uN = j < n - 1 ? u[c + n] : 0.0;
  const int64_t fx = (int64_t)j * (n + 1) + i, fy = (int64_t)j * n + i;
  double t = __dmul_rn(A.dg[c], u[c]);
  t = __fma_rn(-A.kx[fx], uW, t);
  t = __fma_rn(-A.kx[fx + 1], uE, t);
  t = __fma_rn(-A.ky[fy], uS, t);
  t = __fma_rn(-A.ky[fy + n], uN, t);
  return t;
}
__device__ __forceinline__ float av32(const OpView<float>& A, const float* u, int j, int i) {
  const int n = A.n;
  const int64_t c = (int64_t)j * n + i;
  const float uW = i > 0 ? u[c - 1] : 0.0f;
  const float uE = i < n - 1 ? u[c + 1] : 0.0f;
  const float uS = j > 0 ? u[c - n] : 0.0f;
  const float uN = j < n - 1 ? u[c + n] : 0.0f;
  const int64_t fx = (int64_t)j * (n + 1) + i, fy = (int64_t)j * n + i;
  float t = __fmul_rn(A.dg[c], u[c]);
  t = __fmaf_rn(-A.kx[fx], uW, t);
  t = __fmaf_rn(-A.kx[fx + 1], uE, t);
  t = __fmaf_rn(-A.ky[fy], uS, t);
  t = __fmaf_rn(-A.ky[fy + n], uN, t);
  return t;
}

// The operator at one cell from the five values of its stencil (outside: 0),
// in the term order of av32.
__device__ __forceinline__ float av32v(const OpView<float>& A, int j, int i, float uC, float uW, float uE, float uS,
                                       float uN) {
  const int n = A.n;
  const int64_t c = (int64_t)j * n + i, fx = (int64_t)j * (n + 1) + i, fy = (int64_t)j * n + i;
  float t = __fmul_rn(A.dg[c], uC);
  t = __fmaf_rn(-A.kx[fx], uW, t);
  t = __fmaf_rn(-A.kx[fx + 1], uE, t);
  t = __fmaf_rn(-A.ky[fy], uS, t);
  t = __fmaf_rn(-A.ky[fy + n], uN, t);
  return t;
}

// Visit the points of a unit: rows [j0, j0+nr) x columns [c0, c0+w); narrow
// units put several rows side by side in the block (division once per unit).
template <class F>
__device__ __forceinline__ void for_unit(const CgUnit& U, F f) {
  if (U.w >= kCgThreads) {
    for (int r = 0; r < U.nr; ++r)
      for (int c = threadIdx.x; c < U.w; c += kCgThreads) f(U.j0 + r, U.c0 + c);
  } else {
    const int rpp = kCgThreads / U.w;
    const int tr = threadIdx.x / U.w, tc = threadIdx.x - tr * U.w;
    if (tr < rpp)
      for (int r = tr; r < U.nr; r += rpp) f(U.j0 + r, U.c0 + tc);
  }
}

// FP32 -> FP64 widening on the integer pipe: the double's bits are assembled
// from the float's sign, exponent (rebiased by 1023 - 127) and mantissa
// (shifted up 29 bits); a subnormal float is normalised (its leading one
// moved to the implicit bit), zero keeps its sign, infinity and NaN keep the
// all-ones exponent.  Exact for every input, and branch-free: on GB300 the
// FP64 pipe issues about two operations per clock per SM, so the FP32 sweeps
// keep it for the one FP64 fma per dot-product term.
__device__ __forceinline__ double widen(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  const unsigned sh = (unsigned)__clz((int)m) - 8u;  // subnormal: shifts that bring the leading one to bit 23
  const bool sub = e == 0u;
  const unsigned E = sub ? (m ? 897u - sh : 0u) : (e == 0xffu ? 2047u : e + 896u);
  const unsigned M = (sub && m) ? (m << sh) & 0x7fffffu : m;
  return __hiloint2double((int)((u & 0x80000000u) | (E << 20) | (M >> 3)), (int)(M << 29));
}

// The same points, kCgPts at a time per thread where the unit allows:
// point k of a group feeds accumulator a[k % 4] (a fixed assignment), so
// four independent FP64 chains and kCgPts points' loads are in flight per
// thread.  The callers pass the stored-to arrays as __restrict__
// parameters, so the loads of a group are not held back by its stores.
// (Eight points per group measured slower on GB300 than four.)
constexpr int kCgPts = 4;
template <class F>
__device__ __forceinline__ void for_unit4(const CgUnit& U, double* a, F f) {
  if (U.w >= kCgThreads) {
    for (int r = 0; r < U.nr; ++r) {
      const int j = U.j0 + r;
      for (int c = threadIdx.x; c < U.w; c += kCgPts * kCgThreads) {
#pragma unroll
        for (int k = 0; k < kCgPts; ++k)
          if (c + k * kCgThreads < U.w) f(j, U.c0 + c + k * kCgThreads, a[k & 3]);
      }
    }
  } else {
    const int rpp = kCgThreads / U.w;
    const int tr = threadIdx.x / U.w, tc = threadIdx.x - tr * U.w;
    if (tr < rpp)
      for (int r = tr; r < U.nr; r += kCgPts * rpp) {
#pragma unroll
        for (int k = 0; k < kCgPts; ++k)
          if (r + k * rpp < U.nr) f(U.j0 + r + k * rpp, U.c0 + tc, a[k & 3]);
      }
  }
}
__device__ __forceinline__ double sum4(const double* a) { return __dadd_rn(__dadd_rn(a[0], a[1]), __dadd_rn(a[2], a[3])); }

__device__ __forceinline__ double hmean(double a, double b) {
  return __ddiv_rn(__dmul_rn(__dmul_rn(2.0, a), b), __dadd_rn(a, b));
}

// ---------------------------------------------------------------------------
// set-up: face coefficients from the conductivity (held in P.r on entry)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kCgThreads) k_cg_setup(CgProb* probs, const CgUnit* units, int u0, int u1) {
  for (int u = u0 + blockIdx.x; u < u1; u += gridDim.x) {
    const CgUnit U = units[u];
    CgProb& P = probs[U.prob];
    const int n = P.n;
    const double* kap = P.r;
    for_unit(U, [&](int j, int i) {
      const int64_t c = (int64_t)j * n + i;
      const double kc = kap[c];
      const double kw = i > 0 ? hmean(kap[c - 1], kc) : kc;
      const double ks = j > 0 ? hmean(kap[c - n], kc) : kc;
      const int64_t fx = (int64_t)j * (n + 1) + i, fy = (int64_t)j * n + i;
      P.kx[fx] = kw;
      P.ky[fy] = ks;
      P.kx32[fx] = (float)kw;
      P.ky32[fy] = (float)ks;
      if (i == n - 1) {
        P.kx[fx + 1] = kc;
        P.kx32[fx + 1] = (float)kc;
      }
      if (j == n - 1) {
        P.ky[fy + n] = kc;
        P.ky32[fy + n] = (float)kc;
      }
    });
  }
}
// diagonal once every face is known
__global__ void __launch_bounds__(kCgThreads) k_cg_setup2(CgProb* probs, const CgUnit* units, int u0, int u1) {
  for (int u = u0 + blockIdx.x; u < u1; u += gridDim.x) {
    const CgUnit U = units[u];
    CgProb& P = probs[U.prob];
    const int n = P.n;
    for_unit(U, [&](int j, int i) {
      const int64_t c = (int64_t)j * n + i;
      const int64_t fx = (int64_t)j * (n + 1) + i, fy = (int64_t)j * n + i;
      double d = __dadd_rn(1.0, P.kx[fx]);
      d = __dadd_rn(d, P.kx[fx + 1]);
      d = __dadd_rn(d, P.ky[fy]);
      d = __dadd_rn(d, P.ky[fy + n]);
      P.dg[c] = d;
      P.dg32[c] = (float)d;
      P.x[c] = 0.0;
    });
  }
}

// ---------------------------------------------------------------------------
// tick kernels
// ---------------------------------------------------------------------------
// A sweeps, one function per state (stored-to arrays are __restrict__)
__device__ __forceinline__ void a_residual(const CgUnit& U, const OpView<double>& A, const double* x,
                                           const double* b, double* __restrict__ r, int n, double* acc) {
  for_unit4(U, acc, [&](int j, int i, double& a) {
    const int64_t c = (int64_t)j * n + i;
    const double rc = __dsub_rn(b[c], av64(A, x, j, i));
    r[c] = rc;
    a = __fma_rn(rc, rc, a);
  });
}
// The direction update p = r + beta p_old is fused into the matvec: every
// thread recomputes it at the five stencil points (the same fma the owner
// of each point evaluates, so the values are identical), writes the new
// direction of its own cell to the other buffer, and applies A to it.
__device__ __forceinline__ void a_inner(const CgUnit& U, const OpView<float>& A, float bf, const float* po,
                                        const float* r, float* __restrict__ pn, float* __restrict__ w, int n,
                                        double* acc) {
  for_unit4(U, acc, [&](int j, int i, double& a) {
    const int64_t c = (int64_t)j * n + i;
    const float pC = __fmaf_rn(bf, po[c], r[c]);
    const float pW = i > 0 ? __fmaf_rn(bf, po[c - 1], r[c - 1]) : 0.0f;
    const float pE = i < n - 1 ? __fmaf_rn(bf, po[c + 1], r[c + 1]) : 0.0f;
    const float pS = j > 0 ? __fmaf_rn(bf, po[c - n], r[c - n]) : 0.0f;
    const float pN = j < n - 1 ? __fmaf_rn(bf, po[c + n], r[c + n]) : 0.0f;
    const float wc = av32v(A, j, i, pC, pW, pE, pS, pN);
    pn[c] = pC;
    w[c] = wc;
    a = __fma_rn(widen(pC), widen(wc), a);
  });
}
// FP64 iterations keep the update in its own sweep: recomputing it at five
// points would add four FP64 fma per cell on GB300's narrow FP64 pipe.
__device__ __forceinline__ void a_cg64(const CgUnit& U, const OpView<double>& A, const double* p,
                                       double* __restrict__ w, int n, double* acc) {
  for_unit4(U, acc, [&](int j, int i, double& a) {
    const int64_t c = (int64_t)j * n + i;
    const double wc = av64(A, p, j, i);
    w[c] = wc;
    a = __fma_rn(p[c], wc, a);
  });
}

// A: FP64 residual r = b - A x and |r|^2 (OUTER, FINISH); w = A p and p.w (INNER, CG64)
__global__ void __launch_bounds__(kCgThreads) k_cg_a(CgProb* probs, const CgUnit* units, const int* cnt, DD* part) {
  __shared__ double sh[32];
  const int nunits = cnt[0];
  for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
    const CgUnit U = units[u];
    const CgProb& P = probs[U.prob];
    const int st = P.state, n = P.n;
    // per-thread FP64 fma accumulation in four fixed chains, then a fixed FP64 tree
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    if (st == CG_OUTER || st == CG_FINISH)
      a_residual(U, OpView<double>{P.kx, P.ky, P.dg, n}, P.x, P.b, P.r, n, acc);
    else if (st == CG_INNER)
      a_inner(U, OpView<float>{P.kx32, P.ky32, P.dg32, n}, (float)P.beta, P.pp ? P.p32b : P.p32, P.r32,
              P.pp ? P.p32 : P.p32b, P.w32, n, acc);
    else if (st == CG64)
      a_cg64(U, OpView<double>{P.kx, P.ky, P.dg, n}, P.p64, P.w64, n, acc);
    const double tot = cg_block_sum_d(sum4(acc), sh);
    if (threadIdx.x == 0) part[u] = DD{tot, 0.0};
  }
}

// B sweeps, one function per state
__device__ __forceinline__ void b_init(const CgUnit& U, double inv, const double* r, float* __restrict__ r32,
                                       float* __restrict__ p32, float* __restrict__ d32, int n, double* acc) {
  for_unit4(U, acc, [&](int j, int i, double& a) {
    const int64_t c = (int64_t)j * n + i;
    const float rs = (float)__dmul_rn(r[c], inv);
    r32[c] = rs;
    p32[c] = rs;
    d32[c] = 0.0f;
    const double rd = widen(rs);
    a = __fma_rn(rd, rd, a);
  });
}
__device__ __forceinline__ void b_inner(const CgUnit& U, float af, const float* p32, const float* w32,
                                        float* __restrict__ r32, float* __restrict__ d32, int n, double* acc) {
  for_unit4(U, acc, [&](int j, int i, double& a) {
    const int64_t c = (int64_t)j * n + i;
    d32[c] = __fmaf_rn(af, p32[c], d32[c]);
    const float r = __fmaf_rn(-af, w32[c], r32[c]);
    r32[c] = r;
    const double rd = widen(r);
    a = __fma_rn(rd, rd, a);
  });
}
__device__ __forceinline__ void b_cg64_init(const CgUnit& U, const double* b, double* __restrict__ x,
                                            double* __restrict__ r, double* __restrict__ p, int n, double* acc) {
  for_unit4(U, acc, [&](int j, int i, double& a) {
    const int64_t c = (int64_t)j * n + i;
    const double bc = b[c];
    x[c] = 0.0;
    r[c] = bc;
    p[c] = bc;
    a = __fma_rn(bc, bc, a);
  });
}
__device__ __forceinline__ void b_cg64(const CgUnit& U, double al, const double* p, const double* w,
                                       double* __restrict__ x, double* __restrict__ r, int n, double* acc) {
  for_unit4(U, acc, [&](int j, int i, double& a) {
    const int64_t c = (int64_t)j * n + i;
    x[c] = __fma_rn(al, p[c], x[c]);
    const double rc = __fma_rn(-al, w[c], r[c]);
    r[c] = rc;
    a = __fma_rn(rc, rc, a);
  });
}

// B: INIT (scaled residual into the FP32 inner vectors), INNER / CG64 updates
__global__ void __launch_bounds__(kCgThreads) k_cg_b(CgProb* probs, const CgUnit* units, const int* cnt, DD* part) {
  __shared__ double sh[32];
  const int nunits = cnt[0];
  for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
    const CgUnit U = units[u];
    const CgProb& P = probs[U.prob];
    const int st = P.state, n = P.n;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    if (st == CG_INIT)
      b_init(U, __ddiv_rn(1.0, P.nr), P.r, P.r32, P.p32, P.d32, n, acc);
    else if (st == CG_INNER)
      b_inner(U, (float)P.alpha, P.pp ? P.p32 : P.p32b, P.w32, P.r32, P.d32, n, acc);
    else if (st == CG64_INIT)
      b_cg64_init(U, P.b, P.x, P.r, P.p64, n, acc);
    else if (st == CG64)
      b_cg64(U, P.alpha, P.p64, P.w64, P.x, P.r, n, acc);
    const double tot = cg_block_sum_d(sum4(acc), sh);
    if (threadIdx.x == 0) part[u] = DD{tot, 0.0};
  }
}

// C sweep: the refinement correction x += |r| d (FINISH) and the FP64
// direction update p = r + beta p (CG64); the inner (FP32) direction update
// is fused into the next A sweep
__device__ __forceinline__ void c_cg64(const CgUnit& U, double bt, const double* r, double* __restrict__ p, int n) {
  double dummy[4];
  for_unit4(U, dummy, [&](int j, int i, double&) {
    const int64_t c = (int64_t)j * n + i;
    p[c] = __fma_rn(bt, p[c], r[c]);
  });
}
__device__ __forceinline__ void c_finish(const CgUnit& U, double nr, const float* d32, double* __restrict__ x,
                                         int n) {
  double dummy[4];
  for_unit4(U, dummy, [&](int j, int i, double&) {
    const int64_t c = (int64_t)j * n + i;
    x[c] = __fma_rn(nr, (double)d32[c], x[c]);
  });
}

__global__ void __launch_bounds__(kCgThreads) k_cg_c(CgProb* probs, const CgUnit* units, const int* cnt) {
  const int nunits = cnt[0];
  for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
    const CgUnit U = units[u];
    const CgProb& P = probs[U.prob];
    if (P.state == CG_FINISH)
      c_finish(U, P.nr, P.d32, P.x, P.n);
    else if (P.state == CG64)
      c_cg64(U, P.beta, P.r, P.p64, P.n);
  }
}

// One operator application for one slot: FP64 reads u from x and writes
// A u to r; FP32 reads p32 and writes w32.
__global__ void __launch_bounds__(kCgThreads) k_cg_apply(const CgProb* probs, const CgUnit* units, int u0, int u1,
                                                         int prec) {
  for (int u = u0 + blockIdx.x; u < u1; u += gridDim.x) {
    const CgUnit U = units[u];
    const CgProb& P = probs[U.prob];
    const int n = P.n;
    if (prec == 0) {
      const OpView<double> A{P.kx, P.ky, P.dg, n};
      const double* x = P.x;
      double* r = P.r;
      for_unit(U, [&](int j, int i) { r[(int64_t)j * n + i] = av64(A, x, j, i); });
    } else {
      const OpView<float> A{P.kx32, P.ky32, P.dg32, n};
      const float* p = P.p32;
      float* w = P.w32;
      for_unit(U, [&](int j, int i) { w[(int64_t)j * n + i] = av32(A, p, j, i); });
    }
  }
}

// Sum of a problem's unit partials in a fixed order (one block per problem,
// thread-strided then a fixed tree); valid in thread 0.
__device__ __forceinline__ double block_partial_sum(const DD* part, int u0, int u1, double* sh) {
  double v = 0.0;
  for (int u = u0 + (int)threadIdx.x; u < u1; u += blockDim.x) v = __dadd_rn(v, __dadd_rn(part[u].hi, part[u].lo));
  return cg_block_sum_d(v, sh);
}

// Scalars after kernel A.
__global__ void k_cg_s1(CgProb* probs, const int2* ranges, const int* cnt, const DD* part) {
  __shared__ double sh[32];
  const int p = blockIdx.x;
  if (p >= cnt[1]) return;
  CgProb& P = probs[p];
  const int st = P.state;  // uniform over the block
  if (st != CG_OUTER && st != CG_FINISH && st != CG_INNER && st != CG64) return;
  const double s = block_partial_sum(part, ranges[p].x, ranges[p].y, sh);
  if (threadIdx.x != 0) return;
  if (st == CG_OUTER || st == CG_FINISH) {
    if (st == CG_FINISH) ++P.outer;
    const double nr = sqrt(s);
    if (P.outer == 0) P.nb = nr;
    const double rel = P.nb > 0.0 ? nr / P.nb : 0.0;
    P.rel = rel;
    if (rel <= P.tol) {
      P.conv = 1;
      P.state = CG_DONE;
    } else if (P.outer >= P.maxouter || P.it >= P.maxit) {
      P.state = CG_DONE;
    } else {
      P.nr = nr;
      P.state = CG_INIT;
      P.pp = 0;  // the inner solve starts from buffer 0, which the INIT sweep fills with r
    }
  } else {
    P.alpha = P.rho / s;
  }
}

// Scalars after kernel B.
__global__ void k_cg_s2(CgProb* probs, const int2* ranges, const int* cnt, const DD* part) {
  __shared__ double sh[32];
  const int p = blockIdx.x;
  if (p >= cnt[1]) return;
  CgProb& P = probs[p];
  const int st = P.state;  // uniform over the block
  if (st != CG_INIT && st != CG_INNER && st != CG64_INIT && st != CG64) return;
  const double s = block_partial_sum(part, ranges[p].x, ranges[p].y, sh);
  if (threadIdx.x != 0) return;
  if (st == CG_INIT) {
    P.rho = s;
    P.rho0 = s;
    P.beta = 0.0;  // the first direction of every inner solve is r itself
    P.state = s > 0.0 ? CG_INNER : CG_FINISH;
  } else if (st == CG_INNER) {
    ++P.it;
    if (sqrt(s) <= P.inner_tol * sqrt(P.rho0) || P.it >= P.maxit) {
      P.state = CG_FINISH;
    } else {
      P.beta = s / P.rho;
      P.rho = s;
      P.pp ^= 1;  // the direction the A sweep wrote becomes the old one
    }
  } else if (st == CG64_INIT) {
    P.rho = s;
    P.nb = sqrt(s);
    P.rel = 1.0;
    if (s == 0.0) {
      P.rel = 0.0;
      P.conv = 1;
      P.state = CG_DONE;
    } else {
      P.state = CG64;
    }
  } else {
    ++P.it;
    P.beta = s / P.rho;
    P.rho = s;
    P.rel = sqrt(s) / P.nb;
    if (sqrt(s) <= P.tol * P.nb) {
      P.conv = 1;
      P.state = CG_DONE;
    } else if (P.it >= P.maxit) {
      P.state = CG_DONE;
    }
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {
size_t al256(size_t b) { return (b + 255) / 256 * 256; }
}  // namespace

int64_t cg_problem_bytes(int n) {
  const size_t N = (size_t)n * n, F = (size_t)n * (n + 1);
  return (int64_t)(5 * al256(8 * N) + 2 * al256(8 * F) + al256(8 * N) + 2 * al256(4 * F) + 6 * al256(4 * N));
}

CgBatch::CgBatch(cudaStream_t stream, int num_sms) : stream_(stream), num_sms_(num_sms) {}

CgBatch::CgBatch(cudaStream_t stream, int num_sms, int max_slots, int max_units)
    : stream_(stream), num_sms_(num_sms), fixed_(true) {
  // every table at its final size, once: adding and removing problems then
  // never allocates, and the captured tick graph stays valid
  dprob_cap_ = std::max(1, max_slots);
  dranges_cap_ = dprob_cap_;
  dunits_cap_ = std::max(1, max_units);
  dpart_cap_ = dunits_cap_;
  if (cudaMalloc(&dprob_, sizeof(CgProb) * dprob_cap_) != cudaSuccess ||
      cudaMalloc(&dranges_, sizeof(int2) * dranges_cap_) != cudaSuccess ||
      cudaMalloc(&dunits_, sizeof(CgUnit) * dunits_cap_) != cudaSuccess ||
      cudaMalloc(&dpart_, sizeof(DD) * dpart_cap_) != cudaSuccess || cudaMalloc(&dcnt_, 2 * sizeof(int)) != cudaSuccess)
    init_error_ = cudaErrorMemoryAllocation;
  else if (cudaMemsetAsync(dprob_, 0, sizeof(CgProb) * dprob_cap_, stream_) != cudaSuccess ||
           cudaMemsetAsync(dcnt_, 0, 2 * sizeof(int), stream_) != cudaSuccess)
    init_error_ = cudaErrorUnknown;
}

CgBatch::~CgBatch() {
  cudaStreamSynchronize(stream_);
  if (gexec_) cudaGraphExecDestroy(gexec_);
  cudaFree(dprob_);
  cudaFree(dunits_);
  cudaFree(dranges_);
  cudaFree(dpart_);
  cudaFree(dcnt_);
}

int cg_unit_count(int n) {
  const int pts = cg_unit_pts();
  if (n > pts) return n * ((n + pts - 1) / pts);
  const int nr = std::max(1, pts / n);
  return (n + nr - 1) / nr;
}

// Units of whole rows holding about cg_unit_pts() cells (rows wider than
// that are cut into column chunks); they depend only on n, never on the batch.
static void units_for(int slot, int n, std::vector<CgUnit>& out) {
  const int pts = cg_unit_pts();
  if (n > pts) {
    for (int j = 0; j < n; ++j)
      for (int c0 = 0; c0 < n; c0 += pts) out.push_back(CgUnit{slot, j, 1, c0, std::min(pts, n - c0)});
  } else {
    const int nr = std::max(1, pts / n);
    for (int j = 0; j < n; j += nr) out.push_back(CgUnit{slot, j, std::min(nr, n - j), 0, n});
  }
}

int CgBatch::add(int n, const double* kappa, const double* rhs, double tol, int prec, double inner_tol, int maxit,
                 int maxouter, void* slab) {
  int slot = -1;
  for (size_t i = 0; i < live_.size(); ++i)
    if (!live_[i]) {
      slot = (int)i;
      break;
    }
  if (slot < 0) {
    slot = (int)live_.size();
    live_.push_back(0);
    reported_.push_back(0);
    hprob_.push_back(CgProb());
  }
  const size_t N = (size_t)n * n, F = (size_t)n * (n + 1);
  CgProb P;
  std::memset(&P, 0, sizeof P);
  P.n = n;
  P.prec = prec;
  P.state = prec == 0 ? CG64_INIT : CG_OUTER;
  P.maxit = maxit;
  P.maxouter = maxouter;
  P.tol = tol;
  P.inner_tol = inner_tol;
  char* s = (char*)slab;
  auto take = [&](size_t bytes) {
    char* p = s;
    s += al256(bytes);
    return p;
  };
  P.b = (double*)take(8 * N);
  P.x = (double*)take(8 * N);
  P.r = (double*)take(8 * N);
  P.p64 = (double*)take(8 * N);
  P.w64 = (double*)take(8 * N);
  P.kx = (double*)take(8 * F);
  P.ky = (double*)take(8 * F);
  P.dg = (double*)take(8 * N);
  P.kx32 = (float*)take(4 * F);
  P.ky32 = (float*)take(4 * F);
  P.dg32 = (float*)take(4 * N);
  P.r32 = (float*)take(4 * N);
  P.p32 = (float*)take(4 * N);
  P.w32 = (float*)take(4 * N);
  P.d32 = (float*)take(4 * N);
  P.p32b = (float*)take(4 * N);
  hprob_[slot] = P;
  live_[slot] = 1;
  reported_[slot] = 0;
  if ((int)hstate_.size() > slot) hstate_[slot] = -1;  // upload and set up at the next rebuild
  ++nlive_;
  units_dirty_ = true;
  // conductivity goes to P.r for the set-up kernels, the right-hand side to P.b
  cudaMemcpyAsync(P.r, kappa, 8 * N, cudaMemcpyHostToDevice, stream_);
  cudaMemcpyAsync(P.b, rhs, 8 * N, cudaMemcpyHostToDevice, stream_);
  return slot;
}

void CgBatch::remove(int slot) {
  if (slot < 0 || slot >= (int)live_.size() || !live_[slot]) return;
  live_[slot] = 0;
  hprob_[slot].state = CG_FREE;
  --nlive_;
  units_dirty_ = true;
}

cudaError_t CgBatch::rebuild_units() {
  // the device array of problems must hold every slot; slots keep their
  // device state across rebuilds (only new problems are uploaded)
  const int nslots = (int)hprob_.size();
  if (fixed_) {
    if (init_error_ != cudaSuccess) return init_error_;
    int nu = 0;
    for (int s = 0; s < nslots; ++s)
      if (live_[s]) nu += cg_unit_count(hprob_[s].n);
    if (nslots > dprob_cap_ || nu > dunits_cap_) return cudaErrorMemoryAllocation;
  }
  if (!dcnt_) {
    cudaError_t e = cudaMalloc(&dcnt_, 2 * sizeof(int));
    if (e != cudaSuccess) return e;
  }
  if (nslots > dprob_cap_) {
    CgProb* nd = nullptr;
    const int cap = std::max(nslots, 2 * dprob_cap_);
    cudaError_t e = cudaMalloc(&nd, sizeof(CgProb) * cap);
    if (e != cudaSuccess) return e;
    if (dprob_) {
      cudaMemcpyAsync(nd, dprob_, sizeof(CgProb) * dprob_cap_, cudaMemcpyDeviceToDevice, stream_);
      cudaStreamSynchronize(stream_);
      cudaFree(dprob_);
    }
    dprob_ = nd;
    dprob_cap_ = cap;
  }
  std::vector<CgUnit> units;
  std::vector<int2> ranges(nslots);
  std::vector<int> fresh;
  for (int s = 0; s < nslots; ++s) {
    const int u0 = (int)units.size();
    if (live_[s]) units_for(s, hprob_[s].n, units);
    ranges[s] = make_int2(u0, (int)units.size());
  }
  nunits_ = (int)units.size();
  const int need_units = std::max(1, nunits_);
  if (need_units > dunits_cap_) {
    cudaStreamSynchronize(stream_);
    cudaFree(dunits_);
    dunits_cap_ = std::max(need_units, 2 * dunits_cap_);
    cudaError_t e = cudaMalloc(&dunits_, sizeof(CgUnit) * dunits_cap_);
    if (e != cudaSuccess) return e;
  }
  if (nslots > dranges_cap_) {
    cudaStreamSynchronize(stream_);
    cudaFree(dranges_);
    dranges_cap_ = std::max(nslots, 2 * dranges_cap_);
    cudaError_t e = cudaMalloc(&dranges_, sizeof(int2) * dranges_cap_);
    if (e != cudaSuccess) return e;
  }
  if (need_units > dpart_cap_) {
    cudaStreamSynchronize(stream_);
    cudaFree(dpart_);
    dpart_cap_ = std::max(need_units, 2 * dpart_cap_);
    cudaError_t e = cudaMalloc(&dpart_, sizeof(DD) * dpart_cap_);
    if (e != cudaSuccess) return e;
  }
  if (nunits_)
    cudaMemcpyAsync(dunits_, units.data(), sizeof(CgUnit) * nunits_, cudaMemcpyHostToDevice, stream_);
  cudaMemcpyAsync(dranges_, ranges.data(), sizeof(int2) * nslots, cudaMemcpyHostToDevice, stream_);
  // upload the problems added since the last rebuild and run their set-up
  cudaError_t e = cudaSuccess;
  for (int s = 0; s < nslots; ++s) {
    const bool is_new = live_[s] && ((int)hstate_.size() <= s || hstate_[s] == -1);
    if ((int)hstate_.size() <= s) hstate_.push_back(-1);
    if (!live_[s]) {
      hstate_[s] = -1;
      // a freed slot must read as free on the device
      CgProb P;
      std::memset(&P, 0, sizeof P);
      P.state = CG_FREE;
      cudaMemcpyAsync(dprob_ + s, &P, sizeof P, cudaMemcpyHostToDevice, stream_);
      continue;
    }
    if (is_new) {
      cudaMemcpyAsync(dprob_ + s, &hprob_[s], sizeof(CgProb), cudaMemcpyHostToDevice, stream_);
      const int u0 = ranges[s].x, u1 = ranges[s].y;
      const int g = std::max(1, std::min(u1 - u0, num_sms_ * 4));
      k_cg_setup<<<g, kCgThreads, 0, stream_>>>(dprob_, dunits_, u0, u1);
      k_cg_setup2<<<g, kCgThreads, 0, stream_>>>(dprob_, dunits_, u0, u1);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      hstate_[s] = hprob_[s].state;
    }
  }
  // the kernels read the unit and slot counts from the device
  hcnt_[0] = nunits_;
  hcnt_[1] = nslots;
  e = cudaMemcpyAsync(dcnt_, hcnt_, 2 * sizeof(int), cudaMemcpyHostToDevice, stream_);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(stream_);  // hcnt_ is host memory the copy reads
  if (e != cudaSuccess) return e;
  units_dirty_ = false;
  return cudaSuccess;
}

cudaError_t CgBatch::run(int ticks) {
  if (units_dirty_) {
    cudaError_t e = rebuild_units();
    if (e != cudaSuccess) return e;
  }
  if (nunits_ == 0) return cudaSuccess;
  const int nslots = (int)hprob_.size();
  const int2* ranges = dranges_;
  int per_sm = cg_grid_per_sm();
  if (per_sm == 0) {
    // as many CTAs as the A sweep keeps resident (the B and C sweeps keep at least as many)
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cg_a, kCgThreads, 0) != cudaSuccess || per_sm < 1)
      per_sm = 4;
  }
  // fixed tables: one wave of resident CTAs whatever the batch holds, and a
  // scalar block per possible slot, so the graph never has to change
  const int g = fixed_ ? num_sms_ * per_sm : std::max(1, std::min(nunits_, num_sms_ * per_sm));
  const int gs = fixed_ ? dprob_cap_ : nslots;  // scalar kernels: one block per problem slot
  // the tick sequence is captured once and replayed; it is captured again
  // only when a table moved or the launch shape changed
  const std::array<const void*, 5> args = {dprob_, dunits_, dranges_, dpart_, dcnt_};
  if (!gexec_ || gticks_ != ticks || gargs_ != args || gg_ != g || ggs_ != gs) {
    if (gexec_) cudaGraphExecDestroy(gexec_);
    gexec_ = nullptr;
    cudaError_t e = cudaStreamBeginCapture(stream_, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    for (int t = 0; t < ticks; ++t) {
      k_cg_a<<<g, kCgThreads, 0, stream_>>>(dprob_, dunits_, dcnt_, dpart_);
      k_cg_s1<<<gs, 256, 0, stream_>>>(dprob_, ranges, dcnt_, dpart_);
      k_cg_b<<<g, kCgThreads, 0, stream_>>>(dprob_, dunits_, dcnt_, dpart_);
      k_cg_s2<<<gs, 256, 0, stream_>>>(dprob_, ranges, dcnt_, dpart_);
      k_cg_c<<<g, kCgThreads, 0, stream_>>>(dprob_, dunits_, dcnt_);
    }
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(stream_, &graph);
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(&gexec_, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return e;
    gticks_ = ticks;
    gargs_ = args;
    gg_ = g;
    ggs_ = gs;
  }
  return cudaGraphLaunch(gexec_, stream_);
}

cudaError_t CgBatch::poll(std::vector<int>& done, std::vector<CgProb>* infos) {
  done.clear();
  if (infos) infos->clear();
  const int nslots = (int)hprob_.size();
  if (!nslots || !dprob_) return cudaSuccess;
  std::vector<CgProb> tmp(nslots);
  cudaError_t e = cudaMemcpyAsync(tmp.data(), dprob_, sizeof(CgProb) * nslots, cudaMemcpyDeviceToHost, stream_);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(stream_);
  if (e != cudaSuccess) return e;
  for (int s = 0; s < nslots; ++s)
    if (live_[s] && !reported_[s] && tmp[s].state == CG_DONE) {
      reported_[s] = 1;
      done.push_back(s);
      if (infos) infos->push_back(tmp[s]);
    }
  return cudaSuccess;
}

cudaError_t CgBatch::apply(int slot, int prec, const double* host_u, double* host_w) {
  if (units_dirty_) {
    cudaError_t e = rebuild_units();
    if (e != cudaSuccess) return e;
  }
  const CgProb& H = hprob_[slot];
  const size_t N = (size_t)H.n * H.n;
  std::vector<int2> ranges(hprob_.size());
  cudaError_t e = cudaMemcpyAsync(ranges.data(), dranges_, sizeof(int2) * ranges.size(), cudaMemcpyDeviceToHost,
                                  stream_);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream_);
  if (e != cudaSuccess) return e;
  std::vector<float> f;
  if (prec == 0) {
    e = cudaMemcpyAsync(H.x, host_u, 8 * N, cudaMemcpyHostToDevice, stream_);
  } else {
    f.resize(N);
    for (size_t i = 0; i < N; ++i) f[i] = (float)host_u[i];
    e = cudaMemcpyAsync(H.p32, f.data(), 4 * N, cudaMemcpyHostToDevice, stream_);
  }
  if (e != cudaSuccess) return e;
  const int u0 = ranges[slot].x, u1 = ranges[slot].y;
  k_cg_apply<<<std::max(1, std::min(u1 - u0, num_sms_ * 4)), kCgThreads, 0, stream_>>>(dprob_, dunits_, u0, u1, prec);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (prec == 0) {
    e = cudaMemcpyAsync(host_w, H.r, 8 * N, cudaMemcpyDeviceToHost, stream_);
  } else {
    e = cudaMemcpyAsync(f.data(), H.w32, 4 * N, cudaMemcpyDeviceToHost, stream_);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream_);
    for (size_t i = 0; i < N && e == cudaSuccess; ++i) host_w[i] = (double)f[i];
  }
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(stream_);
}

cudaError_t CgBatch::fetch(int slot, double* host_x, CgProb* info) {
  const CgProb& H = hprob_[slot];
  const size_t N = (size_t)H.n * H.n;
  cudaError_t e = cudaSuccess;
  if (host_x) e = cudaMemcpyAsync(host_x, H.x, 8 * N, cudaMemcpyDeviceToHost, stream_);
  if (e != cudaSuccess) return e;
  if (info) e = cudaMemcpyAsync(info, dprob_ + slot, sizeof(CgProb), cudaMemcpyDeviceToHost, stream_);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(stream_);
}

}  // namespace opstile

// ===========================================================================
// C ABI
// ===========================================================================
using namespace opstile;

extern "C" int ops_cg_solve_batch(ops_ctx ctx, int count, const int* n, const double* const* host_kappa,
                                  const double* const* host_rhs, const ops_cg_params* params,
                                  double* const* host_x, ops_cg_stats* stats) {
  if (!ctx || count < 1 || !n || !host_kappa || !host_rhs || !params || !host_x) return OPS_ERR_INVALID_ARG;
  if (ctx_host_only(ctx)) return ctx_fail(ctx, OPS_ERR_NO_DEVICE, "host-only context");
  const ops_cg_params& P = *params;
  if (!(P.tol > 0.0) || (P.precision != OPS_PREC_FP64 && P.precision != OPS_PREC_MIXED) || P.maxit < 1)
    return ctx_fail(ctx, OPS_ERR_INVALID_ARG, "cg: tol > 0, precision FP64/MIXED and maxit >= 1 required");
  for (int i = 0; i < count; ++i)
    if (n[i] < 1 || n[i] > 46000 || !host_kappa[i] || !host_rhs[i] || !host_x[i])
      return ctx_fail(ctx, OPS_ERR_INVALID_ARG, "cg: grid side must be 1..46000 with all arrays given");
  const double inner_tol = P.inner_tol > 0.0 ? P.inner_tol : 1e-4;
  const int maxouter = P.maxouter > 0 ? P.maxouter : 100;
  std::vector<void*> slabs(count, nullptr);
  std::vector<int> slots(count, -1);
  int rc = OPS_OK;
  {
    CgBatch B(ctx_stream(ctx), ctx_num_sms(ctx));
    for (int i = 0; i < count && rc == OPS_OK; ++i) {
      rc = ctx_alloc(ctx, &slabs[i], (size_t)cg_problem_bytes(n[i]));
      if (rc == OPS_OK)
        slots[i] = B.add(n[i], host_kappa[i], host_rhs[i], P.tol, P.precision, inner_tol, P.maxit, maxouter,
                         slabs[i]);
    }
    int remaining = count;
    std::vector<int> done;
    // every live problem reaches CG_DONE within maxit iterations plus one
    // refinement step per correction; the loop bound only guards the host
    const long long max_ticks = 2ll * P.maxit + 4ll * maxouter + 64;
    long long ticks = 0;
    while (rc == OPS_OK && remaining > 0) {
      if (ticks > max_ticks) {
        rc = ctx_fail(ctx, OPS_ERR_NOT_CONVERGED, "cg: tick limit reached");
        break;
      }
      const int chunk = 8;
      cudaError_t e = B.run(chunk);
      ticks += chunk;
      if (e == cudaSuccess) e = B.poll(done);
      if (e != cudaSuccess) {
        rc = ctx_fail(ctx, OPS_ERR_CUDA, cudaGetErrorString(e));
        break;
      }
      remaining -= (int)done.size();
    }
    bool all_conv = true;
    for (int i = 0; i < count && rc == OPS_OK; ++i) {
      CgProb info;
      cudaError_t e = B.fetch(slots[i], host_x[i], &info);
      if (e != cudaSuccess) {
        rc = ctx_fail(ctx, OPS_ERR_CUDA, cudaGetErrorString(e));
        break;
      }
      if (stats) {
        stats[i].iterations = info.it;
        stats[i].outer = info.outer;
        stats[i].converged = info.conv;
        stats[i].relres = info.rel;
      }
      all_conv = all_conv && info.conv;
    }
    if (rc == OPS_OK && !all_conv) rc = ctx_fail(ctx, OPS_ERR_NOT_CONVERGED, "cg: iteration cap reached");
  }
  for (int i = 0; i < count; ++i)
    if (slabs[i]) ctx_free(ctx, slabs[i], (size_t)cg_problem_bytes(n[i]));
  return rc;
}

extern "C" int ops_cg_solve(ops_ctx ctx, int n, const double* host_kappa, const double* host_rhs,
                            const ops_cg_params* params, double* host_x, ops_cg_stats* stats) {
  return ops_cg_solve_batch(ctx, 1, &n, &host_kappa, &host_rhs, params, &host_x, stats);
}

extern "C" int ops_heat_apply(ops_ctx ctx, int n, const double* host_kappa, const double* host_u, int precision,
                              double* host_w) {
  if (!ctx || n < 1 || n > 46000 || !host_kappa || !host_u || !host_w) return OPS_ERR_INVALID_ARG;
  if (ctx_host_only(ctx)) return ctx_fail(ctx, OPS_ERR_NO_DEVICE, "host-only context");
  if (precision != OPS_PREC_FP64 && precision != OPS_PREC_MIXED)
    return ctx_fail(ctx, OPS_ERR_INVALID_ARG, "precision must be OPS_PREC_FP64 or OPS_PREC_MIXED");
  void* slab = nullptr;
  const size_t bytes = (size_t)cg_problem_bytes(n);
  int rc = ctx_alloc(ctx, &slab, bytes);
  if (rc) return rc;
  {
    CgBatch B(ctx_stream(ctx), ctx_num_sms(ctx));
    std::vector<double> zero((size_t)n * n, 0.0);
    const int slot = B.add(n, host_kappa, zero.data(), 1.0, OPS_PREC_FP64, 1e-4, 1, 1, slab);
    cudaError_t e = B.apply(slot, precision == OPS_PREC_FP64 ? 0 : 1, host_u, host_w);
    if (e != cudaSuccess) rc = ctx_fail(ctx, OPS_ERR_CUDA, cudaGetErrorString(e));
  }
  ctx_free(ctx, slab, bytes);
  return rc;
}
