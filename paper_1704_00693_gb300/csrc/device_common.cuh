// Device helpers shared by the interpreter kernels (chain_kernels.cu, which
// includes this file inside namespace opstile) and the loop bodies compiled
// at run time (jit.cpp embeds this file's text into every generated
// module).  Self-contained: it uses only the DD struct {double hi, lo;} of
// its includer and CUDA built-ins.  Reduction operators are 0 sum, 1 min,
// 2 max (OPS_RED_SUM, OPS_RED_MIN, OPS_RED_MAX).

// compensated accumulation (Knuth's two-sum; order fixed by the launch shape)
__device__ __forceinline__ DD dd_add(DD a, double x) {
  const double s = __dadd_rn(a.hi, x);
  const double bp = __dsub_rn(s, a.hi);
  const double e = __dadd_rn(__dsub_rn(a.hi, __dsub_rn(s, bp)), __dsub_rn(x, bp));
  DD r;
  r.hi = s;
  r.lo = __dadd_rn(a.lo, e);
  return r;
}
__device__ __forceinline__ DD dd_merge(DD a, DD b) {
  DD t = dd_add(a, b.hi);
  t.lo = __dadd_rn(t.lo, b.lo);
  return t;
}
__device__ __forceinline__ DD dd_of(double v) {
  DD r;
  r.hi = v;
  r.lo = 0.0;
  return r;
}
__device__ __forceinline__ double red_identity(int op) {
  return op == 0 ? 0.0 : (op == 1 ? __longlong_as_double(0x7ff0000000000000ll) : __longlong_as_double(0xfff0000000000000ll));
}
__device__ __forceinline__ DD red_combine(int op, DD a, DD b) {
  if (op == 0) return dd_merge(a, b);
  if (op == 1) return dd_of((b.hi < a.hi) ? b.hi : a.hi);
  return dd_of((b.hi > a.hi) ? b.hi : a.hi);
}
__device__ __forceinline__ DD red_sum(DD a, double x) { return dd_add(a, x); }
__device__ __forceinline__ DD red_min(DD a, double x) { return dd_of((x < a.hi) ? x : a.hi); }
__device__ __forceinline__ DD red_max(DD a, double x) { return dd_of((x > a.hi) ? x : a.hi); }
__device__ __forceinline__ DD red_add(int op, DD a, double x) {
  return op == 0 ? red_sum(a, x) : (op == 1 ? red_min(a, x) : red_max(a, x));
}
__device__ __forceinline__ DD shfl_down_dd(DD v, int o) {
  DD w;
  w.hi = __shfl_down_sync(0xffffffffu, v.hi, o);
  w.lo = __shfl_down_sync(0xffffffffu, v.lo, o);
  return w;
}

// Block-wide combine in a fixed tree (sh: 32 entries of shared memory);
// the result is valid in thread 0.
__device__ __forceinline__ DD block_combine(int op, DD v, DD* sh) {
  for (int o = 16; o > 0; o >>= 1) v = red_combine(op, v, shfl_down_dd(v, o));
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    v = lane < nw ? sh[lane] : dd_of(red_identity(op));
    for (int o = 16; o > 0; o >>= 1) v = red_combine(op, v, shfl_down_dd(v, o));
  }
  return v;
}

// Copy a box between a global dat (strides gp, gq) and a shared footprint
// whose origin is the box corner fb (strides sp, sq); rows are spread over
// the warps, x over the lanes (coalesced).
template <class T>
__device__ __forceinline__ void copy_box(const int* box, const int* fb, T* sm, int sp, int sq, const T* g0, T* g1,
                                         long long gp, long long gq, bool to_shared) {
  const int nx = box[1] - box[0], ny = box[3] - box[2], nz = box[5] - box[4];
  if (nx <= 0 || ny <= 0 || nz <= 0) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int r = warp; r < ny * nz; r += nw) {
    const int y = box[2] + r % ny, z = box[4] + r / ny;
    T* s = sm + (long long)(z - fb[4]) * sq + (long long)(y - fb[2]) * sp - fb[0];
    const long long g = (long long)y * gp + (long long)z * gq;
    if (to_shared)
      for (int x = box[0] + lane; x < box[1]; x += 32) s[x] = g0[g + x];
    else
      for (int x = box[0] + lane; x < box[1]; x += 32) g1[g + x] = s[x];
  }
}
