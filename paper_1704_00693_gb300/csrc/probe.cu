// Hardware probes behind the roofline the library reports: the rates and
// latencies that decide whether a loop chain on this GPU is bound by HBM,
// by L2, by the FP64 pipe or by synchronisation.  Each probe is a small
// kernel timed with CUDA events on a private stream; every wait in them is
// bounded in wall-clock time.
#include <cuda_runtime.h>

#include <cstring>

#include "internal.h"
#include "opstile.h"

namespace opstile {
namespace {

constexpr int kChains = 8;  // independent dependency chains per thread

__global__ void k_dfma(double* out, double b, double c, int iters) {
  double a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = threadIdx.x * 1e-9 + k;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = __fma_rn(a[k], b, c);
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s = __dadd_rn(s, a[k]);
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_dadd(double* out, double b, int iters) {
  double a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = threadIdx.x * 1e-9 + k;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = __dadd_rn(a[k], b);
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s = __dadd_rn(s, a[k]);
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_ffma(float* out, float b, float c, int iters) {
  float a[2 * kChains];
#pragma unroll
  for (int k = 0; k < 2 * kChains; ++k) a[k] = threadIdx.x * 1e-9f + k;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < 2 * kChains; ++k) a[k] = __fmaf_rn(a[k], b, c);
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < 2 * kChains; ++k) s = __fadd_rn(s, a[k]);
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// every thread sums its share of buf, `passes` times over
__global__ void k_read(const float4* __restrict__ buf, size_t n4, int passes, float* out) {
  float s = 0.0f;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (int p = 0; p < passes; ++p)
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
      const float4 v = __ldcg(buf + i);
      s += v.x + v.y + v.z + v.w;
    }
  if (s == 1.2345f) out[0] = s;  // keeps the loads
}

__global__ void k_copy(const float4* __restrict__ a, float4* __restrict__ b, size_t n4) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) b[i] = __ldcs(a + i);
}

__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// `rounds` grid-wide barriers (arrival counter and generation word); one
// small CTA per SM, so every CTA is resident
__global__ void k_barrier(unsigned* w, int rounds, long long timeout_ns, int* err) {
  __shared__ int s_stop;
  unsigned gen = 0;
  for (int r = 0; r < rounds; ++r) {
    __syncthreads();
    if (threadIdx.x == 0) {
      volatile unsigned* g = w + 1;
      const unsigned mine = gen;
      __threadfence();
      if (atomicAdd(w, 1u) == gridDim.x - 1) {
        w[0] = 0;
        __threadfence();
        atomicAdd(w + 1, 1u);
      } else {
        const unsigned long long t0 = gtime();
        while (*g == mine) {
          if ((long long)(gtime() - t0) > timeout_ns) {
            atomicExch(err, 1);
            break;
          }
        }
      }
      gen = mine + 1;
      s_stop = *(volatile int*)err;
    }
    __syncthreads();
    if (s_stop) return;
  }
}

// two CTAs answer each other's release stores `rounds` times
__global__ void k_pingpong(int* f, int rounds, long long timeout_ns, int* err) {
  if (threadIdx.x != 0) return;
  int* mine = f + 32 * blockIdx.x;
  const int* theirs = f + 32 * (1 - blockIdx.x);
  for (int r = 1; r <= rounds; ++r) {
    if (blockIdx.x == 0) asm volatile("st.release.gpu.global.b32 [%0], %1;" :: "l"(mine), "r"(r) : "memory");
    const unsigned long long t0 = gtime();
    for (;;) {
      int v;
      asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(theirs) : "memory");
      if (v >= r) break;
      if ((long long)(gtime() - t0) > timeout_ns || *(volatile int*)err) {
        atomicExch(err, 1);
        return;
      }
    }
    if (blockIdx.x == 1) asm volatile("st.release.gpu.global.b32 [%0], %1;" :: "l"(mine), "r"(r) : "memory");
  }
}

struct Timer {
  cudaStream_t s;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  explicit Timer(cudaStream_t st) : s(st) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
  }
  ~Timer() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
  void start() { cudaEventRecord(e0, s); }
  double stop_ms() {
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms;
  }
};

}  // namespace
}  // namespace opstile

using namespace opstile;

#define PROBE_TRY(x)                  \
  do {                                \
    if ((x) != cudaSuccess) {         \
      rc = OPS_ERR_CUDA;              \
      goto done;                      \
    }                                 \
  } while (0)

extern "C" int ops_probe_device(int device, ops_probe_result* out) {
  if (!out) return OPS_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof *out);
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess) return OPS_ERR_NO_DEVICE;
  if (cudaSetDevice(device) != cudaSuccess) return OPS_ERR_NO_DEVICE;
  int rc = OPS_OK;
  cudaStream_t s = nullptr;
  double* dbuf = nullptr;
  float4 *b0 = nullptr, *b1 = nullptr;
  unsigned* w = nullptr;
  int* err = nullptr;
  {
    cudaDeviceProp prop;
    PROBE_TRY(cudaGetDeviceProperties(&prop, device));
    int clk = 0, persist = 0;
    cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, device);
    cudaDeviceGetAttribute(&persist, cudaDevAttrMaxPersistingL2CacheSize, device);
    out->num_sms = prop.multiProcessorCount;
    out->l2_bytes = prop.l2CacheSize;
    out->persisting_l2_max_bytes = persist;
    out->sm_clock_khz_max = clk;
    const int sms = prop.multiProcessorCount;
    PROBE_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    Timer T(s);
    const int ctas = sms * 8, thr = 256, iters = 4096;
    PROBE_TRY(cudaMalloc(&dbuf, sizeof(double) * ctas * thr));
    // FP64 fma and add rates: warm up once, then time
    k_dfma<<<ctas, thr, 0, s>>>(dbuf, 0.999999, 1e-7, 64);
    T.start();
    k_dfma<<<ctas, thr, 0, s>>>(dbuf, 0.999999, 1e-7, iters);
    double ms = T.stop_ms();
    PROBE_TRY(cudaGetLastError());
    out->fp64_fma_tflops = 2.0 * ctas * thr * (double)iters * kChains / (ms * 1e-3) / 1e12;
    T.start();
    k_dadd<<<ctas, thr, 0, s>>>(dbuf, 1e-7, iters);
    ms = T.stop_ms();
    PROBE_TRY(cudaGetLastError());
    out->fp64_add_tops = (double)ctas * thr * iters * kChains / (ms * 1e-3) / 1e12;
    T.start();
    k_ffma<<<ctas, thr, 0, s>>>((float*)dbuf, 0.999999f, 1e-7f, iters);
    ms = T.stop_ms();
    PROBE_TRY(cudaGetLastError());
    out->fp32_fma_tflops = 2.0 * ctas * thr * (double)iters * 2 * kChains / (ms * 1e-3) / 1e12;
    // L2: a buffer of a third of L2, read over and over; HBM: a copy of 1 GiB
    const size_t l2n4 = (size_t)prop.l2CacheSize / 3 / sizeof(float4);
    const size_t hn4 = ((size_t)1 << 30) / sizeof(float4);
    PROBE_TRY(cudaMalloc(&b0, sizeof(float4) * hn4));
    PROBE_TRY(cudaMalloc(&b1, sizeof(float4) * hn4));
    PROBE_TRY(cudaMemsetAsync(b0, 0, sizeof(float4) * hn4, s));
    k_read<<<sms * 8, 512, 0, s>>>(b0, l2n4, 1, (float*)dbuf);
    const int passes = 40;
    T.start();
    k_read<<<sms * 8, 512, 0, s>>>(b0, l2n4, passes, (float*)dbuf);
    ms = T.stop_ms();
    PROBE_TRY(cudaGetLastError());
    out->l2_read_gbs = (double)l2n4 * sizeof(float4) * passes / (ms * 1e-3) / 1e9;
    k_copy<<<sms * 8, 512, 0, s>>>(b0, b1, hn4);
    T.start();
    for (int r = 0; r < 4; ++r) k_copy<<<sms * 8, 512, 0, s>>>(r % 2 ? b1 : b0, r % 2 ? b0 : b1, hn4);
    ms = T.stop_ms();
    PROBE_TRY(cudaGetLastError());
    out->hbm_copy_gbs = 4.0 * 2.0 * (double)hn4 * sizeof(float4) / (ms * 1e-3) / 1e9;
    // synchronisation: grid barriers (one CTA per SM) and a two-CTA flag round trip
    PROBE_TRY(cudaMalloc(&w, 64 * sizeof(unsigned)));
    PROBE_TRY(cudaMalloc(&err, sizeof(int)));
    PROBE_TRY(cudaMemsetAsync(w, 0, 64 * sizeof(unsigned), s));
    PROBE_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
    const long long lim = 2000ll * 1000 * 1000;
    const int rounds = 2000;
    k_barrier<<<sms, 32, 0, s>>>(w, 10, lim, err);
    T.start();
    k_barrier<<<sms, 32, 0, s>>>(w, rounds, lim, err);
    ms = T.stop_ms();
    PROBE_TRY(cudaGetLastError());
    out->grid_barrier_us = ms * 1e3 / rounds;
    PROBE_TRY(cudaMemsetAsync(w, 0, 64 * sizeof(unsigned), s));
    T.start();
    k_pingpong<<<2, 32, 0, s>>>((int*)w, rounds, lim, err);
    ms = T.stop_ms();
    PROBE_TRY(cudaGetLastError());
    out->flag_roundtrip_us = ms * 1e3 / rounds;
    int herr = 0;
    PROBE_TRY(cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr) rc = OPS_ERR_TIMEOUT;
  }
done:
  if (s) cudaStreamSynchronize(s);
  cudaFree(dbuf);
  cudaFree(b0);
  cudaFree(b1);
  cudaFree(w);
  cudaFree(err);
  if (s) cudaStreamDestroy(s);
  cudaSetDevice(prev);
  return rc;
}
