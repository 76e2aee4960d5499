// ops_loop_noalloc: one parallel loop (with reductions) that allocates no
// device memory.
//
// Who needs it: callers that are not allowed to call cudaMalloc/cudaFree.
// cudaMalloc and cudaFree may synchronise the whole device, which a serving
// loop sharing the GPU with other streams cannot afford; and programs whose
// device memory is owned by another allocator (a framework's caching
// allocator, a fixed pre-reserved pool) must not grow their footprint behind
// its back.  The regular path allocates its scratch per context; this entry
// point takes the scratch from a fixed array that every GPU loading the
// library holds until the process exits.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "internal.h"
#include "opstile.h"

namespace opstile {

// Scratch of ops_loop_noalloc (see OPS_NOALLOC_SCRATCH_BYTES):
//   [0, sizeof(DLoop))              the loop descriptor
//   then 64 doubles                 scalar / reduction slots
//   then 8 FoldRow                  reduction rows
//   then 1 int                      device error word
//   then partials                   OPS_MAX_REDS_PER_LOOP x kNoallocMaxGrid DD
constexpr int kNoallocMaxGrid = 1024;
constexpr size_t kOffLoop = 0;
constexpr size_t kOffScal = (sizeof(DLoop) + 255) / 256 * 256;
constexpr size_t kOffRows = kOffScal + 64 * sizeof(double);
constexpr size_t kOffErr = kOffRows + 8 * sizeof(FoldRow);
constexpr size_t kOffPart = (kOffErr + sizeof(int) + 255) / 256 * 256;
constexpr size_t kNoallocBytes = kOffPart + (size_t)OPS_MAX_REDS_PER_LOOP * kNoallocMaxGrid * sizeof(DD);
static_assert(kNoallocBytes <= OPS_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds the documented maximum");

static __device__ __align__(256) unsigned char g_noalloc_scratch[OPS_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_scratch_ptr[kMaxDevices];  // device address of g_noalloc_scratch, per device
int g_num_sms[kMaxDevices];

// Once per device, with that device current: the device address of the
// scratch array (host code may not use the symbol's name as an address).
cudaError_t scratch_for_current_device(unsigned char** out, int* num_sms) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = chain_kernels_setup();
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = (unsigned char*)p;
    g_num_sms[dev] = sms;
  }
  *out = g_scratch_ptr[dev];
  *num_sms = g_num_sms[dev];
  return cudaSuccess;
}

bool reg_ok(int r) { return r >= 0 && r < kNReg; }

// What one call stages into the scratch array: it travels as a kernel
// parameter (copied when the launch is issued), so no host buffer has to
// outlive the call and no host-to-device copy is queued.
struct Staged {
  DLoop L;
  double scal[64];
  FoldRow rows[8];
};
static_assert(sizeof(Staged) <= 32000, "kernel parameters are limited to 32 KB");
static_assert(kOffScal >= sizeof(DLoop) && kOffRows == kOffScal + sizeof(double) * 64, "scratch layout");

__global__ void k_stage(const Staged in, unsigned char* S) {
  const int n0 = (int)(sizeof(DLoop) / sizeof(int)), n1 = 64, n2 = (int)(sizeof(FoldRow) * 8 / sizeof(int));
  const int* L = (const int*)&in.L;
  const int* R = (const int*)in.rows;
  for (int i = threadIdx.x; i < n0; i += blockDim.x) ((int*)(S + kOffLoop))[i] = L[i];
  for (int i = threadIdx.x; i < n1; i += blockDim.x) ((double*)(S + kOffScal))[i] = in.scal[i];
  for (int i = threadIdx.x; i < n2; i += blockDim.x) ((int*)(S + kOffRows))[i] = R[i];
  if (threadIdx.x == 0) *(int*)(S + kOffErr) = 0;
}

// bytes [first, last) a view's allocation box spans
void view_span(const ops_dat_view& V, uintptr_t* first, uintptr_t* last) {
  const int64_t lo = (int64_t)V.lo[0] + (int64_t)V.lo[1] * V.pitch + (int64_t)V.lo[2] * V.plane;
  const int64_t hi = (int64_t)(V.hi[0] - 1) + (int64_t)(V.hi[1] - 1) * V.pitch + (int64_t)(V.hi[2] - 1) * V.plane;
  *first = (uintptr_t)(V.ptr0 + lo);
  *last = (uintptr_t)(V.ptr0 + hi + 1);
}
}  // namespace

}  // namespace opstile

using namespace opstile;

extern "C" int ops_loop_noalloc(int dims, const int* range, int nargs, const ops_arg* args,
                                const ops_dat_view* views, const int* stencil_npts, const int* stencil_offsets,
                                int nins, const int32_t* code, int nconsts, const double* consts,
                                const double* scalar_values, const int* red_ops, double* host_red_out,
                                void* stream) {
  if (nargs > OPS_MAX_ARGS || nins > OPS_MAX_INS || nconsts > OPS_MAX_CONSTS) return OPS_ERR_NOMEM;
  if (dims < 1 || dims > 3 || !range || nargs < 0 || (nargs && !args) || nins < 0 || (nins && !code) ||
      nconsts < 0 || (nconsts && !consts))
    return OPS_ERR_INVALID_ARG;
  // ---- describe the loop (host side, no heap) ----
  DLoop L;
  std::memset(&L, 0, sizeof L);
  L.nargs = nargs;
  L.nins = nins;
  for (int d = 0; d < 3; ++d) {
    L.rng[2 * d] = d < dims ? range[2 * d] : 0;
    L.rng[2 * d + 1] = d < dims ? range[2 * d + 1] : 1;
    if (L.rng[2 * d + 1] < L.rng[2 * d]) return OPS_ERR_INVALID_ARG;
  }
  if ((int64_t)(L.rng[1] - L.rng[0]) * (L.rng[3] - L.rng[2]) * (L.rng[5] - L.rng[4]) > (int64_t)kMaxLoopPoints)
    return OPS_ERR_INVALID_ARG;
  double scal[64] = {0.0};
  FoldRow rows[8] = {};
  int nreds = 0, off_pos = 0;
  for (int i = 0; i < nargs; ++i) {
    const ops_arg& a = args[i];
    DArg& A = L.args[i];
    A.kind = a.kind;
    A.access = a.access;
    if (a.kind == OPS_ARG_DAT) {
      if (!views || !stencil_npts || !stencil_offsets || !views[i].ptr0) return OPS_ERR_INVALID_ARG;
      const int np = stencil_npts[i];
      if (np > OPS_MAX_STENCIL_POINTS) return OPS_ERR_NOMEM;
      if (np < 1) return OPS_ERR_INVALID_ARG;
      if (a.access < OPS_READ || a.access > OPS_INC) return OPS_ERR_INVALID_ARG;
      const ops_dat_view& V = views[i];
      // a view's rows (and planes) must not overlap one another
      for (int d = 0; d < 3; ++d)
        if (V.hi[d] <= V.lo[d] || (d >= dims && (V.lo[d] != 0 || V.hi[d] != 1))) return OPS_ERR_INVALID_ARG;
      if (V.pitch < V.hi[0] - V.lo[0] || (dims > 2 && V.plane < V.pitch * (V.hi[1] - V.lo[1])))
        return OPS_ERR_INVALID_ARG;
      A.ptr0 = V.ptr0;
      A.pitch = V.pitch;
      A.plane = V.plane;
      A.npts = np;
      for (int d = 0; d < 3; ++d) {
        A.alo[d] = V.lo[d];
        A.ahi[d] = V.hi[d];
        A.slo[d] = 0;
        A.shi[d] = 0;
      }
      for (int p = 0; p < np; ++p) {
        const int* o = stencil_offsets + 3 * (off_pos + p);
        for (int d = 0; d < 3; ++d) {
          if (d >= dims && o[d] != 0) return OPS_ERR_INVALID_ARG;
          A.slo[d] = o[d] < A.slo[d] ? o[d] : A.slo[d];
          A.shi[d] = o[d] > A.shi[d] ? o[d] : A.shi[d];
        }
        A.off[p] = (int32_t)(o[0] + o[1] * V.pitch + o[2] * V.plane);
      }
      off_pos += np;
      if (a.access != OPS_READ && (np != 1 || A.slo[0] || A.slo[1] || A.slo[2] || A.shi[0] || A.shi[1] || A.shi[2]))
        return OPS_ERR_INVALID_ARG;
      for (int d = 0; d < 3; ++d)  // every access inside the caller's allocation box
        if (L.rng[2 * d + 1] > L.rng[2 * d] &&
            (L.rng[2 * d] + A.slo[d] < V.lo[d] || L.rng[2 * d + 1] - 1 + A.shi[d] >= V.hi[d]))
          return OPS_ERR_BOUNDS;
    } else if (a.kind == OPS_ARG_SCALAR) {
      if (!scalar_values) return OPS_ERR_INVALID_ARG;
      A.slot = 8 + i;
      scal[8 + i] = scalar_values[i];
    } else if (a.kind == OPS_ARG_RED) {
      if (nreds >= OPS_MAX_REDS_PER_LOOP) return OPS_ERR_NOMEM;
      if (!red_ops || !host_red_out) return OPS_ERR_INVALID_ARG;
      const int op = red_ops[i];
      if (op < OPS_RED_SUM || op > OPS_RED_MAX) return OPS_ERR_INVALID_ARG;
      A.slot = nreds;
      L.red_op[nreds] = op;
      rows[nreds] = FoldRow{nreds, op};
      scal[nreds] = op == OPS_RED_SUM ? 0.0 : (op == OPS_RED_MIN ? __builtin_inf() : -__builtin_inf());
      ++nreds;
    } else {
      return OPS_ERR_INVALID_ARG;
    }
  }
  L.nreds = nreds;
  L.part_row = 0;
  // as in ops_par_loop, a loop's dats are distinct: two views whose memory
  // overlaps, one of them written, would make the result depend on the
  // order of the points
  for (int i = 0; i < nargs; ++i)
    for (int j = i + 1; j < nargs; ++j) {
      if (args[i].kind != OPS_ARG_DAT || args[j].kind != OPS_ARG_DAT) continue;
      if (args[i].access == OPS_READ && args[j].access == OPS_READ) continue;
      uintptr_t a0, a1, b0, b1;
      view_span(views[i], &a0, &a1);
      view_span(views[j], &b0, &b1);
      if (a0 < b1 && b0 < a1) return OPS_ERR_INVALID_ARG;
    }
  // ---- IR well-formedness (same rules as ops_par_loop) ----
  std::memcpy(L.ins, code, sizeof(int32_t) * 6 * (size_t)nins);
  if (nconsts) std::memcpy(L.K, consts, sizeof(double) * (size_t)nconsts);
  for (int pc = 0; pc < nins; ++pc) {
    const int32_t* I = code + 6 * pc;
    const int op = I[0], d = I[1], a = I[2], b = I[3], c = I[4], e = I[5];
    bool ok;
    switch (op) {
      case OPS_IR_LD:
        ok = reg_ok(d) && a >= 0 && a < nargs &&
             ((args[a].kind == OPS_ARG_DAT && (args[a].access == OPS_READ || args[a].access == OPS_RW) && b >= 0 &&
               b < L.args[a].npts) ||
              (args[a].kind == OPS_ARG_SCALAR && b == 0));
        break;
      case OPS_IR_CST: ok = reg_ok(d) && a >= 0 && a < nconsts; break;
      case OPS_IR_ADD: case OPS_IR_SUB: case OPS_IR_MUL: case OPS_IR_DIV: case OPS_IR_MIN: case OPS_IR_MAX:
        ok = reg_ok(d) && reg_ok(a) && reg_ok(b);
        break;
      case OPS_IR_FMA: ok = reg_ok(d) && reg_ok(a) && reg_ok(b) && reg_ok(c); break;
      case OPS_IR_SGT: ok = reg_ok(d) && reg_ok(a) && reg_ok(b) && reg_ok(c) && reg_ok(e); break;
      case OPS_IR_WSUM: case OPS_IR_WACC:
        ok = reg_ok(d) && a >= 0 && a < nargs && args[a].kind == OPS_ARG_DAT &&
             (args[a].access == OPS_READ || args[a].access == OPS_RW) && b >= 0 && b + L.args[a].npts <= nconsts;
        break;
      case OPS_IR_POLY: ok = reg_ok(d) && reg_ok(a) && b >= 0 && c >= 0 && b + c < nconsts; break;
      case OPS_IR_ST:
        ok = d >= 0 && d < nargs && args[d].kind == OPS_ARG_DAT && args[d].access != OPS_READ && reg_ok(a);
        break;
      case OPS_IR_RED: ok = d >= 0 && d < nargs && args[d].kind == OPS_ARG_RED && reg_ok(a); break;
      default: ok = false;
    }
    if (!ok) return OPS_ERR_INVALID_ARG;
  }
  finish_dloop(L);
  // ---- scratch and launch shape ----
  unsigned char* S = nullptr;
  int sms = 0;
  if (scratch_for_current_device(&S, &sms) != cudaSuccess) return OPS_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  LaunchEnv env;
  env.stream = st;
  env.num_sms = sms;
  env.scal = (double*)(S + kOffScal);
  env.part = (DD*)(S + kOffPart);
  env.part_stride = kNoallocMaxGrid;
  env.rows = (const FoldRow*)(S + kOffRows);
  env.err = (int*)(S + kOffErr);
  env.bar = nullptr;
  env.check = 0;
  env.timeout_ns = 0;
  env.skip_block = -1;
  int box[6];
  bool empty = false;
  for (int i = 0; i < 6; ++i) box[i] = L.rng[i];
  for (int d = 0; d < 3; ++d)
    if (box[2 * d + 1] <= box[2 * d]) empty = true;
  int grid = empty ? 1 : untiled_grid(env, box);
  if (grid > kNoallocMaxGrid) grid = kNoallocMaxGrid;
  // ---- stage descriptor, slots, rows and a cleared error word ----
  Staged in;
  std::memcpy(&in.L, &L, sizeof L);
  std::memcpy(in.scal, scal, sizeof scal);
  std::memcpy(in.rows, rows, sizeof rows);
  k_stage<<<1, 256, 0, st>>>(in, S);
  if (cudaGetLastError() != cudaSuccess) return OPS_ERR_CUDA;
  if (!empty) {
    if (launch_untiled(env, (const DLoop*)(S + kOffLoop), box, grid) != cudaSuccess) return OPS_ERR_CUDA;
    if (nreds && launch_fold(env, 0, nreds, grid) != cudaSuccess) return OPS_ERR_CUDA;
  }
  if (nreds) {
    double out[OPS_MAX_REDS_PER_LOOP];
    if (cudaMemcpyAsync(out, S + kOffScal, sizeof(double) * nreds, cudaMemcpyDeviceToHost, st) != cudaSuccess)
      return OPS_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return OPS_ERR_CUDA;
    int k = 0;
    for (int i = 0; i < nargs; ++i)
      if (args[i].kind == OPS_ARG_RED) host_red_out[i] = out[k++];
  }
  return OPS_OK;
}
