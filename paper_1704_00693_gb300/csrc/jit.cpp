// Run-time compiled loop bodies (see jit.h).
//
// Code shape.  For loop i of a segment the generator emits body<i>, which
// enumerates its CTA's share of a box as the interpreter does (units of 256
// consecutive x by 4 consecutive rows for rows of >= 128 points, flattened
// groups otherwise) and evaluates the loop's IR per point with the
// same explicitly rounded operations in the same order, so every stored
// value is bit-identical to the interpreter's and the oracle's.  A unit of 4
// full rows is evaluated instruction by instruction across its 4 points (the
// interpreter's order, 4 independent dependency chains per thread); partial
// units and thin boxes take a one-point path.  The constants, dat pointers
// and scalar slots of a loop are read from its descriptor at run time, so
// one compiled segment serves every step whatever the host sets them to.
//
// Kernel u<i> runs loop i over a box with grid-stride units.  The untiled
// form launches it once per loop over the loop's range; the skewed form
// launches it once per (tile, loop) phase of the plan in plan order, the
// stream order standing in for the grid barriers of a persistent kernel.
// The loops of a segment are split over several modules that compile in
// parallel; compiled code is cached in memory and on disk by its source.
//
// NVRTC and the driver's module calls are reached at run time (dlopen and
// cudaGetDriverEntryPointByVersion), so the library loads on hosts without
// a GPU driver.
#include "jit.h"

#include <cuda.h>
#include <dlfcn.h>
#include <nvrtc.h>
#include <sys/stat.h>
#include <unistd.h>

#include <chrono>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <memory>
#include <mutex>
#include <sstream>
#include <thread>

namespace opstile {

namespace {

// Shape of the compiled kernels: rows per unit (independent points per
// thread; FP64 and FP32 loops) and the CTAs per SM the register budget is
// sized for.  Defaults from measurement on GB300 (FP32 loops, with half the
// registers per value, run 3.6% faster at 8 rows than at 4; FP64 loops do
// not); OPSTILE_JIT_PTS / OPSTILE_JIT_PTS32 / OPSTILE_JIT_MINB override.
int env_int(const char* name, int def, int lo, int hi) {
  const char* e = getenv(name);
  if (!e || !*e) return def;
  const int v = atoi(e);
  return v < lo ? lo : (v > hi ? hi : v);
}
const int kJitPts = env_int("OPSTILE_JIT_PTS", 4, 1, 8);
const int kJitPts32 = env_int("OPSTILE_JIT_PTS32", 8, 1, 8);
int pts_for(int es) { return es == 4 ? kJitPts32 : kJitPts; }
const int kJitMinCtas = env_int("OPSTILE_JIT_MINB", 2, 1, 8);
// Overlapped tiles: one CTA per SM holds the footprints, so it takes twice
// the threads of the untiled kernels; one point per thread at a time keeps
// the bodies within the 128 registers that 512 threads leave (1024 threads
// would spill them).
constexpr int kOvThreads = 512;
constexpr int kOvPts = 1;
constexpr int kJitChunk = 6;  // loops per compiled module (modules compile in parallel)
constexpr int kTwMaxGroup = 8;  // loops of one tile-wavefront step at most
// FP64 MIN / MAX / SGT on the integer pipe (dlt); 0 = IEEE double compares
const int kIntCmp = env_int("OPSTILE_JIT_INTCMP", 1, 0, 1);

// ---------------------------------------------------------------------------
// entry points reached at run time
// ---------------------------------------------------------------------------
struct Api {
  bool tried = false, ok = false;
  std::string why;
  // NVRTC
  nvrtcResult (*create)(nvrtcProgram*, const char*, const char*, int, const char* const*, const char* const*);
  nvrtcResult (*compile)(nvrtcProgram, int, const char* const*);
  nvrtcResult (*log_size)(nvrtcProgram, size_t*);
  nvrtcResult (*log)(nvrtcProgram, char*);
  nvrtcResult (*cubin_size)(nvrtcProgram, size_t*);
  nvrtcResult (*cubin)(nvrtcProgram, char*);
  nvrtcResult (*destroy)(nvrtcProgram*);
  // driver
  CUresult (*load)(CUmodule*, const void*);
  CUresult (*get_function)(CUfunction*, CUmodule, const char*);
  CUresult (*launch)(CUfunction, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned, CUstream,
                     void**, void**);
  CUresult (*launch_coop)(CUfunction, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned, CUstream,
                          void**);
  CUresult (*occupancy)(int*, CUfunction, int, size_t);
  CUresult (*attribute)(int*, CUfunction_attribute, CUfunction);
  CUresult (*set_attribute)(CUfunction, CUfunction_attribute, int);
  CUresult (*launch_ex)(const CUlaunchConfig*, CUfunction, void**, void**) = nullptr;  // optional
};

Api g_api;
std::mutex g_mu;

template <class F>
bool sym(void* lib, const char* name, F* f) {
  *f = reinterpret_cast<F>(dlsym(lib, name));
  return *f != nullptr;
}

template <class F>
bool drv(const char* name, F* f) {
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !p) {
    cudaGetLastError();
    return false;
  }
  *f = reinterpret_cast<F>(p);
  return true;
}

// call with g_mu held; nvrtc_only: skip the driver entry points
bool api_ready(std::string* why, bool nvrtc_only = false) {
  if (nvrtc_only && g_api.create) return true;
  if (!g_api.tried) {
    g_api.tried = !nvrtc_only;
    void* lib = nullptr;
    for (const char* n : {"libnvrtc.so.13", "/usr/local/cuda/lib64/libnvrtc.so.13", "libnvrtc.so"}) {
      lib = dlopen(n, RTLD_NOW | RTLD_LOCAL);
      if (lib) break;
    }
    if (!lib) {
      g_api.why = "libnvrtc.so.13 not found";
    } else if (!(sym(lib, "nvrtcCreateProgram", &g_api.create) && sym(lib, "nvrtcCompileProgram", &g_api.compile) &&
                 sym(lib, "nvrtcGetProgramLogSize", &g_api.log_size) &&
                 sym(lib, "nvrtcGetProgramLog", &g_api.log) && sym(lib, "nvrtcGetCUBINSize", &g_api.cubin_size) &&
                 sym(lib, "nvrtcGetCUBIN", &g_api.cubin) && sym(lib, "nvrtcDestroyProgram", &g_api.destroy))) {
      g_api.why = "libnvrtc lacks an entry point";
      g_api.create = nullptr;
    } else if (nvrtc_only) {
      return true;
    } else if (!(drv("cuModuleLoadData", &g_api.load) && drv("cuModuleGetFunction", &g_api.get_function) &&
                 drv("cuLaunchKernel", &g_api.launch) && drv("cuLaunchCooperativeKernel", &g_api.launch_coop) &&
                 drv("cuOccupancyMaxActiveBlocksPerMultiprocessor", &g_api.occupancy) &&
                 drv("cuFuncGetAttribute", &g_api.attribute) &&
                 drv("cuFuncSetAttribute", &g_api.set_attribute))) {
      g_api.why = "driver module entry points unavailable";
    } else {
      g_api.ok = true;
      if (!drv("cuLaunchKernelEx", &g_api.launch_ex)) g_api.launch_ex = nullptr;
    }
  }
  if (!g_api.ok && why) *why = g_api.why;
  return g_api.ok;
}

cudaError_t to_cuda(CUresult r) {
  if (r == CUDA_SUCCESS) return cudaSuccess;
  if (r == CUDA_ERROR_COOPERATIVE_LAUNCH_TOO_LARGE) return cudaErrorCooperativeLaunchTooLarge;
  if (r == CUDA_ERROR_INVALID_VALUE) return cudaErrorInvalidValue;
  return cudaErrorLaunchFailure;
}

// ---------------------------------------------------------------------------
// device code shared by every module (the generator appends the bodies)
// ---------------------------------------------------------------------------
const char* kPrelude = R"PRE(
typedef long long i64;
struct DD { double hi, lo; };
struct DArg {
  double* ptr0; i64 pitch; i64 plane; int kind, access, npts, slot;
  int alo[3], ahi[3]; int slo[3], shi[3]; int off[32];
};
struct DLoop {
  int nargs, nins, nreds; int rng[6]; int red_op[4]; int part_row; int zmask; int pad_;
  int ins[64][6]; double K[128]; DArg args[8];
};
struct Phase { int loop; int barrier; int box[6]; };
)PRE";

// device_common.cuh, embedded at build time (the interpreter kernels include the same file)
const char* kDeviceCommon =
#include "device_common.inc"
    ;

const char* kPreludeTail = R"PRE(
__shared__ DD g_sh[32];

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// b < a for doubles, decided on the integer pipe (the FP64 pipe is the
// narrow one on GB300): the IEEE order of non-NaN doubles is the signed
// integer order of their bit patterns once negative ones have their
// magnitude bits flipped, except that -0 and +0 compare equal; a NaN
// operand makes the comparison false.
__device__ __forceinline__ bool dlt(double b, double a) {
  const unsigned long long m = 0x7fffffffffffffffull, inf = 0x7ff0000000000000ull;
  const long long A = __double_as_longlong(a), B = __double_as_longlong(b);
  const bool nan = ((unsigned long long)A & m) > inf || ((unsigned long long)B & m) > inf;
  const bool zeros = (((unsigned long long)A | (unsigned long long)B) << 1) == 0;
  const long long ka = A >= 0 ? A : (A ^ (long long)m), kb = B >= 0 ? B : (B ^ (long long)m);
  return !nan && !zeros && kb < ka;
}

__device__ __forceinline__ void flush_red(int op, DD v, DD* part, int stride, int row, int assign) {
  v = block_combine(op, v, g_sh);
  if (threadIdx.x == 0) {
    DD* dst = part + (size_t)row * stride + blockIdx.x;
    *dst = assign ? v : red_combine(op, *dst, v);
  }
  __syncthreads();
}

// A CTA's (or a warp's) share of a box: rows of >= 128 points in units of NT
// x by P rows (u = part, part + nparts, ...), thinner boxes in flattened
// groups of P points NT apart (NT = threads per part: a CTA's, or 32 when
// the parts are warps; a thread's lane in its part is threadIdx.x % NT).  full(x, y, z) takes rows
// y .. y+P-1 at x; one(x, y, z) a single point.
template <int P, int NT, class F1, class FP>
__device__ __forceinline__ void run_units(int x0, int x1, int y0, int y1, int z0, int z1, int part, int nparts,
                                          F1& one, FP& full) {
  const int nx = x1 - x0, ny = y1 - y0, nz = z1 - z0;
  if (nx <= 0 || ny <= 0 || nz <= 0) return;
  if (nx >= (NT >= 128 ? 128 : NT)) {
    const int xch = (nx + NT - 1) / NT;
    const int nrg = (ny + P - 1) / P;
    const int nunits = xch * nrg * nz;
    int u = part;
    int xc = u % xch, rg = (u / xch) % nrg, z = u / (xch * nrg);
    const int dxc = nparts % xch, drg = (nparts / xch) % nrg, dz = nparts / (xch * nrg);
    while (u < nunits) {
      const int x = x0 + xc * NT + (int)(threadIdx.x % NT);
      if (x < x1) {
        const int yb = rg * P;
        if (yb + P <= ny) {
          full(x, y0 + yb, z0 + z);
        } else {
          for (int p = 0; p < ny - yb; ++p) one(x, y0 + yb + p, z0 + z);
        }
      }
      u += nparts; xc += dxc; rg += drg; z += dz;
      if (xc >= xch) { xc -= xch; ++rg; }
      if (rg >= nrg) { rg -= nrg; ++z; }
    }
  } else {
    const int npts = nx * ny * nz;
    const int step = nparts * NT * P;
    for (int i = part * NT * P + (int)(threadIdx.x % NT); i < npts; i += step) {
      for (int p = 0; p < P; ++p) {
        const int j = i + p * NT;
        if (j >= npts) break;
        const int r = j / nx;
        one(x0 + (j - r * nx), y0 + r % ny, z0 + r / ny);
      }
    }
  }
}


// overlapped tiles: one dat of a run (the library's OvDat)
struct OvDat { const double* src; double* dst; i64 gpitch, gplane; int written, smem_off, spitch, splane; };
)PRE";

// ---------------------------------------------------------------------------
// generator
// ---------------------------------------------------------------------------
std::string dbl_sfx(int reg, int p) { return "r" + std::to_string(reg) + "_" + std::to_string(p); }

struct LoopGen {
  const DLoop& L;
  const std::vector<char>& ro;
  std::vector<int> cls;               // pitch class of each DAT arg (-1 otherwise)
  std::vector<std::pair<int64_t, int64_t>> classes;
  std::ostringstream& os;
  bool ov = false;                    // overlapped tile: dats in shared footprints, owned-point reductions
  bool f32 = false;                   // FP32 dats and arithmetic
  // every dat pointer __restrict__: a dat appears at most once in a loop
  // (checked at enqueue), so a loop's stores never alias its other
  // arguments' loads and the compiler may overlap consecutive points
  mutable bool restrict_all = false;
  // tile bodies read their dat pointers from the step's shared-memory slot
  // (ptrs[a]), which the control warp fills, instead of the descriptor
  mutable bool staged_ptrs = false;
  std::string ptr_src(int a) const {
    return staged_ptrs ? "ptrs[" + std::to_string(a) + "]" : "L->args[" + std::to_string(a) + "].ptr0";
  }
  int nt = kThreads;                  // threads per CTA of the enumeration (not overlapped)
  const char* T = "double";
  const char *fadd = "__dadd_rn", *fsub = "__dsub_rn", *fmul = "__dmul_rn", *fdiv = "__ddiv_rn", *ffma = "__fma_rn";

  LoopGen(const DLoop& l, const std::vector<char>& r, std::ostringstream& o, bool overlapped = false,
          bool single = false)
      : L(l), ro(r), os(o), ov(overlapped), f32(single) {
    if (f32) {
      T = "float";
      fadd = "__fadd_rn";
      fsub = "__fsub_rn";
      fmul = "__fmul_rn";
      fdiv = "__fdiv_rn";
      ffma = "__fmaf_rn";
    }
    cls.assign(L.nargs, -1);
    for (int a = 0; a < L.nargs; ++a) {
      if (L.args[a].kind != OPS_ARG_DAT) continue;
      std::pair<int64_t, int64_t> pp(L.args[a].pitch, L.args[a].plane);
      int k = -1;
      for (int j = 0; j < (int)classes.size(); ++j)
        if (classes[j] == pp) k = j;
      if (k < 0) {
        k = (int)classes.size();
        classes.push_back(pp);
      }
      cls[a] = k;
    }
  }

  std::string idx(int a, int p) const { return "i" + std::to_string(cls[a]) + "_" + std::to_string(p); }
  std::string load(int a, int q, int p) const {
    std::string addr = "p" + std::to_string(a) + " + (" + idx(a, p) + " + (" + std::to_string(L.args[a].off[q]) + "))";
    return ro[a] ? "__ldg(" + addr + ")" : "*(" + addr + ")";
  }

  // the IR of one loop for points 0..np-1 (instruction-major)
  void emit_points(int np) const {
    for (int p = 0; p < np; ++p) {
      os << "    " << T;
      for (int r = 0; r < kNReg; ++r) os << (r ? ", " : " ") << dbl_sfx(r, p) << " = 0";
      os << ";\n";
      if (ov && L.nreds)  // redundant points of a tile compute but do not reduce
        os << "    const bool own" << p << " = x >= ob[0] && x < ob[1] && y + " << p << " >= ob[2] && y + " << p
           << " < ob[3] && z >= ob[4] && z < ob[5];\n";
    }
    for (int pc = 0; pc < L.nins; ++pc) {
      const int* I = L.ins[pc];
      const int op = I[0], d = I[1], a = I[2], b = I[3], c = I[4], e = I[5];
      for (int p = 0; p < np; ++p) {
        auto R = [&](int r) { return dbl_sfx(r, p); };
        switch (op) {
          case OPS_IR_LD:
            if (L.args[a].kind == OPS_ARG_SCALAR)
              os << "    " << R(d) << " = s" << a << ";\n";
            else
              os << "    " << R(d) << " = " << load(a, b, p) << ";\n";
            break;
          case OPS_IR_CST: os << "    " << R(d) << " = K" << a << ";\n"; break;
          case OPS_IR_ADD: os << "    " << R(d) << " = " << fadd << "(" << R(a) << ", " << R(b) << ");\n"; break;
          case OPS_IR_SUB: os << "    " << R(d) << " = " << fsub << "(" << R(a) << ", " << R(b) << ");\n"; break;
          case OPS_IR_MUL: os << "    " << R(d) << " = " << fmul << "(" << R(a) << ", " << R(b) << ");\n"; break;
          case OPS_IR_DIV: os << "    " << R(d) << " = " << fdiv << "(" << R(a) << ", " << R(b) << ");\n"; break;
          case OPS_IR_FMA:
            os << "    " << R(d) << " = " << ffma << "(" << R(a) << ", " << R(b) << ", " << R(c) << ");\n";
            break;
          // FP64 comparisons go through dlt (integer pipe) unless OPSTILE_JIT_INTCMP=0
          case OPS_IR_MIN:
            if (!f32 && kIntCmp)
              os << "    " << R(d) << " = dlt(" << R(b) << ", " << R(a) << ") ? " << R(b) << " : " << R(a) << ";\n";
            else
              os << "    " << R(d) << " = (" << R(b) << " < " << R(a) << ") ? " << R(b) << " : " << R(a) << ";\n";
            break;
          case OPS_IR_MAX:
            if (!f32 && kIntCmp)
              os << "    " << R(d) << " = dlt(" << R(a) << ", " << R(b) << ") ? " << R(b) << " : " << R(a) << ";\n";
            else
              os << "    " << R(d) << " = (" << R(b) << " > " << R(a) << ") ? " << R(b) << " : " << R(a) << ";\n";
            break;
          case OPS_IR_SGT:
            if (!f32 && kIntCmp)
              os << "    " << R(d) << " = dlt(" << R(b) << ", " << R(a) << ") ? " << R(c) << " : " << R(e) << ";\n";
            else
              os << "    " << R(d) << " = (" << R(a) << " > " << R(b) << ") ? " << R(c) << " : " << R(e) << ";\n";
            break;
          case OPS_IR_WSUM:
          case OPS_IR_WACC: {
            const int n = L.args[a].npts;
            os << "    { " << T << " t = ";
            int q = 0;
            if (op == OPS_IR_WSUM) {
              os << fmul << "(K" << b << ", " << load(a, 0, p) << ");\n";
              q = 1;
            } else {
              os << R(d) << ";\n";
            }
            for (; q < n; ++q) os << "      t = " << ffma << "(K" << (b + q) << ", " << load(a, q, p) << ", t);\n";
            os << "      " << R(d) << " = t; }\n";
            break;
          }
          case OPS_IR_POLY: {
            os << "    { " << T << " t = K" << (b + c) << ";\n";
            for (int i = c - 1; i >= 0; --i)
              os << "      t = " << ffma << "(t, " << R(a) << ", K" << (b + i) << ");\n";
            os << "      " << R(d) << " = t; }\n";
            break;
          }
          case OPS_IR_ST: {
            const std::string q = "p" + std::to_string(d) + "[" + idx(d, p) + "]";
            if (L.args[d].access == OPS_INC)
              os << "    " << q << " = " << fadd << "(" << q << ", " << R(a) << ");\n";
            else
              os << "    " << q << " = " << R(a) << ";\n";
            break;
          }
          case OPS_IR_RED: {
            const int k = L.args[d].slot;
            const int rop = L.red_op[k];
            const char* f = rop == OPS_RED_SUM ? "red_sum" : (rop == OPS_RED_MIN ? "red_min" : "red_max");
            // a float value converts to double exactly
            if (ov)
              os << "    if (own" << p << ") acc" << k << " = " << f << "(acc" << k << ", (double)" << R(a) << ");\n";
            else
              os << "    acc" << k << " = " << f << "(acc" << k << ", (double)" << R(a) << ");\n";
            break;
          }
          default: break;
        }
      }
    }
  }

  // hoisted per call: dat pointers, scalars, constants, reduction accumulators
  void emit_hoist(const OvLayout* lay) const {
    std::vector<char> kused(OPS_MAX_CONSTS, 0);
    std::vector<char> sused(L.nargs, 0);
    for (int pc = 0; pc < L.nins; ++pc) {
      const int* I = L.ins[pc];
      const int op = I[0], a = I[2], b = I[3], c = I[4];
      if (op == OPS_IR_CST) kused[a] = 1;
      if (op == OPS_IR_LD && L.args[a].kind == OPS_ARG_SCALAR) sused[a] = 1;
      if (op == OPS_IR_WSUM || op == OPS_IR_WACC)
        for (int q = 0; q < L.args[a].npts; ++q) kused[b + q] = 1;
      if (op == OPS_IR_POLY)
        for (int q = 0; q <= c; ++q) kused[b + q] = 1;
    }
    for (int a = 0; a < L.nargs; ++a) {
      if (L.args[a].kind == OPS_ARG_DAT) {
        if (ov) {
          const int k = L.args[a].slot;
          os << "  " << T << "* p" << a << " = (" << T << "*)area + " << lay->smem_off[k] << " - (ft[" << 6 * k << "] + (i64)ft["
             << 6 * k + 2 << "] * " << lay->spitch[k] << " + (i64)ft[" << 6 * k + 4 << "] * " << lay->splane[k]
             << ");\n";
        }
        else if (ro[a])
          os << "  const " << T << "* __restrict__ p" << a << " = (const " << T << "*)" << ptr_src(a) << ";\n";
        else if (restrict_all)
          os << "  " << T << "* __restrict__ p" << a << " = (" << T << "*)" << ptr_src(a) << ";\n";
        else
          os << "  " << T << "* p" << a << " = (" << T << "*)L->args[" << a << "].ptr0;\n";
      }
      if (sused[a]) os << "  const " << T << " s" << a << " = (" << T << ")scal[L->args[" << a << "].slot];\n";
    }
    for (int k = 0; k < OPS_MAX_CONSTS; ++k)
      if (kused[k]) os << "  const " << T << " K" << k << " = (" << T << ")L->K[" << k << "];\n";
    for (int k = 0; k < L.nreds; ++k) os << "  DD acc" << k << " = dd_of(red_identity(" << L.red_op[k] << "));\n";
  }

  // lay: shared-memory layout of an overlapped run (footprint of dat slot k
  // at area + smem_off[k], strides spitch[k] / splane[k], corner ft[6k..])
  void emit(int i, const OvLayout* lay = nullptr) const {
    if (ov) {
      os << "\n__device__ __forceinline__ void ovb" << i
         << "(const DLoop* __restrict__ L, const int* bx, double* area, const int* ft,\n"
            "    const double* __restrict__ scal, const int* ob, DD* part, int stride) {\n"
            "  const int x0 = bx[0], x1 = bx[1], y0 = bx[2], y1 = bx[3], z0 = bx[4], z1 = bx[5];\n";
    } else {
      os << "\n__device__ __forceinline__ void body" << i
         << "(const DLoop* __restrict__ L, int x0, int x1, int y0, int y1, int z0, int z1, int ck, int nck,\n"
            "    const double* __restrict__ scal, DD* part, int stride, int assign) {\n";
    }
    emit_hoist(lay);
    // one point
    os << "  auto one = [&](int x, int y, int z) {\n";
    for (int k = 0; k < (int)classes.size(); ++k)
      os << "    const i64 i" << k << "_0 = (i64)x + (i64)y * " << classes[k].first << "ll + (i64)z * "
         << classes[k].second << "ll;\n";
    emit_points(1);
    os << "  };\n";
    // P consecutive rows
    const int P = ov ? kOvPts : (f32 ? kJitPts32 : kJitPts);
    os << "  auto full = [&](int x, int y, int z) {\n";
    for (int k = 0; k < (int)classes.size(); ++k) {
      os << "    const i64 i" << k << "_0 = (i64)x + (i64)y * " << classes[k].first << "ll + (i64)z * "
         << classes[k].second << "ll;\n";
      for (int p = 1; p < P; ++p)
        os << "    const i64 i" << k << "_" << p << " = i" << k << "_0 + " << (int64_t)p * classes[k].first
           << "ll;\n";
    }
    emit_points(P);
    os << "  };\n";
    if (ov)
      os << "  run_units<" << P << ", " << kOvThreads << ">(x0, x1, y0, y1, z0, z1, 0, 1, one, full);\n";
    else
      os << "  run_units<" << P << ", " << nt << ">(x0, x1, y0, y1, z0, z1, ck, nck, one, full);\n";
    for (int k = 0; k < L.nreds; ++k)
      os << "  flush_red(" << L.red_op[k] << ", acc" << k << ", part, stride, L->part_row + " << k << ", "
         << (ov ? "0" : "assign") << ");\n";
    os << "}\n";
  }

  // Tile wavefront: the compute warps share one box in units of 32 x by P
  // rows (a unit per warp at a time, round robin over the warps; boxes
  // narrower than 128 in flattened groups), as the per-loop kernels do with
  // CTAs: a unit's rows sit a compile-time pitch apart, so every stencil
  // load of a point is an immediate offset from one address.  Reductions go
  // to the tile's column `col` of the partial rows (row = the loop's partial
  // row - row0), assigned.
  // warp = true: the tile-per-warp form, one warp evaluates every unit of
  // the box and reduces with shuffles alone.
  void emit_tile(int i, int NT, int P, bool warp = false) const {
    restrict_all = true;
    staged_ptrs = true;
    os << "\n__device__ __forceinline__ void tb" << i
       << "(const DLoop* __restrict__ L, void* const* ptrs, int x0, int x1, int y0, int y1, int z0, int z1,\n"
          "    const double* __restrict__ scal, DD* part, int stride, int row0, int col) {\n";
    emit_hoist(nullptr);
    os << "  auto one = [&](int x, int y, int z) {\n";
    for (int k = 0; k < (int)classes.size(); ++k)
      os << "    const i64 i" << k << "_0 = (i64)x + (i64)y * " << classes[k].first << "ll + (i64)z * "
         << classes[k].second << "ll;\n";
    emit_points(1);
    os << "  };\n";
    os << "  auto full = [&](int x, int y, int z) {\n";
    for (int k = 0; k < (int)classes.size(); ++k) {
      os << "    const i64 i" << k << "_0 = (i64)x + (i64)y * " << classes[k].first << "ll + (i64)z * "
         << classes[k].second << "ll;\n";
      for (int p = 1; p < P; ++p)
        os << "    const i64 i" << k << "_" << p << " = i" << k << "_0 + " << (int64_t)p * classes[k].first
           << "ll;\n";
    }
    emit_points(P);
    os << "  };\n";
    if (warp)
      os << "  run_units<" << P << ", 32>(x0, x1, y0, y1, z0, z1, 0, 1, one, full);\n";
    else
      os << "  run_units<" << P << ", 32>(x0, x1, y0, y1, z0, z1, (int)(threadIdx.x >> 5), " << NT / 32
         << ", one, full);\n";
    for (int k = 0; k < L.nreds; ++k)
      os << (warp ? "  flush_red_warp(" : "  flush_red_col(") << L.red_op[k] << ", acc" << k
         << ", part + (size_t)(L->part_row + " << k << " - row0) * stride + col);\n";
    os << "}\n";
  }
};

// Source of the kernels u<l0> .. u<l1-1> for loops[l0..l1) of a segment.
// batch = true: kernels ub<i> instead, one launch of loop i over several
// instances of the segment (blockIdx.y = instance; each instance's
// descriptors, scalars and reduction partials from its BatchInst).
std::string generate(const DLoop* loops, int l0, int l1, const std::vector<std::vector<char>>& ro, int es,
                     bool batch = false) {
  std::ostringstream os;
  os << "// opstile compiled loop bodies: " << pts_for(es) << " rows per unit, " << kJitMinCtas << " CTAs per SM, "
     << (es == 4 ? "fp32" : "fp64") << (batch ? ", batch of instances" : "") << "\n";
  os << kPrelude << kDeviceCommon << kPreludeTail;
  os << "static_assert(sizeof(DLoop) == " << sizeof(DLoop) << ", \"DLoop layout\");\n";
  os << "static_assert(sizeof(DArg) == " << sizeof(DArg) << ", \"DArg layout\");\n";
  if (batch)
    os << "struct BatchInst { const DLoop* loops; const double* scal; DD* part; };\n"
          "static_assert(sizeof(BatchInst) == " << sizeof(BatchInst) << ", \"BatchInst layout\");\n";
  for (int i = l0; i < l1; ++i) {
    LoopGen g(loops[i], ro[i], os, false, es == 4);
    g.emit(i);
    if (batch) {
      os << "extern \"C\" __global__ void __launch_bounds__(256, " << kJitMinCtas << ") ub" << i
         << "(const BatchInst* __restrict__ B, int x0, int x1, int y0, int y1, int z0, int z1, int stride,\n"
            "    int assign) {\n"
            "  asm volatile(\"griddepcontrol.wait;\" ::: \"memory\");\n"
            "  asm volatile(\"griddepcontrol.launch_dependents;\" ::: \"memory\");\n"
            "  const BatchInst& b = B[blockIdx.y];\n  body"
         << i << "(b.loops + " << i << ", x0, x1, y0, y1, z0, z1, blockIdx.x, gridDim.x, b.scal, b.part, stride, "
         << "assign);\n}\n";
    } else {
      os << "extern \"C\" __global__ void __launch_bounds__(256, " << kJitMinCtas << ") u" << i
         << "(const DLoop* __restrict__ L, int x0, int x1, int y0, int y1, int z0, int z1,\n"
            "    const double* __restrict__ scal, DD* part, int stride, int assign) {\n"
            "  asm volatile(\"griddepcontrol.wait;\" ::: \"memory\");\n"
            "  asm volatile(\"griddepcontrol.launch_dependents;\" ::: \"memory\");\n  body"
         << i << "(L, x0, x1, y0, y1, z0, z1, blockIdx.x, gridDim.x, scal, part, stride, assign);\n}\n";
    }
  }
  return os.str();
}

// Source of the overlapped-tile kernel "ov" for one run of loops with the
// given shared-memory layout (offsets and strides baked in).
// Bulk copies (the TMA unit) of footprint rows into shared memory, counted
// on one mbarrier; waits are bounded by wall-clock time.
const char* kOvTma = R"OVT(
__shared__ __align__(8) unsigned long long g_mbar;
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_to_shared(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               :: "r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
// true once the barrier's phase `parity` completed; false after timeout_ns
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, long long timeout_ns) {
  const unsigned long long t0 = now_ns();
  for (;;) {
    unsigned done;
    asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                 : "=r"(done) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    if (done) return true;
    if ((long long)(now_ns() - t0) > timeout_ns) return false;
  }
}
)OVT";

std::string generate_overlap(const DLoop* loops, int count, const OvLayout& lay) {
  std::ostringstream os;
  const bool f32 = lay.es == 4;
  const char* T = f32 ? "float" : "double";
  os << "// opstile overlapped tiles: " << kOvThreads << " threads, " << kOvPts << " rows per unit, "
     << (f32 ? "fp32" : "fp64") << "\n";
  os << kPrelude << kDeviceCommon << kPreludeTail << kOvTma;
  os << "static_assert(sizeof(DLoop) == " << sizeof(DLoop) << ", \"DLoop layout\");\n";
  os << "static_assert(sizeof(OvDat) == " << sizeof(OvDat) << ", \"OvDat layout\");\n";
  const std::vector<char> none(OPS_MAX_ARGS, 0);
  for (int i = 0; i < count; ++i) {
    LoopGen g(loops[i], none, os, true, f32);
    g.emit(i, &lay);
  }
  const int nd = lay.ndats;
  os << "extern \"C\" __global__ void __launch_bounds__(" << kOvThreads << ", 1) ov(const DLoop* __restrict__ loops,\n"
        "    const OvDat* __restrict__ dats, const int* __restrict__ own, const int* __restrict__ boxes,\n"
        "    const int* __restrict__ foot, int ntiles, const double* __restrict__ scal, DD* part, int stride,\n"
        "    int* err, long long timeout_ns) {\n"
        "  extern __shared__ __align__(128) double area[];\n"
        "  if (threadIdx.x == 0) mbar_init(&g_mbar);\n"
        "  __syncthreads();\n"
        "  unsigned phase = 0;\n"
        "  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {\n"
     << "    const int* ft = foot + (size_t)t * " << nd * 6 << ";\n";
  // Footprint rows start on even x (16-byte aligned in global memory; the
  // shared regions, pitches and planes are even) and hold an even number
  // of doubles, so every row is one bulk copy.  Every thread counts the
  // bytes the same way; one thread announces them on the mbarrier before
  // any copy is issued.
  os << "    unsigned bytes = 0;\n";
  for (int k = 0; k < nd; ++k)
    os << "    bytes += (unsigned)(ft[" << 6 * k + 1 << "] - ft[" << 6 * k << "]) * (unsigned)(ft[" << 6 * k + 3
       << "] - ft[" << 6 * k + 2 << "]) * (unsigned)(ft[" << 6 * k + 5 << "] - ft[" << 6 * k + 4 << "]) * "
       << lay.es << "u;\n";
  os << "    __syncthreads();  // the previous tile's reads and write-back are done\n"
        "    asm volatile(\"fence.proxy.async.shared::cta;\" ::: \"memory\");\n"
        "    if (threadIdx.x == 0) mbar_expect_tx(&g_mbar, bytes);\n"
        "    __syncthreads();\n";
  for (int k = 0; k < nd; ++k) {
    const int o = 6 * k;
    os << "    {\n      const int nx = ft[" << o + 1 << "] - ft[" << o << "], ny = ft[" << o + 3 << "] - ft[" << o + 2
       << "], nz = ft[" << o + 5 << "] - ft[" << o + 4 << "];\n"
       << "      if (nx > 0 && ny > 0 && nz > 0)\n"
       << "        for (int r = threadIdx.x; r < ny * nz; r += blockDim.x) {\n"
       << "          const int y = ft[" << o + 2 << "] + r % ny, z = ft[" << o + 4 << "] + r / ny;\n"
       << "          bulk_to_shared((" << T << "*)area + " << lay.smem_off[k] << " + (i64)(z - ft[" << o + 4
       << "]) * " << lay.splane[k] << " + (i64)(y - ft[" << o + 2 << "]) * " << lay.spitch[k] << ",\n"
       << "                         (const " << T << "*)dats[" << k << "].src + (i64)y * dats[" << k
       << "].gpitch + (i64)z * dats[" << k << "].gplane + ft[" << o << "], (unsigned)nx * " << lay.es
       << "u, &g_mbar);\n"
       << "        }\n    }\n";
  }
  os << "    bool late = !mbar_wait(&g_mbar, phase, timeout_ns);\n"
        "    if (late) {\n"
        "      atomicCAS(err, 0, 1);\n"
        "      mbar_wait(&g_mbar, phase, timeout_ns);  // the copies still in flight\n"
        "    }\n"
        "    if (__syncthreads_or(late)) return;\n"
        "    phase ^= 1u;\n";
  os << "    const int* ob = own + (size_t)t * 6;\n"
     << "    const int* bt = boxes + (size_t)t * " << count * 6 << ";\n";
  for (int i = 0; i < count; ++i) {
    os << "    if (bt[" << 6 * i + 1 << "] > bt[" << 6 * i << "] && bt[" << 6 * i + 3 << "] > bt[" << 6 * i + 2
       << "] && bt[" << 6 * i + 5 << "] > bt[" << 6 * i + 4 << "]) {\n      ovb" << i << "(loops + " << i
       << ", bt + " << 6 * i << ", area, ft, scal, ob, part, stride);\n      __syncthreads();\n    }\n";
  }
  for (int k = 0; k < nd; ++k)
    if (lay.written[k])
      os << "    copy_box<" << T << ">(ob, ft + " << 6 * k << ", (" << T << "*)area + " << lay.smem_off[k] << ", "
         << lay.spitch[k] << ", " << lay.splane[k] << ", nullptr, (" << T << "*)dats[" << k << "].dst, dats[" << k
         << "].gpitch, dats[" << k << "].gplane, false);\n";
  os << "  }\n}\n";
  return os.str();
}

// Source of the wavefront kernel "wf" for the loops of a segment.  Work
// units (a chunk of one phase) are taken in plan order from a ticket
// counter; before running its chunk a CTA waits until every phase its phase
// depends on has all its chunks done.  Every dependency points to an earlier
// phase, whose units were handed out before, to CTAs that are running: the
// earliest unfinished unit can always proceed, so the waits end.  The first
// warp polls up to 32 dependency counters at once; each wait is bounded in
// wall-clock time and a CTA that gives up sets the error word and leaves, as
// does every CTA that finds the word set.  A CTA draws its next ticket while
// the current body runs, and its first warp reports the unit done and waits
// for the next one's dependencies in the same step.
const char* kWfPrelude = R"WFP(
struct WfPhase { int loop, nchunk, ustart, dep0, ndep, pad; int box[6]; };
// Polls are relaxed loads; one acquire fence follows the last of them (an
// acquire on every poll would keep invalidating the SM's L1, which the
// stencil loads of every CTA on the SM rely on).
__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
// add with release semantics: the CTA's writes before the preceding barrier
// are visible to any thread that acquires the new value
__device__ __forceinline__ void red_release(int* p, int v) {
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}
)WFP";

std::string generate_wavefront(const DLoop* loops, int count, const std::vector<std::vector<char>>& ro, int es) {
  const int nt = jit_wave_threads();
  std::ostringstream os;
  os << "// opstile wavefront kernel: " << pts_for(es) << " rows per unit, " << nt << " threads, "
     << jit_wave_min_ctas() << " CTAs per SM, "
     << (es == 4 ? "fp32" : "fp64") << "\n";
  os << kPrelude << kDeviceCommon << kPreludeTail << kWfPrelude;
  os << "static_assert(sizeof(DLoop) == " << sizeof(DLoop) << ", \"DLoop layout\");\n";
  os << "static_assert(sizeof(WfPhase) == " << sizeof(WfPhase) << ", \"WfPhase layout\");\n";
  for (int i = 0; i < count; ++i) {
    LoopGen g(loops[i], ro[i], os, false, es == 4);
    g.nt = nt;
    g.emit(i);
  }
  // Per work unit: the body, a barrier, then the first warp reports the
  // unit done (release), and waits for the dependencies of the next unit,
  // whose ticket thread 0 drew while the body ran.
  os << "extern \"C\" __global__ void __launch_bounds__(" << nt << ", " << jit_wave_min_ctas()
     << ") wf(const DLoop* __restrict__ L,\n"
        "    const WfPhase* __restrict__ ph, const int* __restrict__ deps, const int* __restrict__ uphase,\n"
        "    int nunits, int* done, int* ticket, const double* __restrict__ scal, DD* part, int stride, int* err,\n"
        "    long long timeout_ns, int skip_unit) {\n"
        "  __shared__ int s_u, s_ok;\n"
        "  int nxt = 0;\n"
        "  if (threadIdx.x == 0) nxt = atomicAdd(ticket, 1);\n"
        "  for (int u = -1;;) {\n"
        "    if (threadIdx.x < 32) {\n"
        "      if (u >= 0 && threadIdx.x == 0 && u != skip_unit) red_release(done + uphase[u], 1);\n"
        "      const int v = __shfl_sync(0xffffffffu, nxt, 0);\n"
        "      bool ok = true;\n"
        "      if (v < nunits) {\n"
        "        const WfPhase& Q = ph[uphase[v]];\n"
        "        const int dep0 = Q.dep0, ndep = Q.ndep;\n"
        "        unsigned long long t0 = 0;\n"
        "        for (int j = threadIdx.x; ok && j < ndep; j += 32) {\n"
        "          const int d = deps[dep0 + j];\n"
        "          const int want = ph[d].nchunk;\n"
        "          unsigned spins = 0;\n"
        "          while (ld_relaxed(done + d) < want) {\n"
        "            if ((++spins & 63u) == 0) {\n"
        "              if (t0 == 0) {\n"
        "                t0 = now_ns();\n"
        "              } else if (*(volatile int*)err || (long long)(now_ns() - t0) > timeout_ns) {\n"
        "                ok = false;\n"
        "                break;\n"
        "              }\n"
        "            }\n"
        "          }\n"
        "        }\n"
        "      }\n"
        "      ok = __all_sync(0xffffffffu, ok);\n"
        "      fence_acq_rel();\n"
        "      if (threadIdx.x == 0) {\n"
        "        if (!ok) atomicCAS(err, 0, 1);\n"
        "        s_u = v;\n"
        "        s_ok = ok && !*(volatile int*)err;\n"
        "      }\n"
        "    }\n"
        "    __syncthreads();\n"
        "    u = s_u;\n"
        "    if (u >= nunits || !s_ok) return;\n"
        "    if (threadIdx.x == 0) nxt = atomicAdd(ticket, 1);\n"
        "    const WfPhase P = ph[uphase[u]];\n"
        "    const int ck = u - P.ustart;\n"
        "    switch (P.loop) {\n";
  for (int i = 0; i < count; ++i)
    os << "      case " << i << ": body" << i
       << "(L + " << i << ", P.box[0], P.box[1], P.box[2], P.box[3], P.box[4], P.box[5], ck, P.nchunk, scal, part, "
          "stride, 0); break;\n";
  os << "      default: break;\n"
        "    }\n"
        "    __syncthreads();\n"
        "  }\n"
        "}\n";
  return os.str();
}

// Source of the persistent skewed kernel "sk" (Algorithm 2 in one launch):
// every loop body of the segment behind a switch; the CTAs of one
// cooperative grid run the plan's (tile, loop) phases in order, each phase
// as a grid-stride enumeration of its box, and meet at a grid barrier only
// before the phases the plan marks (where the phase conflicts with one
// since the last barrier).  The barrier counts arrivals and bumps a
// generation word; waits are bounded in wall-clock time, after which the
// CTA sets the error word and every CTA leaves at its next barrier.
// Reductions combine into each CTA's partial column.
const char* kSkPrelude = R"SKP(
struct SkPhase { int loop, barrier; int box[6]; };
__device__ bool sk_barrier(unsigned* bar, int* err, long long timeout_ns, bool skip) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = bar + 1;
    const unsigned gen = *vgen;
    __threadfence();
    bool wait = true;
    if (!skip) {
      if (atomicAdd(bar, 1u) == gridDim.x - 1) {
        atomicExch(bar, 0u);
        __threadfence();
        atomicAdd(bar + 1, 1u);
        wait = false;
      }
    }
    if (wait) {
      const unsigned long long t0 = now_ns();
      unsigned spins = 0;
      while (*vgen == gen) {
        if (*(volatile int*)err) break;
        if ((++spins & 31u) == 0 && (long long)(now_ns() - t0) > timeout_ns) {
          atomicCAS(err, 0, 1);
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile int*)err == 0;
}
)SKP";

std::string generate_skewed(const DLoop* loops, int count, const std::vector<std::vector<char>>& ro, int es) {
  std::ostringstream os;
  os << "// opstile persistent skewed kernel: " << pts_for(es) << " rows per unit, " << kJitMinCtas
     << " CTAs per SM, " << (es == 4 ? "fp32" : "fp64") << "\n";
  os << kPrelude << kDeviceCommon << kPreludeTail << kSkPrelude;
  os << "static_assert(sizeof(DLoop) == " << sizeof(DLoop) << ", \"DLoop layout\");\n";
  os << "static_assert(sizeof(SkPhase) == " << sizeof(Phase) << ", \"Phase layout\");\n";
  for (int i = 0; i < count; ++i) {
    LoopGen g(loops[i], ro[i], os, false, es == 4);
    g.emit(i);
  }
  os << "extern \"C\" __global__ void __launch_bounds__(256, " << kJitMinCtas
     << ") sk(const DLoop* __restrict__ L,\n"
        "    const SkPhase* __restrict__ ph, int nph, const double* __restrict__ scal, DD* part, int stride,\n"
        "    unsigned* bar, int* err, long long timeout_ns, int skip_block) {\n"
        "  const bool skip = (int)blockIdx.x == skip_block;\n"
        "  for (int p = 0; p < nph; ++p) {\n"
        "    const SkPhase P = ph[p];\n"
        "    if (P.barrier && !sk_barrier(bar, err, timeout_ns, skip)) return;\n"
        "    switch (P.loop) {\n";
  for (int i = 0; i < count; ++i)
    os << "      case " << i << ": body" << i
       << "(L + " << i << ", P.box[0], P.box[1], P.box[2], P.box[3], P.box[4], P.box[5], blockIdx.x, gridDim.x, "
          "scal, part, stride, 0); break;\n";
  os << "      default: break;\n"
        "    }\n"
        "  }\n"
        "}\n";
  return os.str();
}

// Source of the tile-wavefront kernel "tw" for the loops of a segment (see
// build_tile_wave).  A persistent grid draws tiles from a ticket counter in
// the plan's order; each CTA runs every loop of its tile in order.  Its
// warps are specialised: NT compute threads evaluate the loop bodies over
// the (tile, loop) boxes, and one control warp runs a step ahead of them.
// Between two steps all threads meet at one named barrier; while the compute
// warps run step s, the control warp
//   - publishes the progress of step s - 1 (a release store of the number
//     of loops the tile has completed),
//   - makes sure step s + 1 may run: each predecessor tile (one step back in
//     a subset of the dimensions) must have completed the loops that loop
//     conflicts with; the last progress value seen of each predecessor is
//     kept, so a counter is polled (relaxed loads, then one acquire fence)
//     only when that value falls short,
//   - writes step s + 1's loop and box into a double-buffered slot.
// At the end of a tile the control warp inserts an empty step, publishes
// the tile's completion before it looks at the next tile's predecessors (a
// tile can precede the next one the same CTA draws), and reads the next
// tile's wait table.  The release and the polls thus stay off the compute
// warps' path, and the compute warps never touch the counters.  The
// earliest unfinished ticket always belongs to a running CTA whose
// predecessors have smaller tickets and are done, so the waits end; each is
// still bounded in wall-clock time, after which the CTA sets the error word
// and leaves, as does every CTA that finds it set.  Reductions combine over
// the compute warps only (a second named barrier).
const char* kTwPrelude = R"TWP(
struct TwArgs {
  const DLoop* loops; const int* rng; const int* order; const int* cls; const unsigned short* need;
  int* prog; int* ticket; const double* scal; DD* part; int* err; long long timeout_ns;
  int nt[3]; int ncls[3]; int roff[3]; int coff[3];
  int ntiles, stride, row0, skip_tile;
  const unsigned char* pf; int ahead, ngroups;
  const int* groups;
};
// Ask L2 to fetch the rows of the arguments of loop l that the mask pf[l]
// selects, over the tile's box of that loop widened by each argument's
// stencil and clipped to the dat's allocation (16-byte aligned inward:
// bulk prefetches take aligned addresses and sizes).  The whole control
// warp takes part, one row per lane.
template <int ES>
__device__ __forceinline__ void tw_prefetch(const TwArgs& A, int NL, int l, const int* tc, int lane) {
  const unsigned m = A.pf[l];
  if (!m) return;
  int b[6];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int* r = A.rng + A.roff[d] + 2 * (tc[d] * NL + l);
    b[2 * d] = r[0];
    b[2 * d + 1] = r[1];
  }
  if (b[1] <= b[0] || b[3] <= b[2] || b[5] <= b[4]) return;
  const DLoop* L = A.loops + l;
  for (int a = 0; a < 8; ++a) {
    if (!((m >> a) & 1u)) continue;
    const DArg& g = L->args[a];
    const int x0 = max(b[0] + g.slo[0], g.alo[0]), x1 = min(b[1] + g.shi[0], g.ahi[0]);
    const int y0 = max(b[2] + g.slo[1], g.alo[1]), y1 = min(b[3] + g.shi[1], g.ahi[1]);
    const int z0 = max(b[4] + g.slo[2], g.alo[2]), z1 = min(b[5] + g.shi[2], g.ahi[2]);
    if (x1 <= x0 || y1 <= y0 || z1 <= z0) continue;
    const int ny = y1 - y0, rows = ny * (z1 - z0);
    for (int r = lane; r < rows; r += 32) {
      const long long y = y0 + r % ny, z = z0 + r / ny;
      const char* base = (const char*)g.ptr0 + (y * g.pitch + z * g.plane) * ES;
      const unsigned long long a0 = ((unsigned long long)(base + (long long)x0 * ES) + 15) & ~15ull;
      const unsigned long long a1 = ((unsigned long long)(base + (long long)x1 * ES)) & ~15ull;
      if (a1 > a0)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" :: "l"(a0), "r"((unsigned)(a1 - a0)) : "memory");
    }
  }
}
__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}
// the compute warps' own barrier (named barrier 2; the step barrier is 1)
__device__ __forceinline__ void bar_compute() { asm volatile("bar.sync 2, %0;" :: "n"(kTwNtc) : "memory"); }
__device__ __forceinline__ void bar_step() { asm volatile("bar.sync 1, %0;" :: "n"(kTwNtc + 32) : "memory"); }
__device__ __forceinline__ void flush_red_warp(int op, DD v, DD* dst) {
  for (int o = 16; o > 0; o >>= 1) v = red_combine(op, v, shfl_down_dd(v, o));
  if ((threadIdx.x & 31) == 0) *dst = v;
}
__device__ __forceinline__ void flush_red_col(int op, DD v, DD* dst) {
  for (int o = 16; o > 0; o >>= 1) v = red_combine(op, v, shfl_down_dd(v, o));
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  bar_compute();
  if (lane == 0) g_sh[w] = v;
  bar_compute();
  if (w == 0) {
    v = lane < kTwNtc / 32 ? g_sh[lane] : dd_of(red_identity(op));
    for (int o = 16; o > 0; o >>= 1) v = red_combine(op, v, shfl_down_dd(v, o));
    if (lane == 0) *dst = v;
  }
  bar_compute();
}
)TWP";

// Source of the tile-per-warp kernel "tww": the tile wavefront's plan and
// arguments, but every warp is a worker of its own.  A warp draws a tile
// from the ticket counter, stages the tile's boxes and wait table in its
// slice of shared memory, and runs the tile's steps: its lanes below the
// number of predecessor directions poll the predecessors' progress
// (relaxed loads, one acquire fence, bounded wait), the warp runs the
// step's loops over the whole box in units of 32 x by P rows with a
// __syncwarp between loops, and lane 0 publishes the completed loops
// (release store).  Warps never wait for one another except through the
// progress counters, so the SM's warps hide each other's L2 latency; the
// ticket order gives the same progress guarantee as in the tile wavefront
// (the earliest unfinished tile is held by a running warp whose
// predecessors are done).  Dynamic shared memory: per warp NL boxes, the
// wait table and live flags; per CTA every loop's dat pointers.
std::string generate_tilewarp(const DLoop* loops, int count, const std::vector<std::vector<char>>& ro, int es,
                              int ndim) {
  const int wpb = jit_tilewarp_warps(), nt = 32 * wpb, P = jit_tile_pts(es), ndirs = (1 << ndim) - 1;
  std::ostringstream os;
  os << "// opstile tile-per-warp kernel: " << wpb << " warps per CTA, " << P << " rows per unit, " << ndim << "D, "
     << (es == 4 ? "fp32" : "fp64") << "\n";
  os << kPrelude << kDeviceCommon << kPreludeTail;
  os << "constexpr int kTwNtc = " << nt << ";\n" << kTwPrelude;
  os << "static_assert(sizeof(DLoop) == " << sizeof(DLoop) << ", \"DLoop layout\");\n";
  os << "static_assert(sizeof(TwArgs) == " << sizeof(TwArgs) << ", \"TwArgs layout\");\n";
  for (int i = 0; i < count; ++i) {
    LoopGen g(loops[i], ro[i], os, false, es == 4);
    g.emit_tile(i, 32, P, true);
  }
  os << "extern \"C\" __global__ void __launch_bounds__(" << nt << ", " << jit_tilewarp_min_ctas()
     << ") tww(const TwArgs A) {\n"
        "  constexpr int NL = " << count << ", ND = " << ndirs << ", WPB = " << wpb << ";\n"
        "  extern __shared__ __align__(16) unsigned char tww_smem[];\n"
        "  void** s_lptr = (void**)tww_smem;                                   // [NL][8]\n"
        "  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;\n"
        "  int* s_box = (int*)(tww_smem + sizeof(void*) * 8 * NL) + w * 6 * NL;  // [NL][6] of this warp\n"
        "  unsigned short* s_need = (unsigned short*)((int*)(tww_smem + sizeof(void*) * 8 * NL) + WPB * 6 * NL)\n"
        "                           + w * ND * NL;                              // [ND][NL] of this warp\n"
        "  unsigned char* s_live = (unsigned char*)((unsigned short*)((int*)(tww_smem + sizeof(void*) * 8 * NL)\n"
        "                           + WPB * 6 * NL) + WPB * ND * NL) + w * NL;   // [NL] of this warp\n"
        "  asm volatile(\"griddepcontrol.wait;\" ::: \"memory\");\n"
        "  for (int j = threadIdx.x; j < NL * 8; j += blockDim.x) {\n"
        "    const int l = j >> 3, a = j & 7;\n"
        "    s_lptr[j] = a < A.loops[l].nargs ? (void*)A.loops[l].args[a].ptr0 : nullptr;\n"
        "  }\n"
        "  __syncthreads();\n"
        "  int tk = 0;\n"
        "  if (lane == 0) tk = atomicAdd(A.ticket, 1);\n"
        "  tk = __shfl_sync(0xffffffffu, tk, 0);\n"
        "  while (tk < A.ntiles) {\n"
        "    const int tile = A.order[tk];\n"
        "    const int tc[3] = {tile % A.nt[0], (tile / A.nt[0]) % A.nt[1], tile / (A.nt[0] * A.nt[1])};\n"
        "    const int cl = (A.cls[A.coff[2] + tc[2]] * A.ncls[1] + A.cls[A.coff[1] + tc[1]]) * A.ncls[0] +\n"
        "                   A.cls[A.coff[0] + tc[0]];\n"
        "    int nxt = 0;\n"
        "    if (lane == 0) nxt = atomicAdd(A.ticket, 1);\n"
        "    for (int j = lane; j < ND * NL; j += 32) s_need[j] = A.need[(size_t)cl * (ND * NL) + j];\n"
        "    for (int j = lane; j < 6 * NL; j += 32) {\n"
        "      const int l = j / 6, q = j - 6 * l, d = q >> 1;\n"
        "      s_box[j] = A.rng[A.roff[d] + 2 * (tc[d] * NL + l) + (q & 1)];\n"
        "    }\n"
        "    __syncwarp();\n"
        "    for (int l = lane; l < NL; l += 32) {\n"
        "      const int* b = s_box + 6 * l;\n"
        "      s_live[l] = (b[1] > b[0] && b[3] > b[2] && b[5] > b[4]) || A.loops[l].nreds;\n"
        "    }\n"
        "    int pred = -1, have = 0x7fffffff;\n"
        "    if (lane < ND) {\n"
        "      const int m = lane + 1;\n"
        "      const int px = tc[0] - (m & 1), py = tc[1] - ((m >> 1) & 1), pz = tc[2] - ((m >> 2) & 1);\n"
        "      if (px >= 0 && py >= 0 && pz >= 0) {\n"
        "        pred = (pz * A.nt[1] + py) * A.nt[0] + px;\n"
        "        have = 0;\n"
        "      }\n"
        "    }\n"
        "    __syncwarp();\n"
        "    bool stop = false;\n"
        "    for (int g = 0; g < A.ngroups && !stop; ++g) {\n"
        "      const int l0 = A.groups[g], l1 = A.groups[g + 1];\n"
        "      bool any = false;\n"
        "      for (int l = l0; l < l1; ++l) any = any || s_live[l];\n"
        "      if (any) {\n"
        "        // may the step run?  each predecessor must have completed what its loops conflict with\n"
        "        bool ok = true;\n"
        "        if (lane < ND) {\n"
        "          int want = 0;\n"
        "          for (int l = l0; l < l1; ++l) want = max(want, (int)s_need[lane * NL + l]);\n"
        "          if (have < want) {\n"
        "            const int* pp = A.prog + pred;\n"
        "            int v = ld_relaxed(pp);\n"
        "            unsigned spins = 0;\n"
        "            unsigned long long t0 = 0;\n"
        "            while (v < want) {\n"
        "              if ((++spins & 63u) == 0) {\n"
        "                if (t0 == 0) {\n"
        "                  t0 = now_ns();\n"
        "                } else if (*(volatile int*)A.err || (long long)(now_ns() - t0) > A.timeout_ns) {\n"
        "                  ok = false;\n"
        "                  break;\n"
        "                }\n"
        "              }\n"
        "              v = ld_relaxed(pp);\n"
        "            }\n"
        "            fence_acq_rel();\n"
        "            have = v;\n"
        "          }\n"
        "        }\n"
        "        if (!__all_sync(0xffffffffu, ok)) {\n"
        "          if (lane == 0) atomicCAS(A.err, 0, 1);\n"
        "          stop = true;\n"
        "          break;\n"
        "        }\n"
        "        __syncwarp();  // the polling lanes' acquire orders the other lanes' loads\n"
        "        for (int l = l0; l < l1; ++l) {\n"
        "          if (!s_live[l]) continue;\n"
        "          const int* B = s_box + 6 * l;\n"
        "          switch (l) {\n";
  for (int i = 0; i < count; ++i)
    os << "            case " << i << ": tb" << i << "(A.loops + " << i << ", s_lptr + " << 8 * i
       << ", B[0], B[1], B[2], B[3], B[4], B[5], A.scal, A.part, A.stride, A.row0, tile); break;\n";
  os << "            default: break;\n"
        "          }\n"
        "          __syncwarp();\n"
        "        }\n"
        "      }\n"
        "      // the step's writes are ordered before lane 0's release by the __syncwarp above\n"
        "      if (lane == 0 && tile != A.skip_tile) st_release(A.prog + tile, l1);\n"
        "    }\n"
        "    tk = __shfl_sync(0xffffffffu, nxt, 0);\n"
        "    if (stop || *(volatile int*)A.err) break;\n"
        "  }\n"
        "}\n";
  return os.str();
}

std::string generate_tilewave(const DLoop* loops, int count, const std::vector<std::vector<char>>& ro, int es,
                              int ndim, bool batch) {
  const int nt = jit_tile_threads(), P = jit_tile_pts(es), ndirs = (1 << ndim) - 1;
  std::ostringstream os;
  os << "// opstile tile wavefront kernel: " << nt << " compute threads + 1 control warp, " << P
     << " points per thread at a time, " << jit_tile_min_ctas() << " CTAs per SM, " << ndim << "D, "
     << (es == 4 ? "fp32" : "fp64") << (batch ? ", batch of instances" : "") << "\n";
  os << kPrelude << kDeviceCommon << kPreludeTail;
  os << "constexpr int kTwNtc = " << nt << ";\n" << kTwPrelude;
  os << "static_assert(sizeof(DLoop) == " << sizeof(DLoop) << ", \"DLoop layout\");\n";
  os << "static_assert(sizeof(TwArgs) == " << sizeof(TwArgs) << ", \"TwArgs layout\");\n";
  for (int i = 0; i < count; ++i) {
    LoopGen g(loops[i], ro[i], os, false, es == 4);
    g.emit_tile(i, nt, P);
  }
  // Shared state: every loop's dat pointers and argument counts (loaded
  // once per launch), the current tile's box of every loop and its wait
  // table (loaded once per tile), and two slots of the step hand-over:
  // s_n[k] loops (-1: stop), their tile and their loop indices.
  // The batch kernel "twb" runs the segment for several instances (same
  // code, own dats, plans, progress counters and partials): tickets count
  // over every instance's tiles, tmap[ticket] = (instance, tile), and the
  // control warp copies an instance's arguments into shared memory when its
  // next tile belongs to another instance than the last one.
  os << "extern \"C\" __global__ void __launch_bounds__(" << nt + 32 << ", " << jit_tile_min_ctas() << ") "
     << (batch ? "twb(const TwArgs* __restrict__ AA, const int2* __restrict__ tmap, int total, int* ticket) {\n"
               "  __shared__ TwArgs s_A;\n"
               "  const TwArgs& A = s_A;\n"
               : "tw(const TwArgs A) {\n")
     << "  constexpr int NL = " << count << ", ND = " << ndirs << ", ES = " << es << ", MG = " << kTwMaxGroup << ";\n"
        "  __shared__ unsigned short s_need[ND * NL];\n"
        "  __shared__ int s_box[NL][6];\n"
        "  __shared__ void* s_lptr[NL][8];\n"
        "  __shared__ unsigned char s_live[NL];\n"
        "  __shared__ int s_n[2], s_tile[2], s_ent[2][MG];\n"
        "  asm volatile(\"griddepcontrol.wait;\" ::: \"memory\");\n"
        "  const int tid = threadIdx.x;\n"
        "  if (tid < kTwNtc) {\n"
        "    // compute warps: run the loops of each slot in turn\n"
        "    for (int k = 0;; k ^= 1) {\n"
        "      bar_step();\n"
        "      const int ne = s_n[k];\n"
        "      if (ne < 0) return;\n"
        "      const int tile = s_tile[k];\n"
        "      for (int e = 0; e < ne; ++e) {\n"
        "        const int l = s_ent[k][e];\n"
        "        const int* B = s_box[l];\n"
        "        switch (l) {\n";
  for (int i = 0; i < count; ++i)
    os << "          case " << i << ": tb" << i << "(A.loops + " << i
       << ", s_lptr[" << i << "], B[0], B[1], B[2], B[3], B[4], B[5], A.scal, A.part, A.stride, A.row0, tile); break;\n";
  os << "          default: break;\n"
        "        }\n"
        "      }\n"
        "    }\n"
        "  }\n"
        "  // control warp\n"
        "  const int lane = tid - kTwNtc;\n"
        "  auto load_ptrs = [&]() {\n"
        "    for (int j = lane; j < NL * 8; j += 32) {\n"
        "      const int l = j >> 3, a = j & 7;\n"
        "      s_lptr[l][a] = a < A.loops[l].nargs ? (void*)A.loops[l].args[a].ptr0 : nullptr;\n"
        "    }\n"
        "  };\n"
     << (batch ? "  int* const tkt = ticket;\n"
                 "  const int ntk = total;\n"
                 "  int inst = -1;\n"
               : "  load_ptrs();\n"
                 "  int* const tkt = A.ticket;\n"
                 "  const int ntk = A.ntiles;\n")
     << "  int k = 0;                         // slot of the next step\n"
        "  int pub_tile = -1, pub_val = 0;    // progress owed once the running step completes\n"
        "  bool stop = false;\n"
        "  int tk = 0, nxt = 0;\n"
        "  if (lane == 0) tk = atomicAdd(tkt, 1);\n"
        "  tk = __shfl_sync(0xffffffffu, tk, 0);\n"
        "  auto publish = [&]() {\n"
        "    if (lane == 0 && pub_tile >= 0 && pub_tile != A.skip_tile) st_release(A.prog + pub_tile, pub_val);\n"
        "  };\n"
        "  // hand slot k to the compute warps and meet them at the step barrier\n"
        "  auto post = [&](int ne, int tile) {\n"
        "    if (lane == 0) {\n"
        "      s_n[k] = ne;\n"
        "      s_tile[k] = tile;\n"
        "    }\n"
        "    __syncwarp();\n"
        "    bar_step();\n"
        "    k ^= 1;\n"
        "  };\n"
        "  while (!stop && tk < ntk) {\n"
     << (batch ? "    const int2 tm = tmap[tk];\n"
                 "    if (tm.x != inst) {\n"
                 "      // the compute warps wait at the step barrier: the instance can change\n"
                 "      inst = tm.x;\n"
                 "      if (lane == 0) s_A = AA[inst];\n"
                 "      __syncwarp();\n"
                 "      load_ptrs();\n"
                 "    }\n"
                 "    const int tile = tm.y;\n"
               : "    const int tile = A.order[tk];\n")
     << "    const int tc[3] = {tile % A.nt[0], (tile / A.nt[0]) % A.nt[1], tile / (A.nt[0] * A.nt[1])};\n"
        "    const int cl = (A.cls[A.coff[2] + tc[2]] * A.ncls[1] + A.cls[A.coff[1] + tc[1]]) * A.ncls[0] +\n"
        "                   A.cls[A.coff[0] + tc[0]];\n"
        "    if (lane == 0) nxt = atomicAdd(tkt, 1);\n"
        "    // the compute warps are past the previous tile: its boxes can be replaced\n"
        "    for (int j = lane; j < ND * NL; j += 32) s_need[j] = A.need[(size_t)cl * (ND * NL) + j];\n"
        "    for (int j = lane; j < 6 * NL; j += 32) {\n"
        "      const int l = j / 6, q = j - 6 * l, d = q >> 1;\n"
        "      s_box[l][q] = A.rng[A.roff[d] + 2 * (tc[d] * NL + l) + (q & 1)];\n"
        "    }\n"
        "    __syncwarp();\n"
        "    // a loop with reductions always runs: it writes its tile's partials (the identity when its box is empty)\n"
        "    for (int l = lane; l < NL; l += 32) {\n"
        "      const int* b = s_box[l];\n"
        "      s_live[l] = (b[1] > b[0] && b[3] > b[2] && b[5] > b[4]) || A.loops[l].nreds;\n"
        "    }\n"
        "    int pred = -1, have = 0x7fffffff;\n"
        "    if (lane < ND) {\n"
        "      const int m = lane + 1;\n"
        "      const int px = tc[0] - (m & 1), py = tc[1] - ((m >> 1) & 1), pz = tc[2] - ((m >> 2) & 1);\n"
        "      if (px >= 0 && py >= 0 && pz >= 0) {\n"
        "        pred = (pz * A.nt[1] + py) * A.nt[0] + px;\n"
        "        have = 0;\n"
        "      }\n"
        "    }\n"
        "    __syncwarp();\n"
        "    for (int l = 0; l < A.ahead && l < NL; ++l) tw_prefetch<ES>(A, NL, l, tc, lane);\n"
        "    for (int g = 0; g < A.ngroups; ++g) {\n"
        "      const int l0 = A.groups[g], l1 = A.groups[g + 1];\n"
        "      for (int l = l0 + A.ahead; l < l1 + A.ahead && l < NL; ++l) tw_prefetch<ES>(A, NL, l, tc, lane);\n"
        "      int ne = 0;\n"
        "      for (int l = l0; l < l1; ++l)\n"
        "        if (s_live[l]) {\n"
        "          if (lane == 0) s_ent[k][ne] = l;\n"
        "          ++ne;\n"
        "        }\n"
        "      if (ne == 0) {  // nothing to run: these loops count as done with the running step\n"
        "        pub_tile = tile;\n"
        "        pub_val = l1;\n"
        "        continue;\n"
        "      }\n"
        "      // may the step run?  each predecessor must have completed what its loops conflict with\n"
        "      bool ok = true;\n"
        "      if (lane < ND) {\n"
        "        int want = 0;\n"
        "        for (int l = l0; l < l1; ++l) want = max(want, (int)s_need[lane * NL + l]);\n"
        "        if (have < want) {\n"
        "          const int* pp = A.prog + pred;\n"
        "          int v = ld_relaxed(pp);\n"
        "          unsigned spins = 0;\n"
        "          unsigned long long t0 = 0;\n"
        "          while (v < want) {\n"
        "            if ((++spins & 63u) == 0) {\n"
        "              if (t0 == 0) {\n"
        "                t0 = now_ns();\n"
        "              } else if (*(volatile int*)A.err || (long long)(now_ns() - t0) > A.timeout_ns) {\n"
        "                ok = false;\n"
        "                break;\n"
        "              }\n"
        "            }\n"
        "            v = ld_relaxed(pp);\n"
        "          }\n"
        "          fence_acq_rel();  // what the predecessor wrote is visible to the compute warps after the barrier\n"
        "          have = v;\n"
        "        }\n"
        "      }\n"
        "      if (!__all_sync(0xffffffffu, ok)) {\n"
        "        if (lane == 0) atomicCAS(A.err, 0, 1);\n"
        "        stop = true;\n"
        "        break;\n"
        "      }\n"
        "      post(ne, tile);\n"
        "      publish();\n"
        "      pub_tile = tile;\n"
        "      pub_val = l1;\n"
        "    }\n"
        "    if (stop) break;\n"
        "    // an empty step: the tile's last loops complete, then its progress is published\n"
        "    post(0, tile);\n"
        "    publish();\n"
        "    pub_tile = -1;\n"
        "    tk = __shfl_sync(0xffffffffu, nxt, 0);\n"
        "    if (*(volatile int*)A.err) stop = true;\n"
        "  }\n"
        "  post(-1, -1);\n"
        "  publish();\n"
        "}\n";
  return os.str();
}

uint64_t fnv64(const std::string& s) {
  uint64_t h = 1469598103934665603ull;
  for (unsigned char ch : s) {
    h ^= ch;
    h *= 1099511628211ull;
  }
  return h;
}

std::string cache_dir() {
  const char* e = getenv("OPSTILE_JIT_CACHE");
  if (e && *e) return e;
  const char* home = getenv("HOME");
  return std::string(home && *home ? home : "/tmp") + "/.cache/opstile-jit";
}

bool read_file(const std::string& path, std::string* out) {
  std::ifstream f(path, std::ios::binary);
  if (!f) return false;
  std::ostringstream ss;
  ss << f.rdbuf();
  *out = ss.str();
  return true;
}

void write_file(const std::string& path, const std::string& data) {
  const std::string tmp = path + ".tmp" + std::to_string((long)getpid());
  {
    std::ofstream f(tmp, std::ios::binary);
    if (!f) return;
    f.write(data.data(), (std::streamsize)data.size());
    if (!f) return;
  }
  std::rename(tmp.c_str(), path.c_str());
}

void mkdirs(const std::string& dir) {
  std::string cur;
  std::stringstream ss(dir);
  std::string part;
  if (!dir.empty() && dir[0] == '/') cur = "/";
  while (std::getline(ss, part, '/')) {
    if (part.empty()) continue;
    cur += part + "/";
    mkdir(cur.c_str(), 0755);
  }
}

// call with g_mu held
bool compile(const std::string& src, std::string* cubin, std::string* why) {
  nvrtcProgram prog;
  if (g_api.create(&prog, src.c_str(), "opstile_segment.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS) {
    *why = "nvrtcCreateProgram failed";
    return false;
  }
  // unused IR registers are declared for every point: silence those notes
  const char* opts[] = {"--gpu-architecture=sm_103a", "-fmad=false", "--std=c++17", "-default-device",
                        "--diag-suppress=177,550"};
  const nvrtcResult rc = g_api.compile(prog, 5, opts);
  if (rc != NVRTC_SUCCESS) {
    size_t n = 0;
    g_api.log_size(prog, &n);
    std::string log(n, '\0');
    if (n) g_api.log(prog, &log[0]);
    *why = "NVRTC: " + log.substr(0, 20000);
    g_api.destroy(&prog);
    return false;
  }
  size_t n = 0;
  g_api.cubin_size(prog, &n);
  cubin->assign(n, '\0');
  g_api.cubin(prog, &(*cubin)[0]);
  g_api.destroy(&prog);
  return true;
}

}  // namespace

struct JitSegment {
  std::vector<CUfunction> u;
  std::vector<int> per_sm;  // resident CTAs per SM of each kernel (0: not queried yet)
};

namespace {
// loaded modules by (device, source); segments by (device, concatenated sources)
std::map<std::pair<int, std::string>, CUmodule> g_modules;
std::map<std::pair<int, std::string>, std::unique_ptr<JitSegment>> g_segments;

std::string cache_base(const std::string& src) {
  char hx[17];
  std::snprintf(hx, sizeof hx, "%016llx", (unsigned long long)fnv64(src));
  return cache_dir() + "/" + hx;
}
}  // namespace

int jit_segment(int device, const DLoop* loops, int count, const std::vector<std::vector<char>>& ro, int es,
                JitSegment** out, std::string* why, double* compile_ms, bool batch) {
  *out = nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!api_ready(why)) return OPS_OK;
  auto t0 = std::chrono::steady_clock::now();
  std::vector<std::string> srcs;
  std::string all;
  for (int l0 = 0; l0 < count; l0 += kJitChunk) {
    srcs.push_back(generate(loops, l0, std::min(count, l0 + kJitChunk), ro, es, batch));
    all += srcs.back();
  }
  auto skey = std::make_pair(device, all);
  auto it = g_segments.find(skey);
  if (it != g_segments.end()) {
    *out = it->second.get();
    return OPS_OK;
  }
  // cubins from the disk cache, the rest compiled in parallel
  const int nm = (int)srcs.size();
  std::vector<std::string> cubin(nm), err(nm);
  std::vector<char> need(nm, 0);
  for (int m = 0; m < nm; ++m) {
    if (g_modules.count(std::make_pair(device, srcs[m]))) continue;
    std::string cached;
    const std::string base = cache_base(srcs[m]);
    if (read_file(base + ".cu", &cached) && cached == srcs[m] && read_file(base + ".cubin", &cubin[m]) &&
        !cubin[m].empty())
      continue;
    need[m] = 1;
  }
  {
    std::vector<std::thread> th;
    for (int m = 0; m < nm; ++m)
      if (need[m]) th.emplace_back([&, m] {
          if (!compile(srcs[m], &cubin[m], &err[m])) cubin[m].clear();
        });
    for (std::thread& t : th) t.join();
  }
  for (int m = 0; m < nm; ++m) {
    if (!need[m]) continue;
    if (cubin[m].empty()) {
      *why = err[m];
      return OPS_ERR_CUDA;
    }
    mkdirs(cache_dir());
    const std::string base = cache_base(srcs[m]);
    write_file(base + ".cubin", cubin[m]);
    write_file(base + ".cu", srcs[m]);
  }
  std::unique_ptr<JitSegment> s(new JitSegment);
  s->u.resize(count);
  for (int m = 0; m < nm; ++m) {
    auto mk = std::make_pair(device, srcs[m]);
    CUmodule mod;
    auto mi = g_modules.find(mk);
    if (mi != g_modules.end()) {
      mod = mi->second;
    } else {
      if (g_api.load(&mod, cubin[m].data()) != CUDA_SUCCESS) {
        *why = "cuModuleLoadData failed";
        return OPS_ERR_CUDA;
      }
      g_modules[mk] = mod;
    }
    for (int i = m * kJitChunk; i < std::min(count, (m + 1) * kJitChunk); ++i) {
      const std::string name = (batch ? "ub" : "u") + std::to_string(i);
      if (g_api.get_function(&s->u[i], mod, name.c_str()) != CUDA_SUCCESS) {
        *why = "cuModuleGetFunction failed";
        return OPS_ERR_CUDA;
      }
    }
  }
  if (compile_ms)
    *compile_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *out = s.get();
  g_segments[skey] = std::move(s);
  return OPS_OK;
}

int jit_compile_only(const DLoop* loops, int count, const std::vector<std::vector<char>>& ro, int es,
                     std::string* src, std::string* why, double* compile_ms) {
  std::lock_guard<std::mutex> lk(g_mu);
  std::vector<std::string> srcs;
  src->clear();
  for (int l0 = 0; l0 < count; l0 += kJitChunk) {
    srcs.push_back(generate(loops, l0, std::min(count, l0 + kJitChunk), ro, es));
    *src += srcs.back();
  }
  if (!api_ready(why, true)) {
    if (why->empty()) *why = g_api.why;
    return OPS_ERR_NO_DEVICE;
  }
  auto t0 = std::chrono::steady_clock::now();
  const int nm = (int)srcs.size();
  std::vector<std::string> cubin(nm), err(nm);
  std::vector<char> ok(nm, 0);
  {
    std::vector<std::thread> th;
    for (int m = 0; m < nm; ++m) th.emplace_back([&, m] { ok[m] = compile(srcs[m], &cubin[m], &err[m]); });
    for (std::thread& t : th) t.join();
  }
  if (compile_ms)
    *compile_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  for (int m = 0; m < nm; ++m)
    if (!ok[m]) {
      *why = err[m];
      return OPS_ERR_CUDA;
    }
  return OPS_OK;
}

struct JitOverlap {
  CUfunction f = nullptr;
  int area_set = -1;  // dynamic shared memory the function is opted into
};

namespace {
std::map<std::pair<int, std::string>, std::unique_ptr<JitOverlap>> g_overlaps;

}  // namespace

int jit_overlap_many(int device, const std::vector<OvRequest>& reqs, std::vector<JitOverlap*>* out, std::string* why,
                     double* compile_ms) {
  out->assign(reqs.size(), nullptr);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!api_ready(why)) return OPS_OK;
  auto t0 = std::chrono::steady_clock::now();
  const int nr = (int)reqs.size();
  std::vector<std::string> src(nr), cubin(nr), err(nr);
  std::vector<char> need(nr, 0), ok(nr, 1);
  for (int r = 0; r < nr; ++r) {
    src[r] = generate_overlap(reqs[r].loops, reqs[r].count, reqs[r].lay);
    auto it = g_overlaps.find(std::make_pair(device, src[r]));
    if (it != g_overlaps.end()) {
      (*out)[r] = it->second.get();
      continue;
    }
    std::string cached;
    const std::string base = cache_base(src[r]);
    if (read_file(base + ".cu", &cached) && cached == src[r] && read_file(base + ".cubin", &cubin[r]) &&
        !cubin[r].empty())
      continue;
    need[r] = 1;
  }
  {
    std::vector<std::thread> th;
    for (int r = 0; r < nr; ++r)
      if (need[r]) th.emplace_back([&, r] { ok[r] = compile(src[r], &cubin[r], &err[r]); });
    for (std::thread& t : th) t.join();
  }
  for (int r = 0; r < nr; ++r) {
    if ((*out)[r]) continue;
    if (!ok[r]) {
      *why = err[r];
      return OPS_ERR_CUDA;
    }
    if (need[r]) {
      mkdirs(cache_dir());
      const std::string base = cache_base(src[r]);
      write_file(base + ".cubin", cubin[r]);
      write_file(base + ".cu", src[r]);
    }
    auto key = std::make_pair(device, src[r]);
    auto it = g_overlaps.find(key);  // an identical run earlier in this batch
    if (it != g_overlaps.end()) {
      (*out)[r] = it->second.get();
      continue;
    }
    CUmodule mod;
    if (g_api.load(&mod, cubin[r].data()) != CUDA_SUCCESS) {
      *why = "cuModuleLoadData failed";
      return OPS_ERR_CUDA;
    }
    std::unique_ptr<JitOverlap> o(new JitOverlap);
    if (g_api.get_function(&o->f, mod, "ov") != CUDA_SUCCESS) {
      *why = "cuModuleGetFunction failed";
      return OPS_ERR_CUDA;
    }
    (*out)[r] = o.get();
    g_overlaps[key] = std::move(o);
  }
  if (compile_ms)
    *compile_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return OPS_OK;
}

int jit_overlap_max_grid(JitOverlap* o, int num_sms, int area_bytes) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (o->area_set != area_bytes) {
    if (g_api.set_attribute(o->f, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, area_bytes) != CUDA_SUCCESS)
      return 0;
    o->area_set = area_bytes;
  }
  int per_sm = 0;
  if (g_api.occupancy(&per_sm, o->f, kOvThreads, (size_t)area_bytes) != CUDA_SUCCESS) return 0;
  return per_sm * num_sms;
}

cudaError_t jit_launch_overlap(const JitOverlap* o, const LaunchEnv& env, const DLoop* d_loops, const OvDat* d_dats,
                               const int* d_own, const int* d_boxes, const int* d_foot, int ntiles, int grid,
                               int area_bytes) {
  const DLoop* a0 = d_loops;
  const OvDat* a1 = d_dats;
  const int *a2 = d_own, *a3 = d_boxes, *a4 = d_foot;
  int a5 = ntiles;
  const double* a6 = env.scal;
  DD* a7 = env.part;
  int a8 = env.part_stride;
  int* a9 = env.err;
  long long a10 = env.timeout_ns;
  void* args[] = {&a0, &a1, &a2, &a3, &a4, &a5, &a6, &a7, &a8, &a9, &a10};
  return to_cuda(g_api.launch(o->f, (unsigned)grid, 1, 1, kOvThreads, 1, 1, (unsigned)area_bytes,
                              (CUstream)env.stream, args, nullptr));
}

int jit_compile_overlap_only(const DLoop* loops, int count, const OvLayout& lay, std::string* src, std::string* why,
                             double* compile_ms) {
  std::lock_guard<std::mutex> lk(g_mu);
  // runs of kJitChunk loops, compiled in parallel (a run's code does not depend on the others)
  std::vector<std::string> srcs;
  src->clear();
  for (int l0 = 0; l0 < count; l0 += kJitChunk) {
    srcs.push_back(generate_overlap(loops + l0, std::min(kJitChunk, count - l0), lay));
    *src += srcs.back();
  }
  if (!api_ready(why, true)) {
    if (why->empty()) *why = g_api.why;
    return OPS_ERR_NO_DEVICE;
  }
  auto t0 = std::chrono::steady_clock::now();
  const int nm = (int)srcs.size();
  std::vector<std::string> cubin(nm), err(nm);
  std::vector<char> ok(nm, 0);
  {
    std::vector<std::thread> th;
    for (int m = 0; m < nm; ++m) th.emplace_back([&, m] { ok[m] = compile(srcs[m], &cubin[m], &err[m]); });
    for (std::thread& t : th) t.join();
  }
  if (compile_ms)
    *compile_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  for (int m = 0; m < nm; ++m)
    if (!ok[m]) {
      *why = err[m];
      return OPS_ERR_CUDA;
    }
  return OPS_OK;
}

bool jit_available() {
  std::lock_guard<std::mutex> lk(g_mu);
  return api_ready(nullptr);
}

int jit_pdl() {
  static const int v = env_int("OPSTILE_PDL", 1, 0, 1);
  return v;
}

int jit_grid_policy() {
  static const int v = env_int("OPSTILE_JIT_GRID", 0, 0, 64);
  return v;
}

int jit_resident(JitSegment* s, int i) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (s->per_sm.size() != s->u.size()) s->per_sm.assign(s->u.size(), 0);
  if (!s->per_sm[i]) {
    int per_sm = 0;
    if (g_api.occupancy(&per_sm, s->u[i], kThreads, 0) != CUDA_SUCCESS || per_sm < 1) per_sm = 1;
    s->per_sm[i] = per_sm;
  }
  return s->per_sm[i];
}

cudaError_t jit_launch(const JitSegment* s, int i, const LaunchEnv& env, const DLoop* d_loop, const int* box,
                       int grid, int assign) {
  const DLoop* a0 = d_loop;
  int b0 = box[0], b1 = box[1], b2 = box[2], b3 = box[3], b4 = box[4], b5 = box[5];
  const double* sc = env.scal;
  DD* pt = env.part;
  int st = env.part_stride;
  int as = assign;
  void* args[] = {&a0, &b0, &b1, &b2, &b3, &b4, &b5, &sc, &pt, &st, &as};
  if (g_api.launch_ex && jit_pdl()) {
    CUlaunchAttribute at[1];
    std::memset(at, 0, sizeof at);
    at[0].id = CU_LAUNCH_ATTRIBUTE_PROGRAMMATIC_STREAM_SERIALIZATION;
    at[0].value.programmaticStreamSerializationAllowed = 1;
    CUlaunchConfig cfg;
    std::memset(&cfg, 0, sizeof cfg);
    cfg.gridDimX = (unsigned)grid;
    cfg.gridDimY = cfg.gridDimZ = 1;
    cfg.blockDimX = kThreads;
    cfg.blockDimY = cfg.blockDimZ = 1;
    cfg.hStream = (CUstream)env.stream;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return to_cuda(g_api.launch_ex(&cfg, s->u[i], args, nullptr));
  }
  return to_cuda(g_api.launch(s->u[i], (unsigned)grid, 1, 1, kThreads, 1, 1, 0, (CUstream)env.stream, args, nullptr));
}

cudaError_t jit_launch_batch(const JitSegment* s, int i, cudaStream_t stream, const BatchInst* d_inst, int ninst,
                             const int* box, int grid, int stride) {
  const BatchInst* a0 = d_inst;
  int b0 = box[0], b1 = box[1], b2 = box[2], b3 = box[3], b4 = box[4], b5 = box[5];
  int st = stride, as = 1;
  void* args[] = {&a0, &b0, &b1, &b2, &b3, &b4, &b5, &st, &as};
  if (g_api.launch_ex && jit_pdl()) {
    CUlaunchAttribute at[1];
    std::memset(at, 0, sizeof at);
    at[0].id = CU_LAUNCH_ATTRIBUTE_PROGRAMMATIC_STREAM_SERIALIZATION;
    at[0].value.programmaticStreamSerializationAllowed = 1;
    CUlaunchConfig cfg;
    std::memset(&cfg, 0, sizeof cfg);
    cfg.gridDimX = (unsigned)grid;
    cfg.gridDimY = (unsigned)ninst;
    cfg.gridDimZ = 1;
    cfg.blockDimX = kThreads;
    cfg.blockDimY = cfg.blockDimZ = 1;
    cfg.hStream = (CUstream)stream;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return to_cuda(g_api.launch_ex(&cfg, s->u[i], args, nullptr));
  }
  return to_cuda(g_api.launch(s->u[i], (unsigned)grid, (unsigned)ninst, 1, kThreads, 1, 1, 0, (CUstream)stream, args,
                              nullptr));
}


int jit_rows_per_unit(int es) { return pts_for(es); }

int jit_wave_units_per_chunk() {
  static const int v = env_int("OPSTILE_WF_UNITS", 16, 1, 1 << 20);
  return v;
}

int jit_wave_threads() {
  // 32, 64, 128 or 256 (OPSTILE_WF_THREADS rounds down to one of them)
  static const int v = [] {
    int t = env_int("OPSTILE_WF_THREADS", 128, 32, 256), p = 32;
    while (p * 2 <= t) p *= 2;
    return p;
  }();
  return v;
}

int jit_wave_min_ctas() {
  static const int v = env_int("OPSTILE_WF_MINB", (kJitMinCtas * kThreads) / jit_wave_threads(), 1, 32);
  return v;
}

int jit_wave_slope() {
  static const int v = env_int("OPSTILE_WF_SLOPE", 1, 0, 1 << 20);
  return v;
}

struct JitWave {
  CUfunction f = nullptr;
};

namespace {
std::map<std::pair<int, std::string>, std::unique_ptr<JitWave>> g_waves;

bool cubin_for(const std::string& src, std::string* cubin, std::string* why) {
  std::string cached;
  const std::string base = cache_base(src);
  if (read_file(base + ".cu", &cached) && cached == src && read_file(base + ".cubin", cubin) && !cubin->empty())
    return true;
  if (!compile(src, cubin, why)) return false;
  mkdirs(cache_dir());
  write_file(base + ".cubin", *cubin);
  write_file(base + ".cu", src);
  return true;
}
}  // namespace

int jit_wavefront(int device, const DLoop* loops, int count, const std::vector<std::vector<char>>& ro, int es,
                  JitWave** out, std::string* why, double* compile_ms) {
  *out = nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!api_ready(why)) return OPS_OK;
  auto t0 = std::chrono::steady_clock::now();
  const std::string src = generate_wavefront(loops, count, ro, es);
  auto key = std::make_pair(device, src);
  auto it = g_waves.find(key);
  if (it != g_waves.end()) {
    *out = it->second.get();
    return OPS_OK;
  }
  std::string cubin;
  if (!cubin_for(src, &cubin, why)) return OPS_ERR_CUDA;
  CUmodule mod;
  if (g_api.load(&mod, cubin.data()) != CUDA_SUCCESS) {
    *why = "cuModuleLoadData failed";
    return OPS_ERR_CUDA;
  }
  std::unique_ptr<JitWave> w(new JitWave);
  if (g_api.get_function(&w->f, mod, "wf") != CUDA_SUCCESS) {
    *why = "cuModuleGetFunction failed";
    return OPS_ERR_CUDA;
  }
  if (compile_ms)
    *compile_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *out = w.get();
  g_waves[key] = std::move(w);
  return OPS_OK;
}

struct JitSkew {
  CUfunction f = nullptr;
  int per_sm = 0;
};

namespace {
std::map<std::pair<int, std::string>, std::unique_ptr<JitSkew>> g_skews;
}  // namespace

int jit_skewed(int device, const DLoop* loops, int count, const std::vector<std::vector<char>>& ro, int es,
               JitSkew** out, std::string* why, double* compile_ms) {
  *out = nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!api_ready(why)) return OPS_OK;
  auto t0 = std::chrono::steady_clock::now();
  const std::string src = generate_skewed(loops, count, ro, es);
  auto key = std::make_pair(device, src);
  auto it = g_skews.find(key);
  if (it != g_skews.end()) {
    *out = it->second.get();
    return OPS_OK;
  }
  std::string cubin;
  if (!cubin_for(src, &cubin, why)) return OPS_ERR_CUDA;
  CUmodule mod;
  if (g_api.load(&mod, cubin.data()) != CUDA_SUCCESS) {
    *why = "cuModuleLoadData failed";
    return OPS_ERR_CUDA;
  }
  std::unique_ptr<JitSkew> k(new JitSkew);
  if (g_api.get_function(&k->f, mod, "sk") != CUDA_SUCCESS) {
    *why = "cuModuleGetFunction failed";
    return OPS_ERR_CUDA;
  }
  if (g_api.occupancy(&k->per_sm, k->f, kThreads, 0) != CUDA_SUCCESS || k->per_sm < 1) {
    *why = "the persistent skewed kernel does not fit an SM";
    return OPS_ERR_CUDA;
  }
  if (compile_ms)
    *compile_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *out = k.get();
  g_skews[key] = std::move(k);
  return OPS_OK;
}

int jit_compile_skewed_only(const DLoop* loops, int count, const std::vector<std::vector<char>>& ro, int es,
                            std::string* src, std::string* why, double* compile_ms) {
  std::lock_guard<std::mutex> lk(g_mu);
  *src = generate_skewed(loops, count, ro, es);
  if (!api_ready(why, true)) {
    if (why->empty()) *why = g_api.why;
    return OPS_ERR_NO_DEVICE;
  }
  auto t0 = std::chrono::steady_clock::now();
  std::string cubin;
  const bool ok = compile(*src, &cubin, why);
  if (compile_ms)
    *compile_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return ok ? OPS_OK : OPS_ERR_CUDA;
}

int jit_skewed_max_grid(JitSkew* k, int num_sms) { return k->per_sm * num_sms; }

cudaError_t jit_launch_skewed(const JitSkew* k, const LaunchEnv& env, const DLoop* d_loops, const Phase* d_phases,
                              int nphases, int grid) {
  cudaError_t e = cudaMemsetAsync(env.bar, 0, 2 * sizeof(unsigned), env.stream);
  if (e != cudaSuccess) return e;
  const DLoop* a0 = d_loops;
  const Phase* a1 = d_phases;
  int a2 = nphases;
  const double* a3 = env.scal;
  DD* a4 = env.part;
  int a5 = env.part_stride;
  unsigned* a6 = env.bar;
  int* a7 = env.err;
  long long a8 = env.timeout_ns;
  int a9 = env.skip_block;
  void* args[] = {&a0, &a1, &a2, &a3, &a4, &a5, &a6, &a7, &a8, &a9};
  return to_cuda(g_api.launch_coop(k->f, (unsigned)grid, 1, 1, kThreads, 1, 1, 0, (CUstream)env.stream, args));
}

int jit_compile_wavefront_only(const DLoop* loops, int count, const std::vector<std::vector<char>>& ro, int es,
                               std::string* src, std::string* why, double* compile_ms) {
  std::lock_guard<std::mutex> lk(g_mu);
  *src = generate_wavefront(loops, count, ro, es);
  if (!api_ready(why, true)) {
    if (why->empty()) *why = g_api.why;
    return OPS_ERR_NO_DEVICE;
  }
  auto t0 = std::chrono::steady_clock::now();
  std::string cubin;
  const bool ok = compile(*src, &cubin, why);
  if (compile_ms)
    *compile_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return ok ? OPS_OK : OPS_ERR_CUDA;
}

int jit_wavefront_max_grid(JitWave* w, int num_sms) {
  std::lock_guard<std::mutex> lk(g_mu);
  int per_sm = 0;
  if (g_api.occupancy(&per_sm, w->f, jit_wave_threads(), 0) != CUDA_SUCCESS) return 0;
  return per_sm * num_sms;
}

cudaError_t jit_launch_wavefront(const JitWave* w, const LaunchEnv& env, const DLoop* d_loops,
                                 const WfPhase* d_phases, const int* d_deps, const int* d_uphase, int nunits,
                                 int* d_done, int* d_ticket, int grid) {
  const DLoop* a0 = d_loops;
  const WfPhase* a1 = d_phases;
  const int *a2 = d_deps, *a3 = d_uphase;
  int a4 = nunits;
  int *a5 = d_done, *a6 = d_ticket;
  const double* a7 = env.scal;
  DD* a8 = env.part;
  int a9 = env.part_stride;
  int* a10 = env.err;
  long long a11 = env.timeout_ns;
  int a12 = env.skip_block;
  void* args[] = {&a0, &a1, &a2, &a3, &a4, &a5, &a6, &a7, &a8, &a9, &a10, &a11, &a12};
  return to_cuda(
      g_api.launch(w->f, (unsigned)grid, 1, 1, jit_wave_threads(), 1, 1, 0, (CUstream)env.stream, args, nullptr));
}


int jit_tile_threads() {
  // whole warps, with room for the control warp in a 1024-thread CTA
  static const int v = env_int("OPSTILE_TW_THREADS", 256, 128, 992) / 32 * 32;
  return v;
}

int jit_tile_min_ctas() {
  static const int v = env_int("OPSTILE_TW_MINB", 2, 1, 16);
  return v;
}

int jit_tile_pts(int es) {
  static const int v32 = env_int("OPSTILE_TW_PTS32", 8, 1, 8), v64 = env_int("OPSTILE_TW_PTS", 4, 1, 8);
  return es == 4 ? v32 : v64;
}

int jit_tile_prefetch() {
  static const int v = env_int("OPSTILE_TW_PREFETCH", 0, 0, 2);
  return v;
}

int jit_tile_group() {
  static const int v = env_int("OPSTILE_TW_GROUP", kTwMaxGroup, 1, kTwMaxGroup);
  return v;
}

int jit_tile_band() {
  static const int v = env_int("OPSTILE_TW_BAND", 16, 0, 1 << 20);
  return v;
}

int jit_tile_ahead() {
  static const int v = env_int("OPSTILE_TW_AHEAD", 3, 0, 64);
  return v;
}

struct JitTile {
  CUfunction f = nullptr;
  int threads = 0;   // block size
  int smem = 0;      // dynamic shared memory bytes
};

namespace {
std::map<std::pair<int, std::string>, std::unique_ptr<JitTile>> g_tiles;
}  // namespace

int jit_tilewave(int device, const DLoop* loops, int count, const std::vector<std::vector<char>>& ro, int es, int ndim,
                 JitTile** out, std::string* why, double* compile_ms, bool batch) {
  *out = nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!api_ready(why)) return OPS_OK;
  auto t0 = std::chrono::steady_clock::now();
  const std::string src = generate_tilewave(loops, count, ro, es, ndim, batch);
  auto key = std::make_pair(device, src);
  auto it = g_tiles.find(key);
  if (it != g_tiles.end()) {
    *out = it->second.get();
    return OPS_OK;
  }
  std::string cubin;
  if (!cubin_for(src, &cubin, why)) return OPS_ERR_CUDA;
  CUmodule mod;
  if (g_api.load(&mod, cubin.data()) != CUDA_SUCCESS) {
    *why = "cuModuleLoadData failed";
    return OPS_ERR_CUDA;
  }
  std::unique_ptr<JitTile> t(new JitTile);
  if (g_api.get_function(&t->f, mod, batch ? "twb" : "tw") != CUDA_SUCCESS) {
    *why = "cuModuleGetFunction failed";
    return OPS_ERR_CUDA;
  }
  t->threads = jit_tile_threads() + 32;
  if (compile_ms)
    *compile_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *out = t.get();
  g_tiles[key] = std::move(t);
  return OPS_OK;
}

int jit_compile_tilewave_only(const DLoop* loops, int count, const std::vector<std::vector<char>>& ro, int es,
                              int ndim, std::string* src, std::string* why, double* compile_ms, bool batch) {
  std::lock_guard<std::mutex> lk(g_mu);
  *src = generate_tilewave(loops, count, ro, es, ndim, batch);
  if (!api_ready(why, true)) {
    if (why->empty()) *why = g_api.why;
    return OPS_ERR_NO_DEVICE;
  }
  auto t0 = std::chrono::steady_clock::now();
  std::string cubin;
  const bool ok = compile(*src, &cubin, why);
  if (compile_ms)
    *compile_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return ok ? OPS_OK : OPS_ERR_CUDA;
}

int jit_tilewave_max_grid(JitTile* t, int num_sms) {
  std::lock_guard<std::mutex> lk(g_mu);
  int per_sm = 0;
  if (g_api.occupancy(&per_sm, t->f, t->threads, (size_t)t->smem) != CUDA_SUCCESS) return 0;
  return per_sm * num_sms;
}

cudaError_t jit_launch_tilewave(const JitTile* t, const TwArgs& args, cudaStream_t stream, int grid) {
  TwArgs a = args;
  void* params[] = {&a};
  return to_cuda(g_api.launch(t->f, (unsigned)grid, 1, 1, (unsigned)t->threads, 1, 1, (unsigned)t->smem,
                              (CUstream)stream, params, nullptr));
}

int jit_tilewarp_warps() {
  static const int v = env_int("OPSTILE_TWW_WARPS", 4, 1, 32);
  return v;
}

int jit_tilewarp_min_ctas() {
  static const int v = env_int("OPSTILE_TWW_MINB", 4, 1, 32);
  return v;
}

int jit_tilewarp_smem(int count, int ndim) {
  const int wpb = jit_tilewarp_warps(), nd = (1 << ndim) - 1;
  return (int)(sizeof(void*) * 8 * count + sizeof(int) * wpb * 6 * count + sizeof(unsigned short) * wpb * nd * count +
               (size_t)wpb * count + 16);
}

std::map<std::pair<int, std::string>, std::unique_ptr<JitTile>> g_warps;

int jit_tilewarp(int device, const DLoop* loops, int count, const std::vector<std::vector<char>>& ro, int es, int ndim,
                 JitTile** out, std::string* why, double* compile_ms) {
  *out = nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!api_ready(why)) return OPS_OK;
  auto t0 = std::chrono::steady_clock::now();
  const std::string src = generate_tilewarp(loops, count, ro, es, ndim);
  auto key = std::make_pair(device, src);
  auto it = g_warps.find(key);
  if (it != g_warps.end()) {
    *out = it->second.get();
    return OPS_OK;
  }
  std::string cubin;
  if (!cubin_for(src, &cubin, why)) return OPS_ERR_CUDA;
  CUmodule mod;
  if (g_api.load(&mod, cubin.data()) != CUDA_SUCCESS) {
    *why = "cuModuleLoadData failed";
    return OPS_ERR_CUDA;
  }
  std::unique_ptr<JitTile> t(new JitTile);
  if (g_api.get_function(&t->f, mod, "tww") != CUDA_SUCCESS) {
    *why = "cuModuleGetFunction failed";
    return OPS_ERR_CUDA;
  }
  t->threads = 32 * jit_tilewarp_warps();
  t->smem = jit_tilewarp_smem(count, ndim);
  if (t->smem > 48 * 1024 &&
      g_api.set_attribute(t->f, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, t->smem) != CUDA_SUCCESS) {
    *why = "the tile-per-warp kernel's shared memory does not fit";
    return OPS_ERR_CUDA;
  }
  if (compile_ms)
    *compile_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *out = t.get();
  g_warps[key] = std::move(t);
  return OPS_OK;
}

int jit_compile_tilewarp_only(const DLoop* loops, int count, const std::vector<std::vector<char>>& ro, int es,
                              int ndim, std::string* src, std::string* why, double* compile_ms) {
  std::lock_guard<std::mutex> lk(g_mu);
  *src = generate_tilewarp(loops, count, ro, es, ndim);
  if (!api_ready(why, true)) {
    if (why->empty()) *why = g_api.why;
    return OPS_ERR_NO_DEVICE;
  }
  auto t0 = std::chrono::steady_clock::now();
  std::string cubin;
  const bool ok = compile(*src, &cubin, why);
  if (compile_ms)
    *compile_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return ok ? OPS_OK : OPS_ERR_CUDA;
}

cudaError_t jit_launch_tilewave_batch(const JitTile* t, const TwArgs* d_args, const int* d_tmap, int total,
                                      int* d_ticket, cudaStream_t stream, int grid) {
  const TwArgs* aa = d_args;
  const int* tm = d_tmap;
  int tot = total;
  int* tk = d_ticket;
  void* params[] = {&aa, &tm, &tot, &tk};
  return to_cuda(g_api.launch(t->f, (unsigned)grid, 1, 1, (unsigned)t->threads, 1, 1, 0, (CUstream)stream, params,
                              nullptr));
}

}  // namespace opstile
