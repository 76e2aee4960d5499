// Internal structures shared by the host runtime (runtime.cpp, plan.cpp) and
// the device kernels (chain_kernels.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "opstile.h"

namespace opstile {

constexpr int kNReg = 8;
constexpr int kThreads = 256;  // threads per CTA of every chain kernel
// Kernels index the points of one loop with 32-bit ints (plus a grid-stride
// margin), so a loop covers fewer than 2^31 - 2^24 points.
constexpr int kMaxLoopPoints = (1 << 30) + ((1 << 30) - (1 << 24));

// Device error word values (first writer wins).
constexpr int kDevErrTimeout = 1;
constexpr int kDevErrBounds = 2;

// One argument of a loop, resolved to device addresses.
struct DArg {
  double* ptr0;       // grid point (0,0,0) of the dat
  int64_t pitch;      // elements between consecutive y
  int64_t plane;      // elements between consecutive z
  int kind;           // OPS_ARG_*
  int access;         // OPS_READ ...
  int npts;           // stencil points (DAT)
  int slot;           // SCALAR: scalar slot; RED: index among this loop's reductions
  int alo[3], ahi[3]; // allocation box of the dat in grid coordinates [alo, ahi)
  int slo[3], shi[3]; // stencil extent (most negative / most positive offset)
  int32_t off[OPS_MAX_STENCIL_POINTS];  // linear element offsets of the stencil points
};

// One loop as the kernels see it (copied to shared memory per CTA).
struct DLoop {
  int nargs, nins, nreds;
  int rng[6];                          // declared range x0 x1 y0 y1 z0 z1
  int red_op[OPS_MAX_REDS_PER_LOOP];   // OPS_RED_* of each reduction
  int part_row;                        // first partial row of this loop's reductions
  int zmask;                           // registers read before written (start at +0.0)
  int pad_;                            // header = 16 ints: ins rows start 8-byte aligned
  int ins[OPS_MAX_INS][6];
  double K[OPS_MAX_CONSTS];
  DArg args[OPS_MAX_ARGS];
};

// Host side: registers of a filled DLoop that an instruction reads before any
// instruction writes them; only those are zeroed per point.
inline void finish_dloop(DLoop& L) {
  int written = 0, zmask = 0;
  auto rd = [&](int r) {
    if (!((written >> r) & 1)) zmask |= 1 << r;
  };
  for (int pc = 0; pc < L.nins; ++pc) {
    const int* I = L.ins[pc];
    const int op = I[0], d = I[1], a = I[2], b = I[3], c = I[4], e = I[5];
    switch (op) {
      case OPS_IR_ADD: case OPS_IR_SUB: case OPS_IR_MUL: case OPS_IR_DIV: case OPS_IR_MIN: case OPS_IR_MAX:
        rd(a); rd(b); break;
      case OPS_IR_FMA: rd(a); rd(b); rd(c); break;
      case OPS_IR_SGT: rd(a); rd(b); rd(c); rd(e); break;
      case OPS_IR_WACC: rd(d); break;
      case OPS_IR_POLY: rd(a); break;
      case OPS_IR_ST: case OPS_IR_RED: rd(a); break;
      default: break;
    }
    if (op != OPS_IR_ST && op != OPS_IR_RED) written |= 1 << d;
  }
  L.zmask = zmask;
}

static_assert(offsetof(DLoop, ins) % 16 == 0, "instruction rows are read as int2");
static_assert(sizeof(DLoop) % 16 == 0, "DLoop is staged with 16-byte copies");

// A (tile, loop) piece of a skewed segment, in execution order.
struct Phase {
  int loop;      // index into the segment's DLoop table
  int barrier;   // 1: grid barrier before this phase
  int box[6];    // x0 x1 y0 y1 z0 z1 (non-empty)
};

// A reduction partial row: which scalar slot it folds into, with which operator.
struct FoldRow {
  int slot;
  int op;
};

// Double-double accumulator for deterministic, compensated sums.
struct DD {
  double hi, lo;
};

struct LaunchEnv {
  cudaStream_t stream;
  int num_sms;
  double* scal;         // reduction / scalar slots
  DD* part;             // reduction partials: rows x part_stride
  int part_stride;      // >= grid size of any chain kernel
  const FoldRow* rows;  // per partial row: target slot and operator
  int* err;             // device error word
  unsigned* bar;        // grid barrier state (2 words)
  int check;
  long long timeout_ns;
  int skip_block;       // test hook: CTA that never arrives at grid barriers (-1 = none)
};

// Context services for the other translation units (runtime.cpp).
cudaStream_t ctx_stream(ops_ctx c);
int ctx_num_sms(ops_ctx c);
bool ctx_host_only(ops_ctx c);
int ctx_alloc(ops_ctx c, void** p, size_t bytes);  // OPS_OK or OPS_ERR_NOMEM (budget-checked)
void ctx_free(ops_ctx c, void* p, size_t bytes);
int ctx_fail(ops_ctx c, int code, const char* msg);

// Overlapped tiles (Sec. 4.D applied per CTA): one dat of a segment as the
// overlapped kernel sees it.  Footprints are copied from src (the dat's
// current buffer) into shared memory at smem_off (doubles) with strides
// spitch / splane; the owned part of a written dat goes to dst (the dat's
// other buffer), which becomes current after the kernel.
struct OvDat {
  const double* src;   // grid point (0,0,0) of the current buffer
  double* dst;         // grid point (0,0,0) of the other buffer (written dats)
  int64_t gpitch, gplane;
  int written;
  int smem_off;
  int spitch, splane;
};

// Launch helpers implemented in chain_kernels.cu.
// chain_kernels_setup: once per device (opts the kernels into their shared memory).
cudaError_t chain_kernels_setup();
// bytes of shared memory the overlapped kernel may use for footprints
int overlap_smem_area_bytes();
int overlap_max_grid(int num_sms, int area_bytes);
// loops: the segment's descriptors with DAT args in shared-memory layout
// (pitch/plane/off for the footprint strides, slot = segment dat index);
// own: 6 ints per tile; boxes: 6 ints per (tile, loop); foot: 6 ints per (tile, dat)
cudaError_t launch_overlap(const LaunchEnv& env, const DLoop* d_loops, int nloops, const OvDat* d_dats, int ndats,
                           const int* d_own, const int* d_boxes, const int* d_foot, int ntiles, int grid,
                           int area_bytes);
int untiled_grid(const LaunchEnv& env, const int* box);
cudaError_t launch_untiled(const LaunchEnv& env, const DLoop* d_loop, const int* box, int grid);
cudaError_t launch_part_init(const LaunchEnv& env, int row0, int nrows);
cudaError_t launch_fold(const LaunchEnv& env, int row0, int nrows, int grid_used);
// the same for partials held elsewhere: row r of the fold at part + (r - row0) * stride, nused columns
cudaError_t launch_fold_rows(const LaunchEnv& env, const DD* part, int stride, int row0, int nrows, int nused);
// One instance of a batched fold: its partials (row r at part + (r - row0) * stride, nused columns),
// fold rows and scalar slots.
struct FoldInst {
  const DD* part;
  const FoldRow* rows;
  double* scal;
  int stride, nused;
};
// rows row0 .. row0 + nrows of every instance of d_fi[0 .. ninst) in one launch; row r of an
// instance's partials at part + (r - rbase) * stride; nused > 0 overrides the instances' nused
cudaError_t launch_fold_batch(cudaStream_t stream, const FoldInst* d_fi, int ninst, int row0, int nrows, int rbase,
                              int nused);
// One instance of a batched per-loop launch: its segment's descriptors, scalar slots and partials.
struct BatchInst {
  const DLoop* loops;
  const double* scal;
  DD* part;
};
int skewed_max_grid(int num_sms, int blocks_per_sm);
cudaError_t launch_skewed(const LaunchEnv& env, const DLoop* d_loops, const Phase* d_phases, int nphases,
                          int grid);
cudaError_t launch_set_scalar(const LaunchEnv& env, int slot, double value);

}  // namespace opstile
