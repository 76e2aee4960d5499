// Compiled loop bodies: the IR of every loop of a segment is turned into
// straight-line CUDA C (IR registers become machine registers, stencil
// offsets become immediates) and compiled for sm_103a at run time with
// NVRTC, once per distinct segment.  OPS generates per-loop code ahead of
// time from the application source (Sec. 3); here the loop bodies arrive as
// IR at run time, so the code is generated at the first flush instead.
// Internal to the library.
#pragma once

#include <string>
#include <vector>

#include "internal.h"

namespace opstile {

struct JitSegment;

// Kernels for the segment whose descriptors are loops[0..count) (as filled
// for this flush; only the fields that shape the code are used) and whose
// dat arguments are read-only in the whole segment where ro[l][a] != 0;
// es = 4 generates FP32 dats and arithmetic, 8 FP64.
// On success *out is a module shared by every context of the process with
// the same device and code.  Returns OPS_OK with *out == nullptr, and the
// reason in *why, when run-time compilation is unavailable.
// batch = true compiles the batch kernels ub<i> instead (jit_launch_batch).
int jit_segment(int device, const DLoop* loops, int count, const std::vector<std::vector<char>>& ro, int es,
                JitSegment** out, std::string* why, double* compile_ms, bool batch = false);

// Host only: the generated source of the segment, compiled for sm_103a
// without loading it (no device needed).  OPS_ERR_CUDA with the compiler's
// log in *why when it does not compile; OPS_ERR_NO_DEVICE without NVRTC.
int jit_compile_only(const DLoop* loops, int count, const std::vector<std::vector<char>>& ro, int es,
                     std::string* src, std::string* why, double* compile_ms);

// 1 (OPSTILE_PDL, default) launches the per-loop kernels with programmatic
// stream serialisation: a kernel's CTAs may become resident while its
// predecessor in the stream drains, and wait on the device
// (griddepcontrol.wait) until the predecessor has completed.
int jit_pdl();
// true when NVRTC and the driver's module calls can be reached
bool jit_available();
// CTAs of kernel u<i> resident per SM (queried once per kernel).
int jit_resident(JitSegment* s, int i);
// Grid policy of the compiled per-loop kernels (OPSTILE_JIT_GRID): 0 (the
// default) = one wave of the kernel's resident CTAs striding over the units,
// with the stride kept coprime to the row's x-chunk count so that no CTA
// always draws the same (possibly short) chunk; k > 0 = up to k CTAs per SM,
// more than stay resident, balanced by the block scheduler instead.
int jit_grid_policy();

// One launch of loop i of the segment over box (grid-stride units, the
// interpreter's enumeration); reductions assign (assign = 1) or combine
// into the CTA's partial column.
cudaError_t jit_launch(const JitSegment* s, int i, const LaunchEnv& env, const DLoop* d_loop, const int* box,
                       int grid, int assign);
// One launch of loop i of a batch segment (jit_segment with batch = true)
// for ninst instances: grid CTAs per instance (blockIdx.y = instance) over
// the box; instance k reads its descriptors at d_inst[k].loops + i, its
// scalars at d_inst[k].scal, and assigns its reductions' partials at
// d_inst[k].part + row * stride + CTA.
cudaError_t jit_launch_batch(const JitSegment* s, int i, cudaStream_t stream, const BatchInst* d_inst, int ninst,
                             const int* box, int grid, int stride);

// Overlapped tiles (Sec. 4.D per CTA): one kernel per run of loops, with
// the run's shared-memory layout compiled in.  loops: the run's descriptors
// in shared-memory layout (DAT args: pitch / plane / off in footprint
// strides, slot = the run's dat index).
struct OvLayout {
  int es = 8;  // bytes per element (8: FP64, 4: FP32); offsets and strides count elements
  int ndats = 0;
  std::vector<int> smem_off, spitch, splane, written;  // per dat of the run
};
struct JitOverlap;
// Kernels for several runs at once: those not compiled yet compile in
// parallel.  (*out)[i] = nullptr for all when compilation is unavailable.
struct OvRequest {
  const DLoop* loops;
  int count;
  OvLayout lay;
};
int jit_overlap_many(int device, const std::vector<OvRequest>& reqs, std::vector<JitOverlap*>* out, std::string* why,
                     double* compile_ms);
// Host only: generate and compile (no load, no device) an overlapped kernel.
int jit_compile_overlap_only(const DLoop* loops, int count, const OvLayout& lay, std::string* src, std::string* why,
                             double* compile_ms);
// CTAs that fit the device at once with area_bytes of dynamic shared memory (0: it does not fit)
int jit_overlap_max_grid(JitOverlap* o, int num_sms, int area_bytes);
cudaError_t jit_launch_overlap(const JitOverlap* o, const LaunchEnv& env, const DLoop* d_loops, const OvDat* d_dats,
                               const int* d_own, const int* d_boxes, const int* d_foot, int ntiles, int grid,
                               int area_bytes);

// Wavefront execution of a skewed plan (Sec. 4.B tiles; the wavefront
// scheduling the paper leaves to future work): one persistent kernel with
// every loop body of the segment, taking (phase, chunk) work units in plan
// order and waiting on per-phase completion counters.
struct WfPhase {
  int loop, nchunk, ustart, dep0, ndep, pad;
  int box[6];
};
struct JitWave;
// P of the compiled enumeration (rows per unit) for elements of es bytes;
// enumeration units per wavefront work unit (OPSTILE_WF_UNITS, default 16)
int jit_rows_per_unit(int es);
int jit_wave_units_per_chunk();
// threads per CTA of the wavefront kernel (OPSTILE_WF_THREADS, default 128)
int jit_wave_threads();
// CTAs per SM the wavefront kernel's registers are sized for (OPSTILE_WF_MINB,
// default: the per-loop kernels' thread count per SM)
int jit_wave_min_ctas();
// slope of the wavefront's ticket order (OPSTILE_WF_SLOPE, default 1; see build_wavefront)
int jit_wave_slope();
int jit_wavefront(int device, const DLoop* loops, int count, const std::vector<std::vector<char>>& ro, int es,
                  JitWave** out, std::string* why, double* compile_ms);
// Host only: generate and compile (no load, no device) the wavefront kernel.
int jit_compile_wavefront_only(const DLoop* loops, int count, const std::vector<std::vector<char>>& ro, int es,
                               std::string* src, std::string* why, double* compile_ms);
// CTAs of the wavefront kernel resident on the device at once
int jit_wavefront_max_grid(JitWave* w, int num_sms);
// d_done: one counter per phase, zero before the launch; d_ticket: zero.
// env.skip_block >= 0 (test hook): that work unit's completion is never
// counted, so the phases waiting on it give up after env.timeout_ns.
cudaError_t jit_launch_wavefront(const JitWave* w, const LaunchEnv& env, const DLoop* d_loops,
                                 const WfPhase* d_phases, const int* d_deps, const int* d_uphase, int nunits,
                                 int* d_done, int* d_ticket, int grid);

// Persistent skewed execution (Algorithm 2 in one cooperative launch of
// compiled bodies, ops_config.skewed_persistent = 1): the plan's phases in
// order, a grid barrier before each phase whose `barrier` flag is set.
struct JitSkew;
int jit_skewed(int device, const DLoop* loops, int count, const std::vector<std::vector<char>>& ro, int es,
               JitSkew** out, std::string* why, double* compile_ms);
int jit_compile_skewed_only(const DLoop* loops, int count, const std::vector<std::vector<char>>& ro, int es,
                            std::string* src, std::string* why, double* compile_ms);
// CTAs co-resident on the device (the cooperative grid's limit)
int jit_skewed_max_grid(JitSkew* k, int num_sms);
// env.bar (2 words) is reset on the stream first; reductions combine into
// env.part's columns (the caller initialises and folds them).
cudaError_t jit_launch_skewed(const JitSkew* k, const LaunchEnv& env, const DLoop* d_loops, const Phase* d_phases,
                              int nphases, int grid);

// Tile wavefront (OPS_MODE_TILEWAVE, see build_tile_wave): one persistent
// kernel with every loop body of the segment; each CTA runs all the loops of
// one tile at a time.  Its arguments travel by value in one struct.
struct TwArgs {
  const DLoop* loops;        // the segment's descriptors
  const int* rng;            // per dimension d at roff[d]: (start, end) of tile t, loop l at 2 (t L + l)
  const int* order;          // ticket -> linear tile index (x fastest)
  const int* cls;            // per dimension d at coff[d]: class of each tile index
  const unsigned short* need;  // per class: ndirs x L loop counts of the predecessor tiles
  int* prog;                 // per tile: loops completed (zero before the launch)
  int* ticket;               // zero before the launch
  const double* scal;
  DD* part;                  // reduction partials: (row - row0) * stride + tile
  int* err;
  long long timeout_ns;
  int nt[3], ncls[3], roff[3], coff[3];
  int ntiles, stride, row0, skip_tile;  // skip_tile >= 0 (test hook): that tile never reports progress
  const unsigned char* pf;   // per loop: arguments whose rows are prefetched into L2 `ahead` loops early
  int ahead, ngroups;
  const int* groups;         // the loops of step g: groups[g] .. groups[g + 1]
};
struct JitTile;
// compute threads per CTA (OPSTILE_TW_THREADS: whole warps, 128..992, default 256), CTAs per
// SM the registers are sized for (OPSTILE_TW_MINB, default 2) and rows a
// thread evaluates at a time (OPSTILE_TW_PTS32 / OPSTILE_TW_PTS; default 8 in
// FP32, 4 in FP64: the fastest measured on GB300)
int jit_tile_threads();
int jit_tile_min_ctas();
int jit_tile_pts(int es);
// L2 prefetch of the tile wavefront (OPSTILE_TW_PREFETCH): 0 (the default:
// measured no faster on GB300) none, 1 the rows a loop reads from dats no
// earlier loop of the segment touched (first reads of the segment's
// inputs), 2 every row a loop reads; issued OPSTILE_TW_AHEAD (default 3)
// loops ahead
int jit_tile_prefetch();
int jit_tile_ahead();
// loops of one tile step at most (OPSTILE_TW_GROUP, 1..8, default 8)
int jit_tile_group();
// tiles along x per strip of the ticket order (OPSTILE_TW_BAND; 0 = one strip)
int jit_tile_band();
// batch = true compiles the batch kernel "twb" instead of "tw": one launch
// runs the segment for several instances of the same code (see
// jit_launch_tilewave_batch).
int jit_tilewave(int device, const DLoop* loops, int count, const std::vector<std::vector<char>>& ro, int es, int ndim,
                 JitTile** out, std::string* why, double* compile_ms, bool batch = false);
int jit_compile_tilewave_only(const DLoop* loops, int count, const std::vector<std::vector<char>>& ro, int es,
                              int ndim, std::string* src, std::string* why, double* compile_ms, bool batch = false);
// The tile-per-warp form (OPS_MODE_TILEWARP): the same plan and arguments,
// each warp a worker running whole tiles; OPSTILE_TWW_WARPS warps per CTA
// (default 4), registers sized for OPSTILE_TWW_MINB CTAs per SM (default 4).
int jit_tilewarp_warps();
int jit_tilewarp_min_ctas();
int jit_tilewarp(int device, const DLoop* loops, int count, const std::vector<std::vector<char>>& ro, int es, int ndim,
                 JitTile** out, std::string* why, double* compile_ms);
int jit_compile_tilewarp_only(const DLoop* loops, int count, const std::vector<std::vector<char>>& ro, int es,
                              int ndim, std::string* src, std::string* why, double* compile_ms);
// CTAs of the kernel (either form) resident on the device at once
int jit_tilewave_max_grid(JitTile* t, int num_sms);
cudaError_t jit_launch_tilewave(const JitTile* t, const TwArgs& args, cudaStream_t stream, int grid);
// The batch kernel: d_args[i] are instance i's arguments (every instance's
// ticket and err pointing at the same words; prog arrays disjoint);
// d_tmap[2 k], d_tmap[2 k + 1] = instance and linear tile index of ticket k
// (each instance's tiles in its plan's order); d_ticket zero before the launch.
cudaError_t jit_launch_tilewave_batch(const JitTile* t, const TwArgs* d_args, const int* d_tmap, int total,
                                      int* d_ticket, cudaStream_t stream, int grid);

}  // namespace opstile
