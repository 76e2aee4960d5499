/*
 * opstile: run-time loop-chain tiling of OPS-style stencil loops on one
 * GB300 (sm_103a).  C ABI.
 *
 * The method is the paper's (Reguly, Mudalige, Giles, "Loop Tiling in
 * Large-Scale Stencil Codes at Run-time with OPS"):
 *   - Sec. 3: blocks, datasets (dats) with halos, stencils, and parallel
 *     loops whose result must not depend on the order of their points;
 *   - Sec. 4.A: ops_par_loop only queues the loop; the queue is executed when
 *     the host needs data back (a reduction result, a fetch) or calls
 *     ops_execute;
 *   - Sec. 4.B, Algorithm 1: at flush time a dependency analysis walks the
 *     queued loops backwards and gives every tile of every loop its own
 *     (skewed) range; Algorithm 2 then runs tile by tile, loop by loop;
 *   - Sec. 4.D: overlapped tiles that recompute what crosses a tile
 *     boundary, so tiles become independent;
 *   - Sec. 4.C: tile-size selection from the bytes per grid point and the
 *     last-level cache size.
 * Loop bodies are not function pointers: they are short programs in a fixed
 * register IR (weighted stencil sums, polynomials, min/max/select,
 * reductions) that the library compiles to sm_103a kernels at the first
 * flush of each segment (NVRTC), or runs through interpreter kernels.
 *
 * Conventions for every function below:
 *   - returns OPS_OK (0) or a negative OPS_ERR_* code; on error
 *     ops_last_error(ctx) describes it (string owned by ctx, valid until the
 *     next call on ctx);
 *   - handles are small non-negative ints inside one context;
 *   - pointers named host_* are host memory, dev_* device memory; the
 *     library copies what it needs before returning unless stated;
 *   - a context is not thread-safe: use one per host thread;
 *   - no call aborts the process; a CUDA failure is returned as
 *     OPS_ERR_CUDA with the CUDA error string.
 */
#ifndef OPSTILE_H
#define OPSTILE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define OPS_OK 0
#define OPS_ERR_INVALID_ARG -1   /* bad argument, handle or IR */
#define OPS_ERR_BOUNDS -2        /* a loop would access outside [-d_m, size + d_p) */
#define OPS_ERR_DEVICE_BOUNDS -3 /* a kernel in checked mode caught an out-of-range access */
#define OPS_ERR_NOMEM -4         /* device allocation failed or over the HBM budget */
#define OPS_ERR_TIMEOUT -5       /* a device-side wait ran past its limit */
#define OPS_ERR_NOT_CONVERGED -6 /* a solve hit its iteration cap */
#define OPS_ERR_CUDA -7          /* a CUDA call failed */
#define OPS_ERR_STATE -8         /* call not allowed in the current state */
#define OPS_ERR_NO_DEVICE -9     /* no usable sm_103a device */

/* ---- execution modes of a flushed chain ---- */
#define OPS_MODE_UNTILED 0    /* one kernel per loop over its full range (the comparator) */
#define OPS_MODE_SKEWED 1     /* Algorithm 1 tiles run tile by tile (Algorithm 2); see
                                 ops_config.skewed_persistent for the two compiled forms */
#define OPS_MODE_OVERLAPPED 2 /* independent shared-memory tiles with halo recomputation (Sec. 4.D) */
/* OPS_MODE_OVERLAPPED applies to a segment whose dats are all library-owned
 * with one common size and halo, and whose tile footprints fit one CTA's
 * shared memory after the tile is shrunk; other segments run skewed.  It
 * writes every written dat into a second buffer of the same shape, which then
 * becomes the dat's storage: ops_dat_info returns the new address. */
#define OPS_MODE_AUTO 3       /* library picks per segment */
#define OPS_MODE_WAVEFRONT 4  /* Algorithm 1 tiles run as a dependence-driven wavefront (Sec. 4.B leaves
                                 wavefront scheduling of the tiles to future work) */
/* OPS_MODE_WAVEFRONT cuts the outermost dimension into thin tiles (tile[ndim-1]
 * points; 0 = about 262144 points per tile) and leaves the other dimensions
 * whole unless tile[] sets them.  Algorithm 1 gives every (tile, loop) phase
 * its range; each phase then depends only on the earlier phases it conflicts
 * with (a shared dat that one of the two writes, in intersecting regions,
 * reads widened by their stencils).  One persistent kernel holding every loop
 * body of the segment (compiled at run time, so this mode needs NVRTC) hands
 * out chunks of phases in order of their dependency level, and each chunk
 * waits only on its phase's dependencies -- no grid-wide barrier.  A segment
 * of one loop runs untiled; with check = 1 or interpret = 1, or without
 * NVRTC, the segment runs in OPS_MODE_SKEWED.  Results are identical to every
 * other mode.  OPS_MODE_AUTO does not try this mode. */

#define OPS_MODE_TILEWAVE 5  /* Algorithm 1 tiles cut in every dimension, each run whole by one CTA (the
                                 inner loop of Algorithm 2), tiles concurrent as a wavefront */
/* OPS_MODE_TILEWAVE cuts every dimension into tiles (tile[d] points; 0 =
 * automatic: about 4096 points per tile, x the widest) and gives every
 * (tile, loop) its Algorithm 1 range.  One persistent kernel holding every
 * loop body of the segment (compiled at run time, so this mode needs NVRTC)
 * hands whole tiles to CTAs in order of the sum of their tile coordinates;
 * a CTA runs the tile's loops in order, and before loop l waits only until
 * the tiles one step back in any subset of the dimensions have completed
 * the loops l conflicts with.  A tile's intermediate values are re-read
 * from the SM's L1 and from L2 while the CTA works through its loops.
 * Tiles smaller than the chain's skew (a conflict two tiles back) are grown
 * until they are not; a segment of one loop runs untiled; with check = 1 or
 * interpret = 1, or without NVRTC, the segment runs in OPS_MODE_SKEWED.
 * Results are identical to every other mode. */
#define OPS_MODE_TILEWARP 6  /* the tile wavefront's plan with a tile per warp instead of per CTA */
/* OPS_MODE_TILEWARP runs OPS_MODE_TILEWAVE's plan (automatic tiles smaller:
 * 64 x 32 in FP32, 32 x 32 in FP64, 32 x 8 x 8 in 3D) with every warp a worker
 * of its own: a warp runs a tile's loops with only warp-level ordering
 * between them and waits on the predecessor tiles' progress counters alone,
 * so the warps of an SM never wait for one another at a CTA barrier.
 * Fallbacks and results as OPS_MODE_TILEWAVE. */

/* ---- argument kinds, access modes, reduction operators ---- */
#define OPS_ARG_DAT 0    /* a dat accessed through a stencil */
#define OPS_ARG_SCALAR 1 /* read the current value of a reduction or scalar handle */
#define OPS_ARG_RED 2    /* contribute to a reduction handle */
#define OPS_READ 0
#define OPS_WRITE 1
#define OPS_RW 2
#define OPS_INC 3
#define OPS_RED_SUM 0
#define OPS_RED_MIN 1
#define OPS_RED_MAX 2

/* ---- loop-body IR opcodes: one instruction = 6 int32 (op, d, a, b, c, e) ----
 * Eight FP64 registers r0..r7 per grid point start at +0.0; K is the loop's
 * constant pool; v(a, p) is the dat of argument a at this point shifted by
 * point p of that argument's stencil.  Arithmetic is IEEE FP64 with round to
 * nearest; fma rounds once; nothing is reassociated or contracted. */
#define OPS_IR_LD 1    /* r[d] = v(a, b); a SCALAR argument gives its value (b = 0) */
#define OPS_IR_CST 2   /* r[d] = K[a] */
#define OPS_IR_ADD 3   /* r[d] = r[a] + r[b] */
#define OPS_IR_SUB 4   /* r[d] = r[a] - r[b] */
#define OPS_IR_MUL 5   /* r[d] = r[a] * r[b] */
#define OPS_IR_FMA 6   /* r[d] = fma(r[a], r[b], r[c]) */
#define OPS_IR_DIV 7   /* r[d] = r[a] / r[b] */
#define OPS_IR_MIN 8   /* r[d] = r[b] < r[a] ? r[b] : r[a] */
#define OPS_IR_MAX 9   /* r[d] = r[b] > r[a] ? r[b] : r[a] */
#define OPS_IR_SGT 10  /* r[d] = r[a] > r[b] ? r[c] : r[e] */
#define OPS_IR_WSUM 11 /* r[d] = K[b] v(a,0); r[d] = fma(K[b+p], v(a,p), r[d]) for p = 1..np-1 */
#define OPS_IR_WACC 12 /* r[d] = fma(K[b+p], v(a,p), r[d]) for p = 0..np-1 */
#define OPS_IR_POLY 13 /* t = K[b+c]; t = fma(t, r[a], K[b+i]) for i = c-1..0; r[d] = t */
#define OPS_IR_ST 14   /* arg d WRITE/RW: dat = r[a]; arg d INC: dat = dat + r[a] */
#define OPS_IR_RED 15  /* reduction arg d takes the contribution r[a] */

/* limits of one loop */
#define OPS_MAX_ARGS 8
#define OPS_MAX_STENCIL_POINTS 32
#define OPS_MAX_INS 64
#define OPS_MAX_CONSTS 128
#define OPS_MAX_REDS_PER_LOOP 4

typedef struct ops_ctx_s* ops_ctx;

/* device = OPS_DEVICE_NONE makes a host-only context: declarations,
 * validation and planning work, anything that would run loops returns
 * OPS_ERR_NO_DEVICE.  No CUDA call is made. */
#define OPS_DEVICE_NONE -1

typedef struct {
  int device;          /* CUDA device ordinal */
  void* stream;        /* cudaStream_t all work is ordered on; NULL: the library creates one */
  int mode;            /* OPS_MODE_* */
  int tile[3];         /* skewed / overlapped tile size per dimension; 0 = automatic */
  int segment;         /* at most this many loops per tiled segment; 0 = up to the flush */
  int check;           /* 1: kernels bounds-check every access (OPS_ERR_DEVICE_BOUNDS) */
  int64_t l2_bytes;    /* cache budget for automatic tile sizes (Sec. 4.C); 0 = 3/4 of L2 */
  int64_t hbm_budget;  /* cap on bytes the library allocates; 0 = no cap */
  int timeout_ms;      /* limit of every device-side wait (grid barriers); 0 = 2000 */
  int blocks_per_sm;   /* persistent-kernel CTAs per SM; 0 = as many as fit */
  int test_skip_barrier_block; /* test hook: this CTA never arrives at grid barriers (skewed), this
                                  work unit's completion is never counted (wavefront); -1 = off */
  int timing;          /* 1: record CUDA events around the chain kernels (kernel_ms in ops_flush_stats) */
  int interpret;       /* 1: run loop bodies through the register-IR interpreter kernels instead of
                          kernels compiled from the IR at the first flush of each segment (NVRTC) */
  int real;            /* OPS_REAL_F64 (default) or OPS_REAL_F32: the element type of every dat of
                          the context and the precision of every loop's arithmetic.  FP32 loops
                          run compiled bodies only (no checked or interpreted mode); constants
                          and scalar arguments are rounded to float on load; reductions take the
                          float values exactly and accumulate as in FP64 */
  int skewed_persistent; /* OPS_MODE_SKEWED with compiled bodies: 1 runs a segment's phases in
                            one cooperative launch of a kernel holding every body, with grid
                            barriers only before the phases the plan marks; 0 (default, measured
                            faster on GB300) launches each phase's loop kernel in plan order */
} ops_config;
#define OPS_REAL_F64 0
#define OPS_REAL_F32 1

/* Fill *cfg with defaults (device 0, own stream, OPS_MODE_AUTO, automatic tiles). */
void ops_config_default(ops_config* cfg);

/* Create a context on cfg->device.  *out receives the context.  Fails with
 * OPS_ERR_NO_DEVICE if the device is not compute capability 10.3. */
int ops_init(ops_ctx* out, const ops_config* cfg);
/* Flush nothing; free every library-owned buffer and the context. */
int ops_finalize(ops_ctx ctx);
const char* ops_last_error(ops_ctx ctx);
/* Turn the per-kernel timing events (ops_config.timing) on or off for later flushes. */
int ops_set_timing(ops_ctx ctx, int timing);
/* Change mode / tile / segment for later flushes (tile may be NULL). */
int ops_set_mode(ops_ctx ctx, int mode, const int* tile, int segment);

/* ---- declarations (Sec. 3) ---- */
/* A structured block of 1, 2 or 3 dimensions. */
int ops_decl_block(ops_ctx ctx, int dims, const char* name, int* out);
/* A dat (FP64, or FP32 in an OPS_REAL_F32 context) of size[0..dims) interior points with halo depths d_m (below)
 * and d_p (above) per dimension (unused dimensions: size 1, halos 0).
 * dev_ptr0 == NULL: the library allocates a zeroed, padded array (x rows
 * start 128-byte aligned) and owns it.  Otherwise dev_ptr0 is borrowed: it
 * must point at grid point (0,0,0) of caller-owned device memory in which
 * point (x,y,z) is dev_ptr0[x + pitch*y + plane*z] for every point of the
 * allocation box; it must outlive the dat. */
int ops_decl_dat(ops_ctx ctx, int block, const int size[3], const int d_m[3], const int d_p[3],
                 double* dev_ptr0, int64_t pitch, int64_t plane, const char* name, int* out);
/* A stencil of npts offsets (3 ints per point; unused dimensions 0). */
int ops_decl_stencil(ops_ctx ctx, int dims, int npts, const int* offsets, const char* name, int* out);
/* A reduction handle (OPS_RED_*), a device-resident FP64 value that starts at
 * the operator's identity, accumulates the contributions of every loop that
 * reduces into it, and is read (and reset) by ops_reduction_result. */
int ops_decl_reduction(ops_ctx ctx, int op, int* out);

/* A device-resident scalar (OPS's global constants; a CG coefficient):
 * SCALAR arguments read its value, which stays on the device.  It starts
 * at init; ops_scalar_set changes it after every loop queued before the
 * call (those read the old value), ops_scalar_get flushes and reads it.
 * Scalars and reductions share one handle space; a scalar cannot be the
 * target of a RED argument, nor be read by ops_reduction_result. */
int ops_decl_scalar(ops_ctx ctx, double init, int* out);
int ops_scalar_set(ops_ctx ctx, int scalar, double value);
int ops_scalar_get(ops_ctx ctx, int scalar, double* host_out);

/* ---- parallel loops (Sec. 3, Sec. 4.A) ---- */
typedef struct {
  int kind;    /* OPS_ARG_DAT / OPS_ARG_SCALAR / OPS_ARG_RED */
  int handle;  /* dat or reduction handle */
  int stencil; /* stencil handle (DAT); ignored otherwise */
  int access;  /* OPS_READ / OPS_WRITE / OPS_RW / OPS_INC (DAT) */
} ops_arg;

/* Queue a loop over range[2*d .. 2*d+1) (half-open, per dimension) of
 * `block`.  The body is `nins` instructions (code: 6 int32 each) with
 * `nconsts` constants; both are copied.  Checked here: handles, IR
 * well-formedness, a dat appears at most once, written args use a stencil
 * whose only point is the origin, every access stays inside
 * [-d_m, size + d_p) (else OPS_ERR_BOUNDS).  Nothing runs. */
int ops_par_loop(ops_ctx ctx, int block, int dims, const int* range, int nargs, const ops_arg* args,
                 int nins, const int32_t* code, int nconsts, const double* consts, const char* name);
/* Run every queued loop (Sec. 4.A flush).  Returns after the work is
 * queued on the stream; device errors surface at the next ops_sync. */
int ops_execute(ops_ctx ctx);
/* Batched flush of several grids' chains (not in the paper, whose chains run
 * one grid per process; the chain and its tiling are those of Sec. 4):
 * ctxs[0 .. count) each hold a queued chain that matches the first
 * context's loop for loop in everything but the dats' addresses and the
 * loops' constants -- the same loop bodies, ranges, stencils, reductions,
 * scalars and dat shapes, declared in the same order (typically the same
 * program run on count grids of one size).  Each segment of the chains
 * runs for every context at once, in ctxs[0]'s mode and tile:
 * OPS_MODE_UNTILED as one launch per loop for all contexts (one CTA row per
 * context); OPS_MODE_TILEWAVE as one launch of the tile wavefront whose
 * tickets interleave every context's tiles (one plan for all; progress
 * counters, reductions and scalars per context); OPS_MODE_AUTO as the batch
 * autotuner picks among those two (the wavefront at its automatic tiles,
 * with the whole grid as one tile, and with half-height tiles), timed per
 * segment signature and batch size; any other mode runs each context's
 * segment on its own.  Every dat and reduction ends exactly as if each
 * context had called ops_execute alone.  The work goes on ctxs[0]'s stream;
 * every other context's stream waits for it, so later calls on any of the
 * contexts follow the batch.  Device-side errors of a batched launch
 * (OPS_ERR_TIMEOUT) surface at ops_sync of ctxs[0].  Errors:
 * OPS_ERR_INVALID_ARG (NULL, count < 1, a context twice, another device or
 * precision, or chains that differ; nothing runs and every queue is kept),
 * any error of ops_execute.  ops_last_stats of each context reports
 * batched = count for segments that ran in one launch. */
int ops_execute_batch(ops_ctx* ctxs, int count);
/* Drop every queued loop without running it. */
int ops_queue_clear(ops_ctx ctx);
/* Flush, wait, copy the reduction's value to *host_out and reset it. */
int ops_reduction_result(ops_ctx ctx, int red, double* host_out);
/* Flush, wait and check the device error word (OPS_ERR_TIMEOUT,
 * OPS_ERR_DEVICE_BOUNDS). */
int ops_sync(ops_ctx ctx);

/* ---- data movement ---- */
/* Flush, then copy the dat's whole allocation box (halos included) into the
 * dense host array host_out of ex*ey*ez elements of the context's type
 * (doubles, or floats with OPS_REAL_F32), x fastest. */
int ops_dat_fetch(ops_ctx ctx, int dat, void* host_out, int64_t nelems);
/* Copy a dense host array of the allocation box into the dat (after the
 * queued loops, in stream order). */
int ops_dat_upload(ops_ctx ctx, int dat, const void* host_in, int64_t nelems);
/* As ops_dat_fetch / ops_dat_upload, but the copy is only queued on the
 * context's stream (after the flushed loops): the host array must stay
 * valid, and unchanged for an upload, until ops_sync (or another waiting
 * call) returns; fetched values are there from then on.  With pinned host
 * memory the copy runs while the host continues. */
int ops_dat_fetch_async(ops_ctx ctx, int dat, void* host_out, int64_t nelems);
int ops_dat_upload_async(ops_ctx ctx, int dat, const void* host_in, int64_t nelems);
/* Current device address of grid point (0,0,0) and strides of a dat; ext
 * receives the allocation extents (may be NULL). */
int ops_dat_info(ops_ctx ctx, int dat, double** dev_ptr0, int64_t* pitch, int64_t* plane, int* ext);

/* ---- statistics of the most recent flush ---- */
typedef struct {
  double plan_ms;        /* host time spent building plans (0 on a cache hit) */
  int segments;          /* tiled segments executed */
  int loops;             /* loops executed */
  int tiles;             /* tiles in the last skewed / overlapped segment */
  int phases;            /* non-empty (tile, loop) pieces executed */
  int barriers;          /* grid barriers executed by persistent kernels; OPS_MODE_TILEWAVE: the
                            CTA-wide steps (groups of loops) over all tiles */
  int launches;          /* kernel launches issued by the flush */
  int plan_cache_hits;   /* segments whose plan came from the cache */
  int mode;              /* OPS_MODE_* of the last segment */
  int tile[3];           /* tile size of the last tiled segment */
  int64_t redundant_points; /* overlapped mode: extra points computed */
  int64_t points;        /* loop points executed (excluding redundancy) */
  int skew[3];           /* largest spread of the loops' tile ends over all but the last tile */
  double kernel_ms;      /* timing=1: device time of the flush's chain kernels (persistent kernel,
                            or the per-loop kernels), measured with CUDA events on the context's stream */
  int kernel_launches;   /* chain kernels covered by kernel_ms */
  int tuning;            /* OPS_MODE_AUTO: 1 while the autotuner is still timing candidates */
  int compiled;          /* 1: the last untiled / skewed segment ran compiled loop bodies */
  double compile_ms;     /* host time spent generating and compiling loop bodies in this flush */
  int batched;           /* ops_execute_batch: contexts whose segments ran in the same launch as
                            this one's (0: not batched) */
} ops_flush_stats;
/* Statistics of the most recent flush; with timing=1 this waits for that
 * flush's kernels to finish. */
int ops_last_stats(ops_ctx ctx, ops_flush_stats* out);

/* ---- plan inspection (host only; no device work) ----
 * Build the skewed plan (Algorithm 1) for the currently queued loops with the
 * given tile sizes, without executing them.  out_ranges receives, for every
 * dimension d < dims, tile t and loop l, the pair (start, end) at
 * out_ranges[2 * (offset_d + t * nloops + l)], offset_d = nloops * sum of
 * ntiles of the dimensions before d; out_ntiles[d] receives the tile counts.
 * cap is the number of ints out_ranges can hold. */
int ops_plan_skewed(ops_ctx ctx, const int* tile, int* out_ntiles, int* out_ranges, int64_t cap);
/* Build the overlapped-tile geometry (Sec. 4.D) of one tile for the currently
 * queued loops, without executing them.  owned = x0 x1 y0 y1 z0 z1 of the
 * tile (half-open).  out_boxes receives 6 ints per queued loop: the box that
 * loop computes inside the tile (all zero when empty); out_foot receives 6
 * ints per declared dat: the box of its values the tile's loops read (lo >
 * hi in every dimension when no loop reads it).  Dimensions >= the loops'
 * dimensionality hold the loops' (0, 1). */
int ops_plan_overlapped(ops_ctx ctx, const int owned[6], int* out_boxes, int* out_foot);
/* Build the wavefront plan (OPS_MODE_WAVEFRONT) of the currently queued loops
 * for the given tile sizes, without executing them.  counts[0..3] receive the
 * number of (tile, loop) phases, of dependency entries, of work units and of
 * dependency levels.  With out_phases != NULL (phase_cap ints, >= 12 per
 * phase) phase q, in Algorithm 2 order, is described by
 *   out_phases[12 q ..] = loop, chunks, first work unit, first dependency
 *   entry, dependency count, level, box (x0 x1 y0 y1 z0 z1),
 * and with out_deps != NULL (dep_cap ints) the dependency entries are the
 * indices of earlier phases.  Call with NULL arrays to learn the sizes. */
int ops_plan_wavefront(ops_ctx ctx, const int* tile, int64_t* counts, int* out_phases, int64_t phase_cap,
                       int* out_deps, int64_t dep_cap);
/* Build the tile-wavefront plan (OPS_MODE_TILEWAVE) of the currently queued
 * loops for the given tile sizes (all >= 1), without executing them.
 * OPS_ERR_INVALID_ARG, with the reason in ops_last_error, when the tiles are
 * smaller than the chain's skew.  counts[0..4] receive the number of tiles,
 * of tile classes, of predecessor directions (2^dims - 1; direction k steps
 * back one tile in dimension d when bit d of k + 1 is set), of loops and of
 * steps (runs of consecutive loops a CTA runs without a barrier between
 * them).  Optional outputs (NULL to skip): out_need (classes x directions x
 * loops ints): the loops of each predecessor tile that must be complete
 * before a tile of that class runs each loop; out_class (tiles ints, x
 * fastest): the class of each tile; out_order (tiles ints): the tile of
 * each ticket; out_steps (loops + 1 ints): the first loop of each step,
 * then the number of loops. */
int ops_plan_tilewave(ops_ctx ctx, const int* tile, int64_t* counts, int* out_need, int64_t need_cap, int* out_class,
                      int* out_order, int64_t tile_cap, int* out_steps);
/* Generate the CUDA source of the compiled loop bodies for the currently
 * queued loops (as one segment) and compile it for sm_103a with NVRTC,
 * without loading it: no device is needed.  src_out (cap bytes, may be NULL)
 * receives the NUL-terminated source, truncated to fit; *src_len its full
 * length; *compile_ms the compile time.  OPS_ERR_CUDA with the compiler's
 * log in ops_last_error when it does not compile; OPS_ERR_NO_DEVICE when
 * NVRTC is not installed.  The queue is left as it was. */
int ops_compile_queued(ops_ctx ctx, char* src_out, int64_t cap, int64_t* src_len, double* compile_ms);
/* The same for the wavefront kernel of the queued loops (OPS_MODE_WAVEFRONT:
 * every loop body in one kernel). */
int ops_compile_queued_wavefront(ops_ctx ctx, char* src_out, int64_t cap, int64_t* src_len, double* compile_ms);

/* The same for the tile-wavefront kernel of the queued loops (OPS_MODE_TILEWAVE). */
int ops_compile_queued_tilewave(ops_ctx ctx, char* src_out, int64_t cap, int64_t* src_len, double* compile_ms);
/* The same for the tile-per-warp kernel of the queued loops (OPS_MODE_TILEWARP). */
int ops_compile_queued_tilewarp(ops_ctx ctx, char* src_out, int64_t cap, int64_t* src_len, double* compile_ms);
/* The same for the persistent skewed kernel of the queued loops (OPS_MODE_SKEWED
 * with compiled bodies: every loop body in one cooperative kernel). */
int ops_compile_queued_skewed(ops_ctx ctx, char* src_out, int64_t cap, int64_t* src_len, double* compile_ms);
/* The same for the batch form of the tile-wavefront kernel (ops_execute_batch). */
int ops_compile_queued_tilewave_batch(ops_ctx ctx, char* src_out, int64_t cap, int64_t* src_len,
                                      double* compile_ms);

/* ---- heat-conduction solves (TeaLeaf-shaped, Sec. 5 and Sec. 6.D) ----
 * Solve A x = b on an n x n cell grid for the implicit heat-conduction
 * operator (A u)_c = u_c + sum over the four faces f of c of
 * k_f (u_c - u_nb), k_f the harmonic mean 2 ka kb / (ka + kb) of the two
 * cells' conductivities; a boundary face takes the cell's own conductivity
 * and u = 0 outside the grid.  Arrays are n*n doubles, x fastest.
 * precision OPS_PREC_FP64: textbook CG in FP64 from x = 0 until
 *   |r|_2 <= tol |b|_2 for the recursively updated residual.
 * precision OPS_PREC_MIXED: iterative refinement; r = b - A x, its norm and
 *   x += |r| d in FP64; each correction d solves A d = r / |r| by CG with FP32
 *   vectors and operator, FP64-accumulated dot products and FP64 scalars, to
 *   relative residual inner_tol; stops when the true FP64 residual
 *   |b - A x| <= tol |b|.
 * Several grids of different sizes can be solved in one batch: they advance
 * together, one CG iteration per group of five kernel launches, and each
 * result is independent of the others in the batch. */
#define OPS_PREC_FP64 0
#define OPS_PREC_MIXED 1
typedef struct {
  double tol;        /* relative residual target */
  double inner_tol;  /* MIXED: relative residual of each inner FP32 solve (0: 1e-4) */
  int precision;     /* OPS_PREC_* */
  int maxit;         /* cap on CG iterations (inner iterations for MIXED) */
  int maxouter;      /* MIXED: cap on refinement corrections (0: 100) */
} ops_cg_params;
typedef struct {
  int iterations;    /* CG iterations (inner iterations in total for MIXED) */
  int outer;         /* refinement corrections applied (MIXED) */
  int converged;     /* 1 if the tolerance was reached */
  double relres;     /* final relative residual (FP64: recursive; MIXED: true FP64 residual) */
} ops_cg_stats;
/* Solve one system; host_x receives n*n doubles.  Returns OPS_OK, or
 * OPS_ERR_NOT_CONVERGED (x and stats still filled) if maxit was reached. */
int ops_cg_solve(ops_ctx ctx, int n, const double* host_kappa, const double* host_rhs, const ops_cg_params* params,
                 double* host_x, ops_cg_stats* stats);
/* w = A u for the operator above, once, through the solver's own device
 * code (precision OPS_PREC_MIXED: u rounded to float, the FP32 operator, w
 * widened back).  host arrays of n*n doubles. */
int ops_heat_apply(ops_ctx ctx, int n, const double* host_kappa, const double* host_u, int precision,
                   double* host_w);
/* Solve count systems of sizes n[i] together (same parameters). */
int ops_cg_solve_batch(ops_ctx ctx, int count, const int* n, const double* const* host_kappa,
                       const double* const* host_rhs, const ops_cg_params* params, double* const* host_x,
                       ops_cg_stats* stats);

/* ---- serving: continuous batching of heat-conduction solves ----
 * A server owns a context on cfg->device and one device pool of
 * cfg->hbm_budget bytes.  Submitted requests queue in FIFO order; a worker
 * thread admits the oldest ones whenever the running batch has fewer than
 * max_batch solves and the pool has room for the request's arrays (about
 * 92 bytes per cell), advances every admitted solve ticks_per_poll CG
 * iterations at a time in one batch, and retires finished ones, so requests
 * arriving while others run join the batch as memory frees up.  Each
 * request's result is the same alone and in any mix (see ops_cg_solve_batch).
 * The pool and the batch's device tables are allocated by ops_serve_open;
 * the serving loop itself makes no device allocation, and the captured
 * graph of a batch iteration is replayed whatever requests come and go. */
typedef struct ops_server_s* ops_server;
typedef struct {
  int device;
  int64_t hbm_budget;    /* bytes of the request pool */
  int max_batch;         /* solves advanced together (0: 1024) */
  int ticks_per_poll;    /* CG iterations between completion checks (0: 4) */
  ops_cg_params params;  /* tolerance, precision, caps for every request */
} ops_serve_config;
typedef struct {
  int iterations, outer, converged;
  double relres;
  double queue_ms;       /* submit -> admitted */
  double service_ms;     /* admitted -> result ready */
  double latency_ms;     /* submit -> result ready */
  double submit_ms, done_ms;  /* host steady-clock stamps (ms) */
} ops_solve_stats;
int ops_serve_open(ops_server* out, const ops_serve_config* cfg);
/* Queue a solve (arrays of n*n doubles are copied) to relative residual
 * tol in precision OPS_PREC_FP64 or OPS_PREC_MIXED (tol <= 0 or precision
 * < 0: the server's params); *id identifies it.  OPS_ERR_NOMEM if it could
 * never fit the pool. */
int ops_serve_submit(ops_server srv, int n, const double* host_kappa, const double* host_rhs, double tol, int precision,
                     uint64_t* id);
/* OPS_OK and x (n*n doubles) + stats once the solve is done (the request is
 * then forgotten); OPS_ERR_STATE while pending (wait = 0); wait = 1 blocks. */
int ops_serve_poll(ops_server srv, uint64_t id, int wait, double* host_x, ops_solve_stats* stats);
/* Finish running solves, drop queued ones, free the pool and the context. */
int ops_serve_close(ops_server srv);
/* Where the server's worker thread has spent its time since open. */
typedef struct {
  int64_t admitted, completed, rounds;  /* requests admitted / retired; batch rounds run */
  double upload_ms;  /* copying admitted requests' arrays to the device */
  double run_ms;     /* queueing a round's iterations and waiting for them */
  double fetch_ms;   /* copying finished solutions back to host memory */
  double idle_ms;    /* waiting for requests with nothing admitted */
} ops_serve_counters;
int ops_serve_stats(ops_server srv, ops_serve_counters* out);

/* ---- hardware probes behind the reported roofline ----
 * The paper sets its roofline from STREAM, the L3 bandwidth and DGEMM on
 * its CPUs (Sec. 6); these are the GB300 counterparts the bench needs:
 * the FP64 and FP32 arithmetic rates (every SM busy, independent chains),
 * the read bandwidth of a buffer resident in L2, the copy bandwidth of
 * HBM, and the cost of the two synchronisations the tiled schedules use (a
 * grid-wide barrier with one CTA per SM; a release store answered through
 * another CTA's acquire poll).  ops_probe_device runs them on `device`
 * (allocating about 2 GiB for a moment) and fills *out; OPS_ERR_TIMEOUT if
 * a synchronisation probe's bounded wait ran out, OPS_ERR_CUDA or
 * OPS_ERR_NO_DEVICE otherwise on failure. */
typedef struct {
  double fp64_fma_tflops;   /* 2 flops per DFMA */
  double fp64_add_tops;     /* DADD per second / 1e12 */
  double fp32_fma_tflops;   /* 2 flops per FFMA */
  double l2_read_gbs;       /* reads of a buffer of a third of L2 */
  double hbm_copy_gbs;      /* read + write bytes of 1 GiB copies */
  double grid_barrier_us;   /* one grid-wide barrier */
  double flag_roundtrip_us; /* release store -> acquire poll -> answer -> acquire poll */
  int64_t l2_bytes;
  int64_t persisting_l2_max_bytes;  /* cudaDevAttrMaxPersistingL2CacheSize */
  int num_sms;
  int sm_clock_khz_max;
} ops_probe_result;
int ops_probe_device(int device, ops_probe_result* out);

/* ---- one loop without any device allocation ----
 * The paper has no counterpart: this is a service for callers that must not
 * allocate device memory.  cudaMalloc and cudaFree can synchronise the whole
 * GPU, which stalls every other stream of a process that serves requests
 * concurrently; and a program whose device memory belongs to another
 * allocator (a framework's caching allocator, a pool reserved up front)
 * must not grow its footprint behind that allocator's back.  Such callers
 * run a loop here instead of through a context.
 *
 * ops_loop_noalloc runs one parallel loop over caller-owned dats and returns
 * its reductions.  The IR and the access rules are those of ops_par_loop;
 * the written dats come out identical to a single queued loop run by
 * ops_par_loop + ops_execute, and reduction sums agree with it within 1e-12
 * relative (min and max exactly): the partial sums are combined over a
 * launch shape of this entry point's own.  Its only scratch (loop descriptor, reduction partials and
 * slots) is a fixed array of OPS_NOALLOC_SCRATCH_BYTES inside the library's
 * device image: every GPU that loads the library holds it until the process
 * exits.  No call allocates: no cudaMalloc, cudaFree or allocating library
 * routine.
 *   - The first call on a device looks the array's device address up
 *     (cudaGetSymbolAddress, with that device current) and caches it.
 *   - Every call on a device shares the one array and overwrites what the
 *     previous call left there; two calls whose work overlaps on the GPU
 *     (different streams, no ordering between them) race and give wrong
 *     results.  Order them on one stream, or synchronise in between.
 *   - Requests beyond the fixed capacity (more than OPS_MAX_ARGS arguments,
 *     OPS_MAX_INS instructions, OPS_MAX_CONSTS constants,
 *     OPS_MAX_STENCIL_POINTS points per stencil or OPS_MAX_REDS_PER_LOOP
 *     reductions) return OPS_ERR_NOMEM and launch nothing.
 * Arguments, all host memory except the addresses inside views:
 *   dims, range: as ops_par_loop; args[i].handle is ignored;
 *   views[i]: for DAT args, the dat (address of grid point (0,0,0), strides,
 *     allocation box [lo, hi) in grid coordinates; every access must lie
 *     inside it, else OPS_ERR_BOUNDS).  OPS_ERR_INVALID_ARG when a pitch is
 *     smaller than the box's x extent (or, in 3D, a plane smaller than
 *     pitch x y extent), or when the memory of two views overlaps and the
 *     loop writes one of them;
 *   stencil_npts[i], stencil_offsets: for DAT args, the number of stencil
 *     points and their offsets (3 ints each), concatenated in argument order;
 *   scalar_values[i]: the value a SCALAR arg reads;
 *   red_ops[i]: OPS_RED_* of a RED arg; host_red_out[i] receives its result;
 *   stream: cudaStream_t the work is ordered on (NULL = legacy stream).
 * With reductions the call waits for the loop; without, it returns once the
 * work is queued.  Other errors: OPS_ERR_INVALID_ARG (malformed IR or
 * arguments), OPS_ERR_CUDA. */
#define OPS_NOALLOC_SCRATCH_BYTES (128 * 1024)
typedef struct {
  double* ptr0;   /* device address of grid point (0,0,0) */
  int64_t pitch;  /* elements between consecutive y */
  int64_t plane;  /* elements between consecutive z */
  int lo[3];      /* allocation box, grid coordinates, inclusive */
  int hi[3];      /* exclusive */
} ops_dat_view;
int ops_loop_noalloc(int dims, const int* range, int nargs, const ops_arg* args, const ops_dat_view* views,
                     const int* stencil_npts, const int* stencil_offsets, int nins, const int32_t* code,
                     int nconsts, const double* consts, const double* scalar_values, const int* red_ops,
                     double* host_red_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* OPSTILE_H */
