// Batched conjugate-gradient engine for the heat-conduction operator
// (host-side interface shared by cg.cu and serve.cpp).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <array>
#include <vector>

#include "internal.h"

namespace opstile {

// Problem states; only the scalar kernels change them.
enum CgState : int {
  CG_FREE = 0,     // slot unused
  CG_DONE = 1,     // converged or stopped
  CG_OUTER = 2,    // mixed: compute r = b - A x in FP64 and its norm
  CG_INIT = 3,     // mixed: start an inner FP32 solve of A d = r / |r|
  CG_INNER = 4,    // mixed: one FP32 CG iteration
  CG_FINISH = 5,   // mixed: x += |r| d, then back to CG_OUTER
  CG64_INIT = 6,   // FP64: r = p = b, x = 0
  CG64 = 7,        // FP64: one CG iteration
};

// One problem as the kernels see it (device array, one entry per slot).
struct CgProb {
  int n, state, prec, conv;   // prec: 0 FP64 CG, 1 FP32 inner + FP64 refinement
  int it, outer, maxit, maxouter;
  int u0, u1, pp, pad1;       // its work units [u0, u1); pp: which p buffer holds the current direction
  double tol, inner_tol;
  double nb, nr, rho, rho0, alpha, beta, rel, pad2;
  double *b, *x, *r, *p64, *w64, *kx, *ky, *dg;      // FP64: N, N, N, N, N, n(n+1), (n+1)n, N
  float *kx32, *ky32, *dg32, *r32, *p32, *w32, *d32;  // FP32 copies and inner vectors
  float* p32b;                                        // second FP32 direction buffer
  double* pad3;
  double* pad4;
};

// A work unit: rows [j0, j0 + nr) x columns [c0, c0 + w) of one problem.
struct CgUnit {
  int prob, j0, nr, c0, w;
};

// Device bytes one problem of side n needs (all arrays above, 256-byte aligned).
int64_t cg_problem_bytes(int n);
// Work units of one problem of side n.
int cg_unit_count(int n);

// A set of problems advanced together one CG iteration per tick.
class CgBatch {
 public:
  CgBatch(cudaStream_t stream, int num_sms);
  // Fixed capacity: every device table is allocated here, at its final
  // size, so adding and removing problems never allocates and the captured
  // tick graph is reused for every batch composition.  Problems beyond
  // max_slots slots or max_units work units in total fail at the next run
  // (the caller admits only what fits).
  CgBatch(cudaStream_t stream, int num_sms, int max_slots, int max_units);
  ~CgBatch();
  // Add a problem in `slab` (cg_problem_bytes(n) device bytes, owned by the
  // caller); kappa and rhs are host arrays of n*n.  Returns the slot.
  int add(int n, const double* kappa, const double* rhs, double tol, int prec, double inner_tol, int maxit,
          int maxouter, void* slab);
  void remove(int slot);
  // Run `ticks` lockstep iterations for every live problem.
  cudaError_t run(int ticks);
  // Copy states back; fills done slots (state CG_DONE) not yet reported
  // and, if infos is given, their final state (iterations, residual).
  cudaError_t poll(std::vector<int>& done, std::vector<CgProb>* infos = nullptr);
  cudaError_t fetch(int slot, double* host_x, CgProb* info);
  // Device address of a problem's solution and its side; a problem in
  // state CG_DONE is no longer written by any kernel, so its solution may be
  // copied on another stream while later iterations of the batch run.
  const double* solution(int slot) const { return hprob_[slot].x; }
  int side(int slot) const { return hprob_[slot].n; }
  // w = A u for one problem's operator (prec 0: FP64; 1: FP32 with u and w
  // rounded to / widened from float); host arrays of n*n doubles.
  cudaError_t apply(int slot, int prec, const double* host_u, double* host_w);
  int live() const { return nlive_; }
  cudaError_t init_status() const { return init_error_; }
  cudaStream_t stream() const { return stream_; }

 private:
  cudaError_t rebuild_units();
  cudaStream_t stream_;
  int num_sms_;
  std::vector<CgProb> hprob_;   // host mirror (pointers and static fields)
  std::vector<int> live_;       // slot used?
  std::vector<int> reported_;
  int nlive_ = 0;
  CgProb* dprob_ = nullptr;
  int dprob_cap_ = 0;
  CgUnit* dunits_ = nullptr;
  int dunits_cap_ = 0;
  int2* dranges_ = nullptr;   // per slot: its units [x, y)
  int dranges_cap_ = 0;
  int nunits_ = 0;
  DD* dpart_ = nullptr;
  int dpart_cap_ = 0;
  bool units_dirty_ = true;
  std::vector<int> hstate_;
  cudaGraphExec_t gexec_ = nullptr;  // captured tick sequence
  int gticks_ = 0, gg_ = 0, ggs_ = 0;
  std::array<const void*, 5> gargs_{};  // the tables the captured kernels point at
  bool fixed_ = false;
  cudaError_t init_error_ = cudaSuccess;
  int* dcnt_ = nullptr;   // device: unit count, slot count
  int hcnt_[2] = {0, 0};
};

}  // namespace opstile
