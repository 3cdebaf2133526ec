// Batched many-instance solver: device descriptors shared by batch.cu and the server.
#pragma once
#include "common.cuh"

namespace pogs {

struct BOut;
struct BLoop;

// One instance, all pointers into a device arena.  Pre-conditioned data (A^ = D A E, folded
// function parameters) and the FP32 inverse factor M = L^{-1} (dense lower triangle, ld q).
struct BInst {
  int m, n, lda, q, tall, stage_smem;
  float* A;
  float* M;
  double* H;            // FP64 q x q factorization workspace
  float *D, *E;
  const uint8_t *fh0, *gh0;                     // raw parameters (as given)
  const float *fa0, *fb0, *fc0, *fd0, *fe0, *ga0, *gb0, *gc0, *gd0, *ge0;
  uint8_t *fh, *gh;                             // folded parameters
  float *fa, *fb, *fc, *fd, *fe, *ga, *gb, *gc, *gd, *ge;
  float *x, *y, *xt, *yt, *xh, *yh, *cx, *dy, *mu, *nu, *r, *z, *w;
  float *ox, *oy, *omu, *onu;                   // unscaled outputs
  BOut* out;                                    // report
  BLoop* loop;                                  // saved loop state (resumable runs) or null
};

// Loop state of an instance saved between launches of the iteration kernel (exact: the next
// launch continues with the same rho, pending rescale and Algorithm 3 counters).
struct BLoop {
  double rho, pend;
  int k, l, u, done, status, started;
};

// Per-instance report (mirrors pogs_info).
struct BOut {
  int status, iters;
  double rho, r_pri, r_dual, eps_pri, eps_dual, gap, obj, r_pri_u, r_dual_u;
};

struct BCfg {
  double abs_tol, rel_tol, rho0, alpha, delta, tau, gamma_scale;
  int max_iter, gap_stop, adaptive, sk_sweeps, equil, mixed_chol;
};

constexpr int kBatchThreads = 256;   // fixed: per-instance arithmetic never depends on the batch
// Shared-memory floats for the vectors an iteration phase reads (after the matrix budget).
constexpr int kBatchVecFloats = 6144;

// setup (one CTA per instance) and the persistent iteration kernel
int batch_setup(BInst* d_inst, int count, const BCfg& cfg, cudaStream_t s);
// Run the iteration for the listed instances; max_steps > 0 stops each instance after that many
// iterations in this launch (its loop state is saved in BInst::loop and resumed next launch).
int batch_iterate(BInst* d_inst, int count, const BCfg& cfg, int* d_queue, const int* d_order, int grid,
                  int smem_bytes, int max_steps, cudaStream_t s);
int batch_max_smem();

}  // namespace pogs
