// Launch wrappers for the device kernels (definitions in iter.cu and setup.cu).
#pragma once
#include "common.cuh"

namespace pogs {

// Epilogues of the column-sum GEMV  t = A^T [v1, v2]  (one column per output element).
enum EpiT : int {
  EPT_RAW = 0,      // out1 = t1, out2 = t2
  EPT_TALL_R = 1,   // tall projection input r = c + A^T d; dual residual from t2 = A^T nu; x~ = -A^T y~
  EPT_FAT_X = 2,    // fat x^{k+1} = c + A^T (d - y^{k+1}); x~ = -A^T y~; dual residual
  EPT_SK_COL = 3,   // Algorithm 2 e-update; Frobenius partial sum e_j * colsum_j
  EPT_REFINE = 4,   // refinement residual out1 = r - x0 - t1 (tall)
  EPT_CG_R = 5,     // CGLS (indirect projection): r_top = top - M u0             (fat: M = A^T)
  EPT_CG_S0 = 6,    //   r_bot = sign*bot - u0, s = M^T r_top + r_bot, p = s       (tall)
  EPT_CG_Q = 7,     //   q = M p                                                  (fat)
  EPT_CG_S = 8,     //   s = M^T r_top + r_bot                                    (tall)
};
// Epilogues of the row-dot GEMV  u = A [x1, x2]  (one row per output element).
enum EpiN : int {
  EPN_RAW = 0,      // out1 = u1, out2 = u2
  EPN_TALL_Y = 1,   // tall y^{k+1} = A x^{k+1}; y~ += d - y^{k+1}; primal residual from u2 = A x^{1/2}
  EPN_FAT_R = 2,    // fat projection input r = A c - d; primal residual
  EPN_SK_ROW = 3,   // Algorithm 2 d-update
  EPN_REFINE = 4,   // refinement residual out1 = r - y0 - u1 (fat)
  EPN_CG_R = 5,     // CGLS: r_top = top - M u0 (tall: M = A)
  EPN_CG_S0 = 6,    //   init gradient (fat)
  EPN_CG_Q = 7,     //   q = M p (tall)
  EPN_CG_S = 8,     //   s = M^T r_top + r_bot (fat)
};
// Epilogues of the packed-triangle products z = M v (M = L^{-1}) and M^T v.
enum EpiR : int {
  EPR_RAW = 0,      // out1 = result (all padded entries)
  EPR_TALL_X = 1,   // x^{k+1} = result (+ in1); x~ += c - x^{k+1}
  EPR_FAT_Y = 2,    // y^{k+1} = d + result (+ in1); y~ += d - y^{k+1}; w = d - y^{k+1}
  EPR_ADD = 3,      // out1 = in1 + result (refinement correction)
};

// Everything an epilogue may read or write.  Unused fields are null.
struct EpiArgs {
  float *out1, *out2;
  const float *in1, *in2;             // extra inputs (refinement)
  const float *cx, *dy, *yh, *mu;     // c, d, y^{1/2}, mu^{1/2}
  float *x, *xt, *y, *yt, *r, *w;
  const float *D, *E;                 // diagonal scalings (unscaled residuals)
  float* sk_vec;                      // SK output vector (d or e)
  float sk_num, sk_reg;               // n and gamma/m (rows) or m and gamma/n (cols)
  Df* res_part;                       // 2 per block: residual^2, unscaled residual^2 (double-float)
  // CGLS (indirect projection): see cgls.cu
  float *cg_rt, *cg_rb, *cg_s, *cg_p;  // r_top, r_bot, s, p
  const float *cg_top, *cg_bot, *cg_u; // top, bot, u0
  float cg_sign;                       // bot enters as cg_sign * cg_bot
  const int* cg_done;                  // a set flag makes the GEMV return at once
};

// Loop parameters in device memory (so a captured graph survives parameter changes).
struct DevCfg {
  double abs_tol, rel_tol, alpha, delta, inv_delta, tau;
  int max_iter, gap_stop, adaptive, pad_;
};

// Geometry of the two GEMV shapes, chosen at setup.
struct GemvGeom {
  int t_cols_per_blk;   // 1024 (fixed: 256 threads x float4)
  int t_ncolblk, t_nsplit, t_rows;
  int keep_rows;   // leading rows of A^ every dense pass reads under the L2 evict-last policy
  int n_rows, n_cols, n_nrowblk, n_ncolsplit;
  // Sparse A (csr.cu): the two passes run the CSR kernels over A^ (m rows) and A^T (n rows)
  // instead; n_nrowblk and t_ncolblk are then their grid sizes (the number of residual
  // partials each pass writes), sp_lanes_* their lanes per row.
  int sparse, sp_lanes_n, sp_lanes_t;
  const int *rp_n, *ci_n, *rp_t, *ci_t;
  const float *va_n, *va_t;
  float* pack;   // max(m, n) x 4 floats: interleaved right-hand sides of the long gathers
};
GemvGeom choose_geometry(int64_t m, int64_t n, int64_t lda, int num_sms);
// Back to normal L2 eviction priority for the first `bytes` of A (see GemvGeom::keep_rows).
void launch_l2_release(const float* A, size_t bytes, cudaStream_t s);

// ---- sparse A (csr.cu) ---------------------------------------------------------------------
void csr_geometry(GemvGeom& g, int64_t m, int64_t n, int64_t nnz, int num_sms);
// One pass over sparse A^ (trans: column sums via the CSR of A^T), with the dense pass's epilogue.
void launch_spmv(bool trans, int nrhs, bool sq, int epi, const GemvGeom& g, int m, int n, const float* v1,
                 const float* v2, const float* v3, const EpiArgs& ep, const DevState* guard, cudaStream_t s);
// Extra launches (right-hand-side interleaving) of one iteration's two main passes.
int csr_pack_launches(const GemvGeom& g, int m, int n);
// Flags POGS_ERR_ARG (structure) or POGS_ERR_NONFINITE (values) in *err.
void launch_csr_check(const int* rp, const int* ci, const float* va, int64_t m, int64_t n, int64_t nnz, int* err,
                      cudaStream_t s);
// Chunks of the stable multi-split (its table holds chunks x n ints).
int csr_transpose_chunks(int64_t nnz, int64_t n);
// CSR of A^T (t_rp: n + 1, t_ci / t_va / perm: nnz) from the CSR of A; scratch rowidx (nnz),
// cnt (chunks x n, zeroed), tot (n).
void launch_csr_transpose(const int* rp, const int* ci, const float* va, int64_t m, int64_t n, int64_t nnz,
                          int nch, int* rowidx, int* cnt, int* tot, int* t_rp, int* t_ci, float* t_va, int* perm,
                          cudaStream_t s);
// va <- D va E on the CSR values; t_va[i] = va[perm[i]].
void launch_csr_scale(const int* rp, const int* ci, float* va, int64_t m, const float* D, const float* E,
                      const int* perm, int64_t nnz, float* t_va, cudaStream_t s);
// Scatter the CSR matrix into a zeroed m x lda row-major buffer.
void launch_csr_densify(const int* rp, const int* ci, const float* va, int64_t m, float* A, int64_t lda,
                        cudaStream_t s);

// ---- iteration kernels (iter.cu) --------------------------------------------------------
void launch_prox_step(int n, int m, const float* x, float* xt, float* xh, float* cx, float* mu,
                      const float* y, float* yt, float* yh, float* dy, float* nu,
                      FnDev g, FnDev f, const DevState* st, const DevCfg* cfg, Df* part,
                      int nblocks, cudaStream_t s);
// Whether a dense column-sum pass with epilogue epi runs as two launches (streaming, then the
// final reduction with the epilogue) instead of one with an in-kernel last-block reduction.
bool colsum_split(const GemvGeom& g, int epi);
void launch_gemv_t(int nrhs, bool sq, int epi, const float* A, int64_t lda, int m, int n,
                   const float* v1, const float* v2, const float* v3, const GemvGeom& g, float* part,
                   unsigned* cnt,
                   const EpiArgs& ep, const DevState* guard, cudaStream_t s);
void launch_gemv_n(int nrhs, bool sq, int epi, const float* A, int64_t lda, int m, int n,
                   const float* x1, const float* x2, const GemvGeom& g, float* part, unsigned* cnt,
                   const EpiArgs& ep, const DevState* guard, cudaStream_t s);
void launch_trmv(bool trans, int epi, const float* Mt, int T, int q, const float* vin, float* part,
                 unsigned* cnt, const EpiArgs& ep, const DevState* guard, cudaStream_t s);
// y = S v with S = M^T M = (I + G)^{-1} as packed lower tiles (diagonal tiles full); part holds
// T x T x 128 floats, cnt T counters.
void launch_symv(int epi, const float* St, int T, int q, const float* vin, float* part, unsigned* cnt,
                 const EpiArgs& ep, const DevState* guard, cudaStream_t s);
void launch_check(DevState* st, const DevCfg* cfg, const Df* prox_part, int nprox,
                  const Df* pri_part, int npri, const Df* dual_part, int ndual,
                  unsigned long long cond_handle, int use_cond, cudaStream_t s);
void launch_prox_eval(FnDev fn, int64_t k, const float* v, const float* rho_vec, float rho, float* out,
                      cudaStream_t s);
void launch_fold(FnDev raw, int64_t k, const float* scale, int is_f, uint8_t* h, float* a, float* b,
                 float* c, float* d, float* e, int* err, cudaStream_t s);
void launch_fill(float* p, int64_t k, float v, cudaStream_t s);
void launch_warm(const float* src, const float* scale, int64_t k, float factor, float* out_pos, float* out_neg,
                 cudaStream_t s);

// ---- CGLS indirect projection (cgls.cu) ----------------------------------------------------
struct CgState {
  double gamma;     // ||s||^2 of the current step
  double pnorm2;    // ||p||^2
  double rnorm2;    // ||r_top||^2 + ||r_bot||^2
  double gmin;      // smallest gamma of this projection (divergence test)
  int done, steps, max_steps;
  float tol;
};
// After the init passes: gamma and ||r||^2 from the init partials, steps = 0, done flag.
void launch_cg_start(CgState* cg, const DevState* st, const Df* r0_part, int nr0, const Df* s0_part, int ns0,
                     cudaStream_t s);
// x += alpha p on u, r_top -= alpha q, r_bot -= alpha p; alpha = gamma / (||q||^2 + ||p||^2).
void launch_cg_alpha(CgState* cg, const DevState* st, const Df* q_part, int nq, float* u, float* rt, float* rb,
                     const float* p, const float* q, int ntop, int nu, Df* r_part, int nblk, cudaStream_t s);
// p = s + beta p (beta = ||s_new||^2 / gamma); the last block updates gamma, ||p||^2, ||r||^2,
// steps and the stop flag (||s|| <= tol ||r|| or the step cap).
void launch_cg_beta(CgState* cg, const DevState* st, const Df* s_part, int ns, const Df* r_part, int nr,
                    float* p, const float* sv, int nu, Df* p_part, unsigned* cnt, int nblk, cudaStream_t s);
// Blocks of the elementwise CGLS kernels for k elements.
int cg_blocks(int64_t k);
// Tall: x~ += c - x.  Fat: y = d + z, w = d - y, y~ += d - y.
void launch_cg_tall_finish(int n, float* xt, const float* cx, const float* x, const DevState* st, cudaStream_t s);
void launch_cg_fat_finish(int m, const float* dy, const float* z, float* y, float* w, float* yt,
                          const DevState* st, cudaStream_t s);
void launch_unscale(int n, int m, const float* xh, const float* mu, const float* yh, const float* nu,
                    const float* D, const float* E, float* x, float* muo, float* y, float* nuo,
                    cudaStream_t s);
void launch_axpby(int64_t k, float a, const float* x, float b, const float* y, float* out, cudaStream_t s);

// ---- setup kernels (setup.cu) -------------------------------------------------------------
void launch_copy_in(const float* src, int64_t m, int64_t n, int64_t lds, bool colmajor, float* A,
                    int64_t lda, int* err, cudaStream_t s);
void launch_scale(float* A, int64_t lda, int64_t m, int64_t n, const float* D, const float* E,
                  cudaStream_t s);
// One Sinkhorn-Knopp sweep (d from e, then e from d) in one pass over A: for lda <= 12288 and
// m >= 2368 (sk_sweep_fits).  part: sk_sweep_blocks() x lda floats; frob_part:
// 2 sk_sweep_finish_blocks(lda) pairs (the Frobenius partials of the sweep's e, as the
// column-sum pass leaves them for launch_sk_finish).
bool sk_sweep_fits(int64_t m, int64_t lda);
int sk_sweep_blocks();
int sk_sweep_finish_blocks(int64_t lda);
int launch_sk_sweep(const float* A, int64_t lda, int64_t m, int64_t n, float* dvec, float* evec, double gamma,
                    float* part, Df* frob_part, cudaStream_t s);
void launch_sk_finish(const float* dvec, const float* evec, int64_t m, int64_t n, const Df* frob_part,
                      int nfrob, int64_t q, float* D, float* E, cudaStream_t s);
// C[M x N] = alpha op(A) op(B) + beta C (row-major, SIMT); lower_only skips tiles above
// the diagonal of C.
void gemm_f32(bool ta, bool tb, int64_t M, int64_t N, int64_t K, float alpha, const float* A, int64_t lda,
              const float* B, int64_t ldb, float beta, float* C, int64_t ldc, bool lower_only,
              cudaStream_t s, int tri = 0);
void gemm_f64(bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t lda,
              const double* B, int64_t ldb, double beta, double* C, int64_t ldc, bool lower_only,
              cudaStream_t s);
void launch_gram_to_f64(const float* G, int64_t ldg, int64_t q, double* H, int64_t ldh, cudaStream_t s);
// FP64 products of FP32-rounded inputs: C (FP64) = alpha op(A) op(B) + beta C with the
// products and their sum over K formed in FP32.
// Right-looking blocked Cholesky of H (lower, in place).  mixed: trailing products in FP32
// (FP64 diagonal blocks, panel solves and Schur complement).
int chol_f64(double* H, int64_t ldh, int64_t q, double* work, int* err, cudaStream_t s);
// Stream-ordered allocation from the library's per-device pool (solver.cu); free with
// cudaFreeAsync on a stream ordered after the last use.  Returns 0 or POGS_ERR_OOM / _CUDA.
int pool_alloc(void** q, size_t bytes, cudaStream_t s);
// Mixed-precision factorization (chol.cu) of I + G: G (lower triangle, ld ldh) is overwritten
// with the hi part of the double-float Schur complement, Hlo (same layout) receives the lo
// part; the FP32 off-diagonal panels of L go to Lf and the diagonal 128-blocks of L^{-1} to
// Md.  ldh, ldf, ldm must be multiples of 4.
int chol_mixed(float* G, float* Hlo, int64_t ldh, int64_t q, float* Lf, int64_t ldf, float* Md, int64_t ldm,
               int* err, cudaStream_t s);
// Recursive factorization of I + G with its inverse (chol.cu): at each level of a 2 x 2 block
// split, L21 = H21 M11^T, H22 -= L21 L21^T on the double-float pair, M21 = -M22 L21 M11; the
// products of blocks of 512 and more on the tensor cores (TF32x3), leaves are the one-CTA 128-block
// kernel.  Writes the whole lower triangle of M = L^{-1} to Md (and the off-diagonal blocks of L
// to Lf); work holds (q/2 + 128) x (q/2) floats.
int chol_inv_mixed(float* G, float* Hlo, int64_t ldh, int64_t q, float* Lf, int64_t ldf, float* Md, int64_t ldm,
                   float* work, int* err, cudaStream_t s);
void launch_leaf_inverse(const double* L, int64_t ldl, int64_t q, float* Minv, int64_t ldm, cudaStream_t s);
void launch_l_to_f32(const double* L, int64_t ldl, int64_t q, float* Lf, int64_t ldf, cudaStream_t s);
// M = L^{-1} (lower, FP32) by recursive 2 x 2 block inversion; tensor: its products of blocks of
// 512 and more in TF32x3 on the tensor cores (else FP32 SIMT).
int tri_inverse_f32(const float* L, int64_t ldl, int64_t q, float* M, int64_t ldm, float* work, bool tensor,
                    int* err, cudaStream_t s);
// Tensor-core GEMM in TF32x3 (gram.cu): C op= X Y^T with X, Y read from row-major A, B (or their
// transposes); TC_EPI_STORE: C = alpha X Y^T; TC_EPI_DF_SUB: (C, Clo) -= X Y^T on and below the
// diagonal (lower: lower tiles only).  scratch == nullptr returns the scratch size in *need_bytes.
enum : int { TC_EPI_STORE = 0, TC_EPI_DF_SUB = 2 };
int tc_gemm_tf32x3(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda, bool transA, const float* B,
                   int64_t ldb, bool transB, float alpha, float* C, float* Clo, int64_t ldc, int epi, bool lower,
                   void* scratch, size_t scratch_bytes, size_t* need_bytes, int* err, cudaStream_t s,
                   bool kskip = false);   // kskip: X[i][k] = Y[i][k] = 0 for k < i (skip those K boxes)
// Status of one bounded barrier wait that no thread completes (POGS_ERR_TIMEOUT expected).
int bounded_wait_probe(cudaStream_t s);
// C = alpha A B (row-major FP32), the special case above.
int tc_gemm_nn_tf32x3(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda, const float* B, int64_t ldb,
                      float alpha, float* C, int64_t ldc, void* scratch, size_t scratch_bytes, size_t* need_bytes,
                      int* err, cudaStream_t s);
// Lower 128-tiles of M (sym: diagonal tiles copied whole, else their upper part zeroed).
void launch_pack_tiles(const float* M, int64_t ldm, int64_t q, int T, float* Mt, cudaStream_t s, bool sym = false);
// Tensor-core Gram (gram.cu): G = X X^T over the K-major packed operand(s).
int gram_tensor(int prec, const float* A, int64_t lda, int64_t m, int64_t n, bool tall, float* G,
                int64_t ldg, void* scratch, size_t scratch_bytes, size_t* need_bytes, int* err,
                cudaStream_t s);

}  // namespace pogs
