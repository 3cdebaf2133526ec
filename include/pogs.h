/*
 * pogs.h -- C interface of a B300-native (sm_103a) graph-form ADMM solver.
 *
 * Problem (Eq. 1):   minimize f(y) + g(x)   subject to   y = A x,
 * with A dense m x n (FP32) and f, g separable in the parametric form of Section 5:
 *
 *     f_i(y_i) = c_i h_i(a_i y_i - b_i) + d_i y_i + (e_i / 2) y_i^2,   a_i != 0, c_i >= 0, e_i >= 0,
 *
 * (g_j likewise).  The solver runs Algorithm 1 (graph projection splitting) with
 * over-relaxation (Section 3.2), the Section 3.4 residual stopping test plus a duality-gap
 * test on the half-step tuple, and Algorithm 3 (adaptive rho), on the problem
 * pre-conditioned by regularized Sinkhorn-Knopp (Algorithm 2) and the Frobenius rescale
 * (Section 4.1.2).  The projection uses the dense reduced updates of Section 3.5 with a
 * factor cached at setup (factorization caching).
 *
 * Conventions shared by every entry point
 *  - Return value: 0 (POGS_OK) or 1 (POGS_MAX_ITER, a valid but unconverged result) on
 *    success, a negative POGS_ERR_* code on failure.  No entry point aborts the process
 *    or traps on the device; device-side failures come back as status codes.
 *  - Pointers documented "host or device" may point to host memory (pageable or pinned)
 *    or to device memory of the current CUDA device; the library detects which.
 *  - All device work is issued on the CUDA stream given to pogs_setup (NULL = legacy
 *    default stream); calls that return results synchronise that stream.
 *  - Vectors are FP32, contiguous, with the lengths stated.  A is row-major
 *    ('R': element (i,j) at A[i*lda + j], lda >= n) or column-major ('C': A[j*lda + i],
 *    lda >= m).
 */
#ifndef POGS_B300_H
#define POGS_B300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Base functions h of the Section 5 library. */
typedef enum {
  POGS_ZERO = 0,      /* 0                                   */
  POGS_ABS = 1,       /* |z|                                 */
  POGS_SQUARE = 2,    /* z^2 / 2                             */
  POGS_HUBER = 3,     /* z^2/2 if |z| <= 1, else |z| - 1/2   */
  POGS_LOGISTIC = 4,  /* log(1 + e^z)                        */
  POGS_HINGE = 5,     /* max(0, 1 - z)                       */
  POGS_MAXPOS = 6,    /* max(0, z)                           */
  POGS_IND_GE0 = 7,   /* indicator of z >= 0                 */
  POGS_IND_LE0 = 8,   /* indicator of z <= 0                 */
  POGS_IND_EQ0 = 9,   /* indicator of z == 0                 */
  POGS_IND_BOX01 = 10, /* indicator of 0 <= z <= 1           */
  POGS_XLOGX = 11      /* z log z (0 at z = 0, +inf for z < 0) */
} pogs_h;

/* Status / error codes. */
enum {
  POGS_OK = 0,
  POGS_MAX_ITER = 1,
  POGS_ERR_ARG = -1,       /* invalid argument (sizes, NULL, a == 0, c < 0, e < 0, bad enum) */
  POGS_ERR_OOM = -2,       /* device allocation failed                                       */
  POGS_ERR_NONFINITE = -3, /* NaN/Inf in the input or in an iterate norm                     */
  POGS_ERR_NUMERIC = -4,   /* non-positive Cholesky pivot (cannot happen for I + G in exact
                              arithmetic; reports corrupted input)                           */
  POGS_ERR_TIMEOUT = -5,   /* a bounded device-side wait gave up                             */
  POGS_ERR_CUDA = -6,      /* a CUDA runtime call failed                                     */
  POGS_ERR_CAPACITY = -7   /* request exceeds a fixed capacity (batch/server/no-alloc sizes) */
};

/* Precision of the one-time Gram formation G = A^T A (m >= n) or A A^T (m < n). */
enum {
  POGS_GRAM_BF16 = 0,   /* BF16 tensor-core MMA, FP32 accumulation                          */
  POGS_GRAM_TF32 = 1,   /* TF32 tensor-core MMA, FP32 accumulation                          */
  POGS_GRAM_BF16X3 = 2, /* split A = hi + lo (both BF16): hi*hi + hi*lo + lo*hi, FP32 accum. */
  POGS_GRAM_FP32 = 3    /* FP32 SIMT                                                        */
};

/* One separable function: per-element parameters, each array of length k (k = m for f,
 * k = n for g), host or device.  NULL a or c means all ones; NULL b, d or e means zeros;
 * h must not be NULL.  Read during pogs_solve only (not retained). */
typedef struct {
  const uint8_t* h;
  const float *a, *b, *c, *d, *e;
} pogs_fn;

/* Solver parameters; pogs_default_params() gives the paper's choices (Section 5). */
typedef struct {
  double abs_tol;    /* eps_abs  (default 1e-4), Section 3.4                          */
  double rel_tol;    /* eps_rel  (default 1e-3)                                        */
  int max_iter;      /* default 10000 (Section 6.1)                                    */
  double rho0;       /* initial rho (default 1)                                        */
  double alpha;      /* over-relaxation (default 1.7, Section 5)                       */
  double delta;      /* Algorithm 3 step (default 1.05)                                */
  double tau;        /* Algorithm 3 hysteresis (default 0.8)                           */
  int sk_sweeps;     /* Algorithm 2 sweeps, fixed count (default 10); 0 = no SK        */
  double gamma;      /* Algorithm 2 regularizer; <= 0 selects (m+n) sqrt(2^-23)        */
  int gram_prec;     /* POGS_GRAM_* (default POGS_GRAM_BF16X3)                         */
  int refine_steps;  /* iterative-refinement steps per projection, 0 or 1 (default 0) */
  int gap_stop;      /* 1: also require |y^T nu + x^T mu| <= eps_abs + eps_rel |f+g|   */
  int adaptive_rho;  /* 1: Algorithm 3 (default); 0: fixed rho                         */
  int equil;         /* 1: Sinkhorn-Knopp + rescale (default); 0: rescale only         */
  int verbose;       /* 0 silent                                                       */
  int loop_mode;     /* 0: device-side loop in one CUDA graph (conditional WHILE node);
                        1: host loop over captured iterations, status read every
                        check_every iterations                                         */
  int check_every;   /* loop_mode 1 only (default 10)                                  */
  int chol_prec;     /* POGS_CHOL_* (default POGS_CHOL_MIXED)                           */
  int proj_mode;     /* POGS_PROJ_DIRECT (default): cached factor of I + A^T A (or I + A A^T);
                        POGS_PROJ_CGLS: indirect projection (Section 3.5), no Gram and no
                        factorization -- CGLS on the reduced least-squares problem, started
                        from the previous projection;
                        POGS_PROJ_LDL (sparse A, pogs_setup_csr only): sparse LDL^T of the
                        quasi-definite K = [I A^T; A -I] (Section 3.5), fill-reducing
                        ordering on the host, factored once on the device and cached;
                        fixed at setup                                                   */
  int cg_max_iter;   /* CGLS steps per projection, at most (default 30)                 */
  double cg_tol;     /* CGLS stop: ||B^T r|| <= cg_tol ||r||, B = [A; I] or [A^T; I]
                        (LSQR's first test with ||B|| = 1; default 1e-4)                */
} pogs_params;

enum { POGS_PROJ_DIRECT = 0, POGS_PROJ_CGLS = 1, POGS_PROJ_LDL = 2 };

/* Arithmetic of the Cholesky factorization of I + G (Section 3.5). */
enum {
  POGS_CHOL_FP64 = 0,  /* every operation in FP64                                          */
  POGS_CHOL_MIXED = 1  /* Schur complement carried as a double-float pair (error-free
                          transformations), 128-blocks factored in FP32, products in FP32
                          (SIMT) or, for blocks of 512 and more, TF32x3 on the tensor cores
                          (about 21 significant bits); from q = 4096 on recursive, with the
                          inverse formed alongside; from q = 1024 on the iteration applies
                          S = (I + G)^{-1} in one symmetric pass                             */
};

/* Timing/precision report of pogs_setup.  factor_ms covers the factorization (and, when it is
 * recursive, the inverse formed alongside); inverse_ms the remaining inverse work, the
 * symmetric operator S and the tile packing. */
typedef struct {
  double ingest_ms, equil_ms, gram_ms, factor_ms, inverse_ms;
  int gram_prec_used, chol_prec_used;
  int64_t device_bytes;  /* device memory the handle owns after setup */
} pogs_setup_report;

/* Per-solve report.  Residuals/tolerances/gap are those of the pre-conditioned problem
 * the iteration runs on (Section 3.4); *_unscaled are ||A x - y|| and ||A^T nu + mu|| of
 * the original problem at the returned tuple. */
typedef struct {
  int status, iters;
  double rho, r_pri, r_dual, eps_pri, eps_dual, gap, obj;
  double r_pri_unscaled, r_dual_unscaled;
  double setup_ms, solve_ms;
} pogs_info;

typedef struct pogs_handle pogs_handle;

/* Fill *p with the defaults listed above. */
void pogs_default_params(pogs_params* p);

/* One-time setup for matrix A (Section 3.5 'factorization caching', Section 4.2, 5):
 * copies A to the device (host or device source), runs Algorithm 2 for p->sk_sweeps
 * sweeps, applies the Frobenius rescale, forms G = A^T A (m >= n) or A A^T (m < n) in
 * p->gram_prec, factors I + G = L L^T in p->chol_prec and caches the result in FP32 packed
 * 128 x 128 lower tiles.  With the default POGS_CHOL_MIXED the Schur complement is carried
 * as a double-float pair (FP64-like) while the block products run in FP32 or, for blocks of
 * 512 and more, in TF32x3 on the tensor cores; POGS_CHOL_FP64 factors entirely in FP64.
 * What is cached: S = (I + G)^{-1} = L^{-T} L^{-1} from q = min(m, n) = 1024 on (mixed
 * precision; one symmetric pass per projection), else M = L^{-1} (two triangular products
 * per projection).  The caller keeps ownership of A.  `stream` is a cudaStream_t
 * (NULL = default).  On success *out owns all device memory until pogs_free.
 * Errors: ARG (m or n < 1, lda too small, order not 'R'/'C', NULL), OOM, NONFINITE,
 * NUMERIC, CUDA. */
int pogs_setup(const float* A, int64_t m, int64_t n, int64_t lda, char order,
               const pogs_params* p, void* stream, pogs_handle** out);

/* Setup for a sparse A given in CSR form (Section 3.5: sparse A; Section 4.1 equilibration
 * over the nonzeros).  rowptr has m + 1 entries with rowptr[0] = 0 and rowptr[m] = nnz;
 * colind and val have nnz entries, the column indices of each row strictly increasing (sorted,
 * no duplicates) and in [0, n); int32 indices, FP32 values; host or device arrays, which the
 * caller keeps.  The handle stores the CSR of A^ and of A^T (a stable device transpose,
 * entries of each column in row order) and runs every pass over A^ as a CSR kernel with the
 * dense pass's epilogue.  p->proj_mode CGLS: no Gram, no factor.  DIRECT: the reduced update's
 * I + A^T A (or I + A A^T) is factored as for dense A, its Gram formed from a temporary dense
 * copy of A^ that setup frees (the factor of a matrix with scattered nonzeros is dense).
 * Errors: ARG (sizes, NULL, a malformed CSR structure), OOM, NONFINITE, NUMERIC, CUDA. */
int pogs_setup_csr(int64_t m, int64_t n, int64_t nnz, const int* rowptr, const int* colind, const float* val,
                   const pogs_params* p, void* stream, pogs_handle** out);

/* Solve with the cached factor: Algorithm 1 + over-relaxation + Algorithm 3 until the
 * Section 3.4 test holds (status 0) or p->max_iter iterations (status 1).  f has m
 * elements, g has n.  Outputs are the unscaled half-step tuple returned by POGS
 * (Section 5): x, mu of length n and y, nu of length m, caller-owned, host or device;
 * any output may be NULL.  info may be NULL.  p may differ from the setup parameters in
 * everything except sk_sweeps, gamma, equil and gram_prec (fixed at setup).
 * Errors: ARG (bad h code, a == 0, c < 0, e < 0), NONFINITE, TIMEOUT, CUDA. */
int pogs_solve(pogs_handle* hdl, const pogs_fn* f, const pogs_fn* g, const pogs_params* p,
               float* x, float* y, float* mu, float* nu, pogs_info* info);

/* pogs_solve from a warm start (Section 5): an initial guess x0 (n, host or device) and/or
 * nu0 (m, host or device), in the original variables; either may be NULL.  The iteration
 * starts on the graph at (x0, A x0) with scaled duals y~ = -nu0 / rho0 and x~ = -A^T y~ (in
 * the pre-conditioned variables: x0 / E, nu0 / D), which keeps x~ + A^T y~ = 0.  A part that
 * is not given starts at zero and the first prox step estimates it (nu^{1/2} is a subgradient
 * of f at y^{1/2}, mu^{1/2} of g at x^{1/2}).  With the handle's cached factor this solves
 * further problems with the same A (new f, g, or a new regularisation weight) from the
 * previous solution.  Outputs, errors and parameters as pogs_solve; pogs_solve is
 * pogs_solve_warm with x0 = nu0 = NULL. */
int pogs_solve_warm(pogs_handle* hdl, const pogs_fn* f, const pogs_fn* g, const pogs_params* p,
                    const float* x0, const float* nu0, float* x, float* y, float* mu, float* nu,
                    pogs_info* info);

/* Release everything the handle owns.  pogs_free(NULL) is a no-op. */
void pogs_free(pogs_handle* hdl);

/* ---- many independent instances ------------------------------------------------------ */

/* One problem of a batch: A row-major m x n (lda >= n), host or device; f has m elements,
 * g has n (same conventions as pogs_solve). */
typedef struct {
  const float* A;
  int64_t m, n, lda;
  pogs_fn f, g;
} pogs_problem;

/* Caller-owned outputs of one problem (host or device, each may be NULL) and its report. */
typedef struct {
  float *x, *y, *mu, *nu;
  pogs_info info;
} pogs_result;

/* Solve `count` independent problems with the same parameters (each one is exactly the
 * problem pogs_setup + pogs_solve would solve).  Problems with min(m, n) <= 512 run in one
 * persistent kernel, one CTA per problem at a time taken from a device work queue, after a
 * batched setup (one CTA per problem); larger ones run through the single-problem path.
 * A problem's result does not depend on which other problems share the batch, on their
 * order, or on the launch configuration (fixed block size and reduction order).  The launch
 * configuration (grid, schedule order, shared-memory staging budget) is chosen by timing a
 * few candidates on the first batch of a given size class (p->verbose > 1 prints them) and
 * cached.  Returns 0 if every problem converged, 1 if some stopped at max_iter (see each
 * out[i].info.status); negative on an error that stopped the batch.  Per-problem setup errors
 * (ARG, NONFINITE, NUMERIC) are reported in out[i].info.status and do not stop the others. */
int pogs_solve_batch(int count, const pogs_problem* probs, const pogs_params* p, pogs_result* out,
                     void* stream);

/* ---- continuous-batching server ---------------------------------------------------------- */

typedef struct pogs_server pogs_server;

/* A finished request: its tag, report and host timestamps (seconds, steady clock) of
 * submission, admission and completion. */
typedef struct {
  int64_t tag;
  pogs_info info;
  double submit_s, admit_s, done_s;
} pogs_server_done;

/* Create a server that keeps admitted requests resident on the device within `hbm_budget`
 * bytes (matrix, factor, scalings and ADMM state; an estimate of each request's footprint is
 * charged at admission and released at completion).  Requests with min(m, n) <= 512 are
 * stepped together by the batched engine, at most `max_resident` of them at a time, admitted
 * first come first served by pogs_server_step; larger ones run on `large_workers` host threads
 * with their own streams through the single-problem path, each admitted (and charged) when a
 * worker starts it, in arrival order.  The two queues are independent: a large request waiting
 * for a worker does not hold back small ones.  The two take turns on the device: a step runs alone, large solves run together, and
 * every large solve that waited through a step starts before the next step.  `stream` carries
 * the batched work.  Errors: ARG, OOM. */
int pogs_server_create(size_t hbm_budget, int large_workers, int max_resident, const pogs_params* p,
                       void* stream, pogs_server** out);

/* Queue a request (host work only: no CUDA call).  The problem's arrays and the output arrays
 * (host or device, may be NULL) must stay valid until the request is returned by
 * pogs_server_poll.  Device inputs are read after work queued before this call on the server's
 * stream (on the legacy default stream when the server was created without one).  Errors: ARG, CAPACITY
 * (a footprint above the whole budget). */
int pogs_server_submit(pogs_server* s, const pogs_problem* prob, float* x, float* y, float* mu, float* nu,
                       int64_t tag);

/* One step of continuous batching: admit waiting small requests (first come, first served)
 * while the budget and the slots allow, set up the new ones, advance every resident batched request by up to
 * `iters` iterations (Algorithm 1 with its adaptive rho, continued exactly from the previous
 * step), and retire the finished ones (outputs copied).  Large requests progress on their own
 * threads between steps; a step waits for the large solves under way to finish.  Returns when
 * the step's device work is done.  Errors: ARG, OOM, CUDA. */
int pogs_server_step(pogs_server* s, int iters);

/* Move up to `max` finished requests into `out`; returns how many. */
int pogs_server_poll(pogs_server* s, pogs_server_done* out, int max);

/* Requests submitted and not yet finished. */
int pogs_server_pending(pogs_server* s);

/* Stop the workers (requests not yet admitted are dropped) and release everything. */
void pogs_server_destroy(pogs_server* s);

/* ---- step-level entry points (the same device code the solver runs) ---------------- */

/* Elementwise parametric prox of Section 5 on device arrays of length k:
 * out_i = argmin_y c_i h_i(a_i y - b_i) + d_i y + (e_i/2) y^2 + (rho_i/2)(y - v_i)^2,
 * rho_i = rho_vec[i] if rho_vec != NULL else rho.  fn arrays, v, rho_vec and out must be
 * device pointers.  Errors: ARG. */
int pogs_prox_eval(const pogs_fn* fn, int64_t k, const float* v, const float* rho_vec,
                   float rho, float* out, void* stream);

/* Copy the equilibration diagonals D (length m) and E (length n) after the rescale
 * (Algorithm 2 + Section 4.1.2); host or device destinations. */
int pogs_get_equil(const pogs_handle* hdl, float* D, float* E);

/* Copy the pre-conditioned matrix A^ = D A E, row-major m x n (ld = n), host or device. */
int pogs_get_ahat(const pogs_handle* hdl, float* Ahat);

/* Apply the cached graph projection (Eq. 9 via the Section 3.5 reduced update) in the
 * pre-conditioned variables: (x, y) = Pi(c, d), c and x of length n, d and y of length m,
 * host or device.  Uses the same kernels as one ADMM iteration (including
 * p->refine_steps refinement steps; p may be NULL for the setup parameters). */
int pogs_project(pogs_handle* hdl, const float* c, const float* d, float* x, float* y,
                 const pogs_params* p);

/* Gram formation of Section 3.5 (the one dense contraction of setup) on its own:
 * G = A^T A (q = n) if m >= n, else G = A A^T (q = m), in precision `gram_prec`
 * (POGS_GRAM_*; BF16, TF32 and BF16x3 run on the tensor cores with FP32 accumulation).
 * A: device, row-major m x n with leading dimension lda >= n.  G: device, q x q row-major
 * (ld q); the lower triangle (i >= j) is written, the strict upper triangle is unspecified.
 * Allocates and frees its own scratch.  Errors: ARG, OOM, CUDA. */
int pogs_gram(const float* A, int64_t m, int64_t n, int64_t lda, int gram_prec, float* G, void* stream);

/* The same Gram formation as pogs_gram for callers that cannot allocate device memory at
 * this point: processes whose device memory is owned by another allocator or admitted
 * against a fixed budget, and latency-critical paths that cannot afford the implicit
 * synchronisation of cudaMalloc/cudaFree.  (The paper has no counterpart; this is an
 * interface convenience.)  Same arguments, results and errors as pogs_gram; it calls no
 * cudaMalloc, cudaFree or other allocating routine.
 * Scratch: one fixed 32 MiB device array inside the library, reserved on every device that
 * loads it and held until the process exits.  Its first 256 bytes hold a status word; the
 * rest holds the packed operands, rp * Kp * b bytes with rp = q rounded up to 128, Kp = the
 * contraction length (m if m >= n, else n) rounded up to 64 (32 for TF32), and b = 2 for
 * BF16, 4 for TF32 and BF16x3; POGS_GRAM_FP32 needs none.  A problem is accepted when
 * rp * Kp * b <= 32 MiB - 512 bytes (the status word's 256 bytes and 256 bytes of slack the
 * packing keeps); larger ones are rejected with POGS_ERR_CAPACITY before any device work.
 * The first call on each device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture.  Each call
 * waits for its own work on `stream` to finish (it reads the status word back) before it
 * returns.  Every call shares the one array and leaves its last contents there: calls that
 * overlap on the GPU (different streams or threads) race and must be serialised by the
 * caller. */
int pogs_gram_noalloc(const float* A, int64_t m, int64_t n, int64_t lda, int gram_prec, float* G, void* stream);

/* ---- instrumentation ------------------------------------------------------------------ */

/* Fill *r with the setup phase times (CUDA events on the setup stream), the Gram and
 * Cholesky precisions actually used, and the device memory the handle owns. */
int pogs_get_setup_report(const pogs_handle* hdl, pogs_setup_report* r);

/* Time each kernel of one ADMM iteration of the last solve on the handle's stream with CUDA
 * events, averaged over `reps` launches (reps >= 1) after one warm-up launch of each.
 * ms[0..5]: prox step, first A pass (column sums if m >= n, row dots if m < n), L^{-1}
 * product, L^{-T} product, second A pass, stopping/adaptive-rho check; ms[6]: one whole
 * iteration.  When the iteration applies S = (I + G)^{-1} in one symmetric pass, ms[2] is that
 * pass and ms[3] (and bytes[3]) are 0.  bytes[0..6]: the algorithmic HBM bytes each launch must move (A once per pass,
 * the triangle q(q+1)/2 once per product, the vectors it reads and writes).  Either array
 * may be NULL.  Overwrites the iterate state of the last solve (solve again before reading
 * results).  Errors: ARG (no prior solve, reps < 1), CUDA. */
int pogs_time_kernels(pogs_handle* hdl, int reps, double* ms, double* bytes);

/* Number of kernel launches this library has issued in the process so far (graph replays
 * included). */
long long pogs_kernel_launches(void);

/* Number of device memory allocations this library has requested in the process so far
 * (stream-ordered pool allocations and cudaMalloc / cudaMallocAsync calls alike). */
long long pogs_device_allocations(void);

/* Failure detection: every device-side wait of the tensor-core kernels (mbarrier phases of the
 * TMA / MMA pipeline) is bounded (about 2 s of SM clock) and reports POGS_ERR_TIMEOUT instead of
 * spinning forever.  This runs that wait once on a barrier no thread completes, on `stream`,
 * and returns its status: POGS_ERR_TIMEOUT when the bound works (the context stays usable),
 * POGS_ERR_CUDA / POGS_ERR_OOM on a runtime failure. */
int pogs_check_bounded_wait(void* stream);

/* Symbolic analysis of the sparse LDL^T factorization of the quasi-definite matrix
 * K = [I A^T; A -I] (Section 3.5: for sparse A, factor K once and cache the factor), for the
 * m x n pattern of A given in CSR (rowptr: m + 1 entries, rowptr[0] = 0; colind: sorted and
 * unique within each row, in [0, n); host arrays the caller keeps).  Host work only, no device
 * call; the ordering runs on up to 16 host threads (same result on any number), and calls from
 * several threads at once are independent.  The unknowns of K are numbered x_0..x_{n-1}, then y_0..y_{m-1} (index n + i).
 * Outputs (each may be NULL): stats[0..7] = N = n + m, structural nonzeros of L below the
 * diagonal, supernodes, levels of the supernodal tree, largest frontal matrix, factor entries
 * stored, update-matrix entries, frontal scratch entries; perm[N]: the fill-reducing ordering
 * (new position -> unknown); colcount[N]: nonzeros of each column of L below the diagonal, in
 * the new order.  Errors: ARG (sizes, NULL, malformed pattern), OOM (host memory). */
int pogs_ldl_analyze(int64_t m, int64_t n, const int* rowptr, const int* colind, int64_t* stats, int* perm,
                     int* colcount);

#ifdef __cplusplus
}
#endif

#endif /* POGS_B300_H */
