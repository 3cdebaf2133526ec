// Host orchestration and the C interface (include/pogs.h).
//
// Setup (Section 3.5 'factorization caching', Algorithm 2, Section 4.1.2, Section 5):
//   ingest A -> Sinkhorn-Knopp sweeps (row pass + column pass per sweep) -> Frobenius rescale
//   -> A^ = D A E in place -> Gram G -> FP64 Cholesky of I + G -> FP32 M = L^{-1} in tiles.
// Solve: fold D, E into the function parameters (Eq. 12), then run the iteration body
//   (iter.cu) inside a CUDA graph whose conditional WHILE node is cleared by the on-device
//   stopping test, so a whole solve is one graph launch with no host round trip.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <mutex>
#include <vector>

#include "kernels.h"
#include "ldl.h"

using namespace pogs;

struct pogs_handle {
  int64_t m = 0, n = 0, lda = 0, q = 0;
  bool tall = true;
  int T = 0;
  int64_t nv = 0, mv = 0;
  int num_sms = 148;
  cudaStream_t stream = nullptr;   // caller's stream
  cudaStream_t cap = nullptr;      // private stream used for graph capture
  pogs_params sp{};
  GemvGeom geom{};
  int nprox = 0;
  int gram_used = -1;
  float* A = nullptr;               // dense A^ (row-major, pitch lda); null for sparse A
  // sparse A: CSR of A^ (m rows) and of A^T (n rows); perm maps the second's entries to the first's
  bool sparse = false;
  int64_t nnz = 0;
  int *csr_rp = nullptr, *csr_ci = nullptr, *csc_rp = nullptr, *csc_ci = nullptr, *csc_perm = nullptr;
  float *csr_va = nullptr, *csc_va = nullptr;
  float *D = nullptr, *E = nullptr;
  float* Mt = nullptr;              // packed lower tiles of M = L^{-1} (two triangular products)
  float* St = nullptr;              // packed lower tiles of S = M^T M = (I + G)^{-1} (one pass), or null
  float* part_sy = nullptr;         // T x T x 128 partials of the symmetric product
  float *x = nullptr, *y = nullptr, *xt = nullptr, *yt = nullptr, *xh = nullptr, *yh = nullptr;
  float *cx = nullptr, *dy = nullptr, *mu = nullptr, *nu = nullptr, *r = nullptr, *z = nullptr, *w = nullptr;
  float *x0 = nullptr, *v0 = nullptr, *r2 = nullptr, *tn = nullptr;
  float *ox = nullptr, *oy = nullptr, *omu = nullptr, *onu = nullptr;
  uint8_t *fh = nullptr, *gh = nullptr, *rh = nullptr;
  float *fa, *fb, *fc, *fd, *fe, *ga, *gb, *gc, *gd, *ge, *ra, *rb, *rc, *rd, *re;
  float *part_t = nullptr, *part_n = nullptr, *part_tr = nullptr;
  unsigned *cnt_t = nullptr, *cnt_n = nullptr, *cnt_tr = nullptr;
  Df *prox_part = nullptr, *pri_part = nullptr, *dual_part = nullptr;   // block partials (double-float)
  // indirect projection (CGLS): vectors, state, partials
  bool indirect = false;             // set up without a factor (proj_mode CGLS)
  LdlFactor* ldl = nullptr;          // sparse LDL^T of K (proj_mode LDL, CSR input)
  float *cg_rt = nullptr, *cg_rb = nullptr, *cg_s = nullptr, *cg_p = nullptr, *cg_q = nullptr, *cg_z = nullptr;
  CgState* cg = nullptr;
  CgState* cg_host = nullptr;        // pinned staging
  Df *cg_r0_part = nullptr, *cg_s0_part = nullptr, *cg_q_part = nullptr, *cg_s_part = nullptr;
  Df *cg_r_part = nullptr, *cg_p_part = nullptr;
  unsigned* cg_cnt = nullptr;
  int cg_nblk = 1;
  int graph_cg = -1;
  DevState* st = nullptr;
  DevCfg* cfg = nullptr;
  DevState* st_host = nullptr;     // pinned mirror
  DevCfg* cfg_host = nullptr;      // pinned staging
  cudaGraphExec_t gexec = nullptr;
  int graph_refine = -1, graph_mode = -1;
  double setup_ms = 0.0;
  double phase_ms[5] = {0, 0, 0, 0, 0};
  cudaEvent_t ev[6] = {};
  bool solved = false;
  int64_t device_bytes = 0;
  std::vector<void*> allocs;
};

std::atomic<long long> pogs::g_launch_count{0};
std::atomic<long long> pogs::g_alloc_count{0};
thread_local int pogs::g_capture_depth = 0;

// Stream-ordered device memory: one pool per device that keeps freed memory cached up to a
// threshold, so that setup, solve and free on one stream never synchronise the device (plain
// cudaMalloc / cudaFree do, which would serialise concurrent solves on other streams).
int pogs::pool_alloc(void** q, size_t bytes, cudaStream_t s) {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  *q = nullptr;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return POGS_ERR_CUDA;
  }
  cudaMemPool_t pool;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!pools[dev]) {
      cudaMemPoolProps props = {};
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      cudaMemPool_t p = nullptr;
      if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
        cudaGetLastError();
        return POGS_ERR_CUDA;
      }
      uint64_t keep = 16ull << 30;   // bytes kept cached across synchronisations
      cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
      pools[dev] = p;
    }
    pool = pools[dev];
  }
  count_alloc();
  if (cudaMallocFromPoolAsync(q, bytes, pool, s) != cudaSuccess) {
    cudaGetLastError();
    *q = nullptr;
    return POGS_ERR_OOM;
  }
  return 0;
}

namespace {

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      if (getenv("POGS_DEBUG")) fprintf(stderr, "pogs: %s failed: %s (%s:%d)\n", #call, \
                                        cudaGetErrorString(e_), __FILE__, __LINE__);  \
      return e_ == cudaErrorMemoryAllocation ? POGS_ERR_OOM : POGS_ERR_CUDA;          \
    }                                                                                 \
  } while (0)

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <class T>
int dalloc(pogs_handle* h, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  void* q = nullptr;
  const int rc = pool_alloc(&q, count * sizeof(T), h->stream);
  if (rc != 0) return rc;
  h->allocs.push_back(q);
  h->device_bytes += (int64_t)(count * sizeof(T));
  *p = static_cast<T*>(q);
  if (cudaMemsetAsync(q, 0, count * sizeof(T), h->stream) != cudaSuccess) return POGS_ERR_CUDA;
  return 0;
}

// Pinned host slots for each handle's status / parameter mirror, allocated in chunks and
// recycled (never released while the library is loaded: cudaFreeHost synchronises the device).
constexpr size_t kPinSlot = 512;
static_assert(sizeof(DevState) + sizeof(DevCfg) + sizeof(CgState) + 16 <= kPinSlot, "pinned slot too small");
std::mutex g_pin_mu;
std::vector<void*> g_pin_free;

void* pin_slot_get() {
  std::lock_guard<std::mutex> lk(g_pin_mu);
  if (g_pin_free.empty()) {
    void* chunk = nullptr;
    if (cudaMallocHost(&chunk, 64 * kPinSlot) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    for (int i = 63; i >= 0; --i) g_pin_free.push_back(static_cast<char*>(chunk) + i * kPinSlot);
  }
  void* p = g_pin_free.back();
  g_pin_free.pop_back();
  memset(p, 0, kPinSlot);
  return p;
}
void pin_slot_put(void* p) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_pin_mu);
  g_pin_free.push_back(p);
}

// Scratch that lives only during setup (stream-ordered: freed on the setup stream).
struct Scratch {
  cudaStream_t s = nullptr;
  std::vector<void*> ptrs;
  ~Scratch() {
    for (void* p : ptrs) cudaFreeAsync(p, s);
  }
  template <class T>
  int get(T** p, size_t count, cudaStream_t st) {
    s = st;
    void* q = nullptr;
    const int rc = pool_alloc(&q, (count ? count : 1) * sizeof(T), st);
    if (rc != 0) return rc;
    ptrs.push_back(q);
    *p = static_cast<T*>(q);
    if (cudaMemsetAsync(q, 0, (count ? count : 1) * sizeof(T), st) != cudaSuccess) return POGS_ERR_CUDA;
    return 0;
  }
};

#define TRY(x)          \
  do {                  \
    int rc_ = (x);      \
    if (rc_ < 0) return rc_; \
  } while (0)

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

FnDev fn_f(const pogs_handle* h) { return FnDev{h->fh, h->fa, h->fb, h->fc, h->fd, h->fe}; }
FnDev fn_g(const pogs_handle* h) { return FnDev{h->gh, h->ga, h->gb, h->gc, h->gd, h->ge}; }

EpiArgs epi0() {
  EpiArgs e;
  memset(&e, 0, sizeof(e));
  return e;
}

// CGLS steps per projection for a solve with parameters p: 0 selects the direct projection.
// A handle set up without a factor always projects indirectly (at least one step).
int cg_steps_for(const pogs_handle* h, const pogs_params* p) {
  if (h->indirect || p->proj_mode == POGS_PROJ_CGLS) return std::max(1, p->cg_max_iter);
  return 0;
}

// Indirect projection of one iteration (Section 3.5): `steps` unrolled CGLS steps, each of
// which returns at once after the stopping test has fired.  Tall: u = x (the previous x is the
// warm start), M = A^; fat: u = z (kept from the previous projection), M = A^T.  The passes
// that give the residual norms, x~ and the final y (tall) or x (fat) are those of the direct
// projection.
void enqueue_projection_cgls(pogs_handle* h, int steps, cudaStream_t s) {
  const int m = (int)h->m, n = (int)h->n;
  const GemvGeom& g = h->geom;
  const int* done = &h->cg->done;
  if (h->tall) {
    // dual residual ||A^T nu + mu||, x~ = -A^T y~ (r = c + A^T d is not needed here)
    EpiArgs e1 = epi0();
    e1.r = h->r; e1.cx = h->cx; e1.mu = h->mu; e1.E = h->E; e1.xt = h->xt; e1.res_part = h->dual_part;
    launch_gemv_t(3, false, EPT_TALL_R, h->A, h->lda, m, n, h->dy, h->nu, h->yt, g, h->part_t, h->cnt_t, e1, h->st, s);
    // r_top = d - A x0 ; r_bot = c - x0, s = A^T r_top + r_bot, p = s
    EpiArgs a = epi0();
    a.cg_top = h->dy; a.cg_rt = h->cg_rt; a.res_part = h->cg_r0_part;
    launch_gemv_n(1, false, EPN_CG_R, h->A, h->lda, m, n, h->x, nullptr, g, h->part_n, h->cnt_n, a, h->st, s);
    EpiArgs b = epi0();
    b.cg_bot = h->cx; b.cg_sign = 1.0f; b.cg_u = h->x; b.cg_rb = h->cg_rb; b.cg_s = h->cg_s; b.cg_p = h->cg_p;
    b.res_part = h->cg_s0_part;
    launch_gemv_t(1, false, EPT_CG_S0, h->A, h->lda, m, n, h->cg_rt, nullptr, nullptr, g, h->part_t, h->cnt_t, b,
                  h->st, s);
    launch_cg_start(h->cg, h->st, h->cg_r0_part, g.n_nrowblk, h->cg_s0_part, g.t_ncolblk, s);
    for (int k = 0; k < steps; ++k) {
      EpiArgs q = epi0();
      q.out1 = h->cg_q; q.res_part = h->cg_q_part; q.cg_done = done;
      launch_gemv_n(1, false, EPN_CG_Q, h->A, h->lda, m, n, h->cg_p, nullptr, g, h->part_n, h->cnt_n, q, h->st, s);
      launch_cg_alpha(h->cg, h->st, h->cg_q_part, g.n_nrowblk, h->x, h->cg_rt, h->cg_rb, h->cg_p, h->cg_q, m, n,
                      h->cg_r_part, h->cg_nblk, s);
      EpiArgs sv = epi0();
      sv.cg_rb = h->cg_rb; sv.cg_s = h->cg_s; sv.res_part = h->cg_s_part; sv.cg_done = done;
      launch_gemv_t(1, false, EPT_CG_S, h->A, h->lda, m, n, h->cg_rt, nullptr, nullptr, g, h->part_t, h->cnt_t, sv,
                    h->st, s);
      launch_cg_beta(h->cg, h->st, h->cg_s_part, g.t_ncolblk, h->cg_r_part, h->cg_nblk, h->cg_p, h->cg_s, n,
                     h->cg_p_part, h->cg_cnt, cg_blocks(n), s);
    }
    launch_cg_tall_finish(n, h->xt, h->cx, h->x, h->st, s);
    // [y, w] = A [x, x^{1/2}] ; y~ += d - y ; primal residual
    EpiArgs e8 = epi0();
    e8.y = h->y; e8.yt = h->yt; e8.dy = h->dy; e8.yh = h->yh; e8.D = h->D; e8.res_part = h->pri_part;
    launch_gemv_n(2, false, EPN_TALL_Y, h->A, h->lda, m, n, h->x, h->xh, g, h->part_n, h->cnt_n, e8, h->st, s);
  } else {
    // primal residual ||A x^{1/2} - y^{1/2}|| (r = A c - d is not needed here)
    EpiArgs e1 = epi0();
    e1.r = h->r; e1.dy = h->dy; e1.yh = h->yh; e1.D = h->D; e1.res_part = h->pri_part;
    launch_gemv_n(2, false, EPN_FAT_R, h->A, h->lda, m, n, h->cx, h->xh, g, h->part_n, h->cnt_n, e1, h->st, s);
    // r_top = c - A^T z0 ; r_bot = -d - z0, s = A r_top + r_bot, p = s
    EpiArgs a = epi0();
    a.cg_top = h->cx; a.cg_rt = h->cg_rt; a.res_part = h->cg_r0_part;
    launch_gemv_t(1, false, EPT_CG_R, h->A, h->lda, m, n, h->cg_z, nullptr, nullptr, g, h->part_t, h->cnt_t, a,
                  h->st, s);
    EpiArgs b = epi0();
    b.cg_bot = h->dy; b.cg_sign = -1.0f; b.cg_u = h->cg_z; b.cg_rb = h->cg_rb; b.cg_s = h->cg_s; b.cg_p = h->cg_p;
    b.res_part = h->cg_s0_part;
    launch_gemv_n(1, false, EPN_CG_S0, h->A, h->lda, m, n, h->cg_rt, nullptr, g, h->part_n, h->cnt_n, b, h->st, s);
    launch_cg_start(h->cg, h->st, h->cg_r0_part, g.t_ncolblk, h->cg_s0_part, g.n_nrowblk, s);
    for (int k = 0; k < steps; ++k) {
      EpiArgs q = epi0();
      q.out1 = h->cg_q; q.res_part = h->cg_q_part; q.cg_done = done;
      launch_gemv_t(1, false, EPT_CG_Q, h->A, h->lda, m, n, h->cg_p, nullptr, nullptr, g, h->part_t, h->cnt_t, q,
                    h->st, s);
      launch_cg_alpha(h->cg, h->st, h->cg_q_part, g.t_ncolblk, h->cg_z, h->cg_rt, h->cg_rb, h->cg_p, h->cg_q, n, m,
                      h->cg_r_part, h->cg_nblk, s);
      EpiArgs sv = epi0();
      sv.cg_rb = h->cg_rb; sv.cg_s = h->cg_s; sv.res_part = h->cg_s_part; sv.cg_done = done;
      launch_gemv_n(1, false, EPN_CG_S, h->A, h->lda, m, n, h->cg_rt, nullptr, g, h->part_n, h->cnt_n, sv, h->st, s);
      launch_cg_beta(h->cg, h->st, h->cg_s_part, g.n_nrowblk, h->cg_r_part, h->cg_nblk, h->cg_p, h->cg_s, m,
                     h->cg_p_part, h->cg_cnt, cg_blocks(m), s);
    }
    launch_cg_fat_finish(m, h->dy, h->cg_z, h->y, h->w, h->yt, h->st, s);
    // x = c + A^T (d - y) ; x~ = -A^T y~ ; dual residual
    EpiArgs e8 = epi0();
    e8.x = h->x; e8.xt = h->xt; e8.cx = h->cx; e8.mu = h->mu; e8.E = h->E; e8.res_part = h->dual_part;
    launch_gemv_t(3, false, EPT_FAT_X, h->A, h->lda, m, n, h->w, h->nu, h->yt, g, h->part_t, h->cnt_t, e8, h->st, s);
  }
}

// (I + G)^{-1} v with the given final epilogue: one symmetric pass over S, or z = M v then M^T z.
void apply_inverse(pogs_handle* h, const float* v, int epi, const EpiArgs& ep, cudaStream_t s) {
  const int q = (int)h->q;
  if (h->ldl) {   // sparse LDL^T of K: (I + A^T A)^{-1} v or (I + A A^T)^{-1} v
    ldl_apply(*h->ldl, h->tall, v, epi, ep, s);
    return;
  }
  if (h->St) {
    launch_symv(epi, h->St, h->T, q, v, h->part_sy, h->cnt_tr, ep, h->st, s);
    return;
  }
  EpiArgs e = epi0();
  e.out1 = h->z;
  launch_trmv(false, EPR_RAW, h->Mt, h->T, q, v, h->part_tr, h->cnt_tr, e, h->st, s);
  launch_trmv(true, epi, h->Mt, h->T, q, h->z, h->part_tr, h->cnt_tr, ep, h->st, s);
}

// The projection of one iteration (tall or fat), optionally with refinement.
void enqueue_projection(pogs_handle* h, int refine, int cg_steps, cudaStream_t s) {
  if (cg_steps > 0 || h->indirect) {
    enqueue_projection_cgls(h, cg_steps, s);
    return;
  }
  const int m = (int)h->m, n = (int)h->n, q = (int)h->q;
  const GemvGeom& g = h->geom;
  if (h->tall) {
    // r = c + A^T d ; dual residual ||A^T nu + mu||
    EpiArgs e1 = epi0();
    e1.r = h->r; e1.cx = h->cx; e1.mu = h->mu; e1.E = h->E; e1.xt = h->xt; e1.res_part = h->dual_part;
    launch_gemv_t(3, false, EPT_TALL_R, h->A, h->lda, m, n, h->dy, h->nu, h->yt, g, h->part_t, h->cnt_t, e1, h->st, s);
    EpiArgs e3 = epi0();
    if (!refine) {
      e3.x = h->x; e3.xt = h->xt; e3.cx = h->cx;
      apply_inverse(h, h->r, EPR_TALL_X, e3, s);
    } else {
      e3.out1 = h->x;   // x0 only; the dual update waits for the refined x
      apply_inverse(h, h->r, EPR_RAW, e3, s);
    }
    if (refine) {
      // r2 = r - x0 - A^T (A x0);  x = x0 + L^{-T} L^{-1} r2
      EpiArgs e4 = epi0();
      e4.out1 = h->v0;
      launch_gemv_n(1, false, EPN_RAW, h->A, h->lda, m, n, h->x, nullptr, g, h->part_n, h->cnt_n, e4, h->st, s);
      EpiArgs e5 = epi0();
      e5.out1 = h->r2; e5.in1 = h->r; e5.in2 = h->x;
      launch_gemv_t(1, false, EPT_REFINE, h->A, h->lda, m, n, h->v0, nullptr, nullptr, g, h->part_t, h->cnt_t, e5,
                    h->st, s);
      EpiArgs e7 = epi0();
      e7.x = h->x; e7.xt = h->xt; e7.cx = h->cx; e7.in1 = h->x;
      apply_inverse(h, h->r2, EPR_TALL_X, e7, s);
    }
    // [y, w] = A [x, x^{1/2}] ; y~ = d - y ; primal residual ||A x^{1/2} - y^{1/2}||
    EpiArgs e8 = epi0();
    e8.y = h->y; e8.yt = h->yt; e8.dy = h->dy; e8.yh = h->yh; e8.D = h->D; e8.res_part = h->pri_part;
    launch_gemv_n(2, false, EPN_TALL_Y, h->A, h->lda, m, n, h->x, h->xh, g, h->part_n, h->cnt_n, e8, h->st, s);
  } else {
    // r = A c - d ; primal residual
    EpiArgs e1 = epi0();
    e1.r = h->r; e1.dy = h->dy; e1.yh = h->yh; e1.D = h->D; e1.res_part = h->pri_part;
    launch_gemv_n(2, false, EPN_FAT_R, h->A, h->lda, m, n, h->cx, h->xh, g, h->part_n, h->cnt_n, e1, h->st, s);
    if (!refine) {
      EpiArgs e3 = epi0();
      e3.y = h->y; e3.yt = h->yt; e3.dy = h->dy; e3.w = h->w;
      apply_inverse(h, h->r, EPR_FAT_Y, e3, s);
    } else {
      EpiArgs e3 = epi0();
      e3.out1 = h->v0;
      apply_inverse(h, h->r, EPR_RAW, e3, s);
      // r2 = r - v0 - A (A^T v0)
      EpiArgs e4 = epi0();
      e4.out1 = h->tn;
      launch_gemv_t(1, false, EPT_RAW, h->A, h->lda, m, n, h->v0, nullptr, nullptr, g, h->part_t, h->cnt_t, e4,
                    h->st, s);
      EpiArgs e5 = epi0();
      e5.out1 = h->r2; e5.in1 = h->r; e5.in2 = h->v0;
      launch_gemv_n(1, false, EPN_REFINE, h->A, h->lda, m, n, h->tn, nullptr, g, h->part_n, h->cnt_n, e5, h->st, s);
      EpiArgs e7 = epi0();
      e7.y = h->y; e7.yt = h->yt; e7.dy = h->dy; e7.w = h->w; e7.in1 = h->v0;
      apply_inverse(h, h->r2, EPR_FAT_Y, e7, s);
    }
    // x = c + A^T (d - y) ; x~ = c - x ; dual residual
    EpiArgs e8 = epi0();
    e8.x = h->x; e8.xt = h->xt; e8.cx = h->cx; e8.mu = h->mu; e8.E = h->E; e8.res_part = h->dual_part;
    launch_gemv_t(3, false, EPT_FAT_X, h->A, h->lda, m, n, h->w, h->nu, h->yt, g, h->part_t, h->cnt_t, e8, h->st, s);
  }
}

// The passes read the leading GemvGeom::keep_rows rows of A^ evict-last; an entry point that ran
// passes hands those lines back to normal L2 priority before it returns.
void release_kept_rows(pogs_handle* h, cudaStream_t s) {
  if (!h->sparse && h->A && h->geom.keep_rows > 0)
    launch_l2_release(h->A, (size_t)h->geom.keep_rows * h->lda * sizeof(float), s);
}

void enqueue_iteration(pogs_handle* h, int refine, int cg_steps, cudaStream_t s, unsigned long long cond,
                       int use_cond) {
  launch_prox_step((int)h->n, (int)h->m, h->x, h->xt, h->xh, h->cx, h->mu, h->y, h->yt, h->yh, h->dy, h->nu,
                   fn_g(h), fn_f(h), h->st, h->cfg, h->prox_part, h->nprox, s);
  enqueue_projection(h, refine, cg_steps, s);
  launch_check(h->st, h->cfg, h->prox_part, h->nprox, h->pri_part, h->geom.n_nrowblk, h->dual_part,
               h->geom.t_ncolblk, cond, use_cond, s);
}

int kernels_per_iteration(const pogs_handle* h, int refine, int cg_steps) {
  // sparse A: the two main passes may interleave their right-hand sides first
  const int pk = csr_pack_launches(h->geom, (int)h->m, (int)h->n);
  if (cg_steps > 0 || h->indirect)   // prox, 2 passes, CGLS init (3), 4 per step, finish, check
    return 8 + 4 * cg_steps + pk;
  // prox, 2 A passes, check, the inverse (one symmetric or two triangular products) (+ refinement:
  // 2 passes and the inverse again)
  const int inv = h->ldl ? ldl_launches(*h->ldl) : h->St ? 1 : 2;
  // a split column-sum pass is two launches (the main pass, and the refinement's)
  const int cs = colsum_split(h->geom, h->tall ? EPT_TALL_R : EPT_FAT_X) ? 1 : 0;
  return 4 + inv + (refine ? 2 + inv : 0) + pk + cs * (refine ? 2 : 1);
}

int build_graph(pogs_handle* h, int refine, int mode, int cg_steps) {
  if (h->gexec && h->graph_refine == refine && h->graph_mode == mode && h->graph_cg == cg_steps) return 0;
  if (h->gexec) {
    cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
  }
  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0));
  if (mode == 0) {
    cudaGraphConditionalHandle ch;
    CK(cudaGraphConditionalHandleCreate(&ch, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = ch;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    CK(cudaStreamBeginCaptureToGraph(h->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    ++g_capture_depth;
    enqueue_iteration(h, refine, cg_steps, h->cap, (unsigned long long)ch, 1);
    --g_capture_depth;
    cudaGraph_t captured = nullptr;
    CK(cudaStreamEndCapture(h->cap, &captured));
  } else {
    CK(cudaStreamBeginCaptureToGraph(h->cap, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    ++g_capture_depth;
    enqueue_iteration(h, refine, cg_steps, h->cap, 0ull, 0);
    --g_capture_depth;
    cudaGraph_t captured = nullptr;
    CK(cudaStreamEndCapture(h->cap, &captured));
  }
  CK(cudaGraphInstantiate(&h->gexec, g, 0));
  cudaGraphDestroy(g);
  h->graph_refine = refine;
  h->graph_mode = mode;
  h->graph_cg = cg_steps;
  return 0;
}

int validate_params(const pogs_params* p) {
  if (!p) return POGS_ERR_ARG;
  if (!(p->abs_tol >= 0) || !(p->rel_tol >= 0) || p->max_iter < 1 || !(p->rho0 > 0) || !(p->alpha > 0) ||
      !(p->alpha < 2) || !(p->delta >= 1) || !(p->tau > 0) || p->sk_sweeps < 0 || p->refine_steps < 0 ||
      p->refine_steps > 1 || p->gram_prec < POGS_GRAM_BF16 || p->gram_prec > POGS_GRAM_FP32 ||
      p->loop_mode < 0 || p->loop_mode > 1 || p->chol_prec < POGS_CHOL_FP64 || p->chol_prec > POGS_CHOL_MIXED ||
      p->proj_mode < POGS_PROJ_DIRECT || p->proj_mode > POGS_PROJ_LDL || p->cg_max_iter < 0 ||
      p->cg_max_iter > 1000 || !(p->cg_tol >= 0))
    return POGS_ERR_ARG;
  return 0;
}

// Sparse input of pogs_setup_csr (host or device arrays).
struct CsrIn {
  const int *rp, *ci;
  const float* va;
};

template <class T>
int copy_in_array(T* dst, const T* src, int64_t count, cudaStream_t s) {
  if (count <= 0) return 0;
  CK(cudaMemcpyAsync(dst, src, (size_t)count * sizeof(T),
                     is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  return 0;
}

int setup_impl(pogs_handle* h, const float* A, int64_t lds, char order, const CsrIn* csr) {
  const int64_t m = h->m, n = h->n, q = h->q;
  cudaStream_t s = h->stream;
  Scratch scr;
  // phase boundaries are CUDA events on the setup stream (no host synchronisation)
  int nphase = 0;
  CK(cudaEventRecord(h->ev[nphase++], s));
  auto phase = [&](const char* name) {
    (void)name;
    if (nphase < 6) cudaEventRecord(h->ev[nphase++], s);
  };
  // ---- ingest -------------------------------------------------------------------------
  int* err = &h->st->err;
  const bool colmajor = (order == 'C' || order == 'c');
  if (csr) {
    const int64_t nnz = h->nnz;
    TRY(dalloc(h, &h->csr_rp, (size_t)(m + 1)));
    TRY(dalloc(h, &h->csr_ci, (size_t)nnz));
    TRY(dalloc(h, &h->csr_va, (size_t)nnz));
    TRY(copy_in_array(h->csr_rp, csr->rp, m + 1, s));
    TRY(copy_in_array(h->csr_ci, csr->ci, nnz, s));
    TRY(copy_in_array(h->csr_va, csr->va, nnz, s));
    launch_csr_check(h->csr_rp, h->csr_ci, h->csr_va, m, n, nnz, err, s);
  } else if (is_device_ptr(A)) {
    TRY(dalloc(h, &h->A, (size_t)(m * h->lda)));
    launch_copy_in(A, m, n, lds, colmajor, h->A, h->lda, err, s);
  } else {
    TRY(dalloc(h, &h->A, (size_t)(m * h->lda)));
    const int64_t rows = colmajor ? n : m, cols = colmajor ? m : n;
    if (!colmajor && lds == n) {
      // contiguous host rows straight into the padded layout
      CK(cudaMemcpy2DAsync(h->A, h->lda * sizeof(float), A, lds * sizeof(float), n * sizeof(float), m,
                           cudaMemcpyHostToDevice, s));
      launch_copy_in(h->A, m, n, h->lda, false, h->A, h->lda, err, s);
    } else {
      float* stage = nullptr;
      TRY(scr.get(&stage, (size_t)(rows * lds), s));
      (void)cols;
      CK(cudaMemcpyAsync(stage, A, (size_t)(rows * lds) * sizeof(float), cudaMemcpyHostToDevice, s));
      launch_copy_in(stage, m, n, lds, colmajor, h->A, h->lda, err, s);
    }
  }
  CK(cudaGetLastError());
  phase("ingest");
  {
    // a non-finite matrix ends setup here (one stream sync; nothing after depends on it)
    int err_host = 0;
    CK(cudaMemcpyAsync(&err_host, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (err_host != 0) return err_host;
  }
  if (csr) {
    // CSR of A^T by a stable multi-split (entries of each column in increasing row order)
    const int64_t nnz = h->nnz;
    TRY(dalloc(h, &h->csc_rp, (size_t)(n + 1)));
    TRY(dalloc(h, &h->csc_ci, (size_t)nnz));
    TRY(dalloc(h, &h->csc_va, (size_t)nnz));
    TRY(dalloc(h, &h->csc_perm, (size_t)nnz));
    const int nch = csr_transpose_chunks(nnz, n);
    int *rowidx = nullptr, *cnt = nullptr, *tot = nullptr;
    TRY(scr.get(&rowidx, (size_t)nnz, s));
    TRY(scr.get(&cnt, (size_t)nch * (size_t)n, s));
    TRY(scr.get(&tot, (size_t)n, s));
    launch_csr_transpose(h->csr_rp, h->csr_ci, h->csr_va, m, n, nnz, nch, rowidx, cnt, tot, h->csc_rp, h->csc_ci,
                         h->csc_va, h->csc_perm, s);
    GemvGeom& g = h->geom;
    TRY(dalloc(h, &g.pack, (size_t)std::max(h->mv, h->nv) * 4));
    g.rp_n = h->csr_rp; g.ci_n = h->csr_ci; g.va_n = h->csr_va;
    g.rp_t = h->csc_rp; g.ci_t = h->csc_ci; g.va_t = h->csc_va;
    CK(cudaGetLastError());
  }
  // ---- Algorithm 2 + rescale ----------------------------------------------------------
  float *dvec = nullptr, *evec = nullptr;
  TRY(scr.get(&dvec, (size_t)h->mv, s));
  TRY(scr.get(&evec, (size_t)h->nv, s));
  launch_fill(evec, n, 1.0f, s);
  launch_fill(dvec, m, 1.0f, s);
  const double gamma = h->sp.gamma > 0 ? h->sp.gamma : (double)(m + n) * sqrt(1.1920928955078125e-07);
  const int sweeps = h->sp.equil ? h->sp.sk_sweeps : 0;
  // dense A with rows of at most 12288 floats and enough of them: each sweep in one pass
  const bool fused = !csr && sweeps > 0 && sk_sweep_fits(m, h->lda);
  float* skpart = nullptr;
  Df* skfrob = nullptr;
  if (fused) {
    TRY(scr.get(&skpart, (size_t)sk_sweep_blocks() * h->lda, s));
    TRY(scr.get(&skfrob, (size_t)sk_sweep_finish_blocks(h->lda) * 2, s));
  }
  for (int it = 0; fused && it < sweeps; ++it)
    TRY(launch_sk_sweep(h->A, h->lda, m, n, dvec, evec, gamma, skpart, skfrob, s));
  for (int it = 0; !fused && it < sweeps; ++it) {
    EpiArgs er = epi0();
    er.sk_vec = dvec; er.sk_num = (float)n; er.sk_reg = (float)(gamma / (double)m);
    launch_gemv_n(1, true, EPN_SK_ROW, h->A, h->lda, (int)m, (int)n, evec, nullptr, h->geom, h->part_n, h->cnt_n,
                  er, nullptr, s);
    EpiArgs ec = epi0();
    ec.sk_vec = evec; ec.sk_num = (float)m; ec.sk_reg = (float)(gamma / (double)n); ec.res_part = h->dual_part;
    launch_gemv_t(1, true, EPT_SK_COL, h->A, h->lda, (int)m, (int)n, dvec, nullptr, nullptr, h->geom, h->part_t,
                  h->cnt_t,
                  ec, nullptr, s);
  }
  if (sweeps == 0) {
    // D = E = I: only the Frobenius norm is needed (sk_num < 0 keeps e = 1)
    EpiArgs ec = epi0();
    ec.sk_vec = evec; ec.sk_num = -1.0f; ec.res_part = h->dual_part;
    launch_gemv_t(1, true, EPT_SK_COL, h->A, h->lda, (int)m, (int)n, dvec, nullptr, nullptr, h->geom, h->part_t,
                  h->cnt_t,
                  ec, nullptr, s);
  }
  launch_sk_finish(dvec, evec, m, n, fused ? skfrob : h->dual_part, fused ? sk_sweep_finish_blocks(h->lda) : h->geom.t_ncolblk, q, h->D, h->E, s);
  if (csr) launch_csr_scale(h->csr_rp, h->csr_ci, h->csr_va, m, h->D, h->E, h->csc_perm, h->nnz, h->csc_va, s);
  else launch_scale(h->A, h->lda, m, n, h->D, h->E, s);
  CK(cudaGetLastError());
  phase("equil");
  if (h->sp.proj_mode == POGS_PROJ_LDL) {
    // sparse direct projection: symbolic analysis of K on the host, numeric LDL^T on the device
    if (!csr) return POGS_ERR_ARG;
    std::vector<int> hrp(m + 1), hci(std::max<int64_t>(1, h->nnz));
    CK(cudaMemcpyAsync(hrp.data(), h->csr_rp, sizeof(int) * (m + 1), cudaMemcpyDeviceToHost, s));
    if (h->nnz > 0) CK(cudaMemcpyAsync(hci.data(), h->csr_ci, sizeof(int) * h->nnz, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    LdlSymbolic S;
    TRY(ldl_analyze((int)m, (int)n, hrp.data(), hci.data(), S));
    phase("gram");
    h->ldl = new (std::nothrow) LdlFactor();
    if (!h->ldl) return POGS_ERR_OOM;
    TRY(ldl_factor(S, h->csr_va, *h->ldl, err, s));
    h->device_bytes += h->ldl->device_bytes;
    CK(cudaGetLastError());
    phase("cholesky");
    phase("inverse");
    CK(cudaStreamSynchronize(s));
    return 0;
  }
  if (h->sp.proj_mode == POGS_PROJ_CGLS) {
    // indirect projection: no Gram, no factorization (the phases are recorded empty)
    h->indirect = true;
    phase("gram");
    phase("cholesky");
    phase("inverse");
    release_kept_rows(h, s);
    CK(cudaStreamSynchronize(s));
    return 0;
  }
  // ---- Gram -----------------------------------------------------------------------------
  // square work matrices share one 128-byte-aligned pitch (vector loads in the factorization)
  const int64_t ldq = round_up(q, 32);
  float* G = nullptr;
  TRY(scr.get(&G, (size_t)(ldq * ldq), s));
  // sparse A: the Gram of the reduced update is formed from a temporary dense copy of A^
  // (for A with scattered nonzeros A^T A is dense anyway); the iterations use the CSR passes
  float* dense = nullptr;
  if (csr) {
    void* q0 = nullptr;
    TRY(pool_alloc(&q0, (size_t)(m * h->lda) * sizeof(float), s));
    dense = static_cast<float*>(q0);
    if (cudaMemsetAsync(dense, 0, (size_t)(m * h->lda) * sizeof(float), s) != cudaSuccess) {
      cudaFreeAsync(dense, s);
      return POGS_ERR_CUDA;
    }
    launch_csr_densify(h->csr_rp, h->csr_ci, h->csr_va, m, dense, h->lda, s);
    h->A = dense;
  }
  struct DenseRelease {
    pogs_handle* h;
    float* p;
    cudaStream_t s;
    ~DenseRelease() {
      if (p) {
        cudaFreeAsync(p, s);
        h->A = nullptr;
      }
    }
  } dense_release{h, dense, s};
  int used = -1;
  if (h->sp.gram_prec != POGS_GRAM_FP32) {
    size_t need = 0;
    int rc = gram_tensor(h->sp.gram_prec, h->A, h->lda, m, n, h->tall, G, ldq, nullptr, 0, &need, err, s);
    if (rc == 0 && need > 0) {
      void* ws = nullptr;
      char* wsc = nullptr;
      TRY(scr.get(&wsc, need, s));
      ws = wsc;
      rc = gram_tensor(h->sp.gram_prec, h->A, h->lda, m, n, h->tall, G, ldq, ws, need, &need, err, s);
      if (rc == 0) used = h->sp.gram_prec;
    }
  }
  if (used < 0) {
    if (h->tall) gemm_f32(true, false, q, q, m, 1.0f, h->A, h->lda, h->A, h->lda, 0.0f, G, ldq, true, s);
    else gemm_f32(false, true, q, q, n, 1.0f, h->A, h->lda, h->A, h->lda, 0.0f, G, ldq, true, s);
    used = POGS_GRAM_FP32;
  }
  h->gram_used = used;
  CK(cudaGetLastError());
  if (dense) {
    cudaFreeAsync(dense, s);
    h->A = nullptr;
    dense_release.p = nullptr;
  }
  phase("gram");
  // ---- Cholesky of I + G -------------------------------------------------------------------
  float *Md = nullptr, *Lf = nullptr;
  TRY(scr.get(&Md, (size_t)(ldq * ldq), s));
  TRY(scr.get(&Lf, (size_t)(ldq * ldq), s));
  float* wk = nullptr;
  TRY(scr.get(&wk, (size_t)(q * (q / 2 + kTile)), s));
  // from q = 4096 on the mixed factorization runs recursively with the inverse formed alongside,
  // its large products on the tensor cores; below that the blocked factorization, whose
  // 128-block leaves overlap its trailing updates, is faster (q = 2000: 2.6 against 2.9 ms)
  const bool recursive = h->sp.chol_prec == POGS_CHOL_MIXED && q >= 4096;
  if (recursive) {
    float* Hlo = nullptr;
    TRY(scr.get(&Hlo, (size_t)(ldq * ldq), s));
    TRY(chol_inv_mixed(G, Hlo, ldq, q, Lf, ldq, Md, ldq, wk, err, s));
  } else if (h->sp.chol_prec == POGS_CHOL_MIXED) {
    // double-float Schur complement (G becomes its hi part); also writes the diagonal blocks of M
    float* Hlo = nullptr;
    TRY(scr.get(&Hlo, (size_t)(ldq * ldq), s));
    TRY(chol_mixed(G, Hlo, ldq, q, Lf, ldq, Md, ldq, err, s));
  } else {
    double* H = nullptr;
    TRY(scr.get(&H, (size_t)(ldq * ldq), s));
    launch_gram_to_f64(G, ldq, q, H, ldq, s);
    double* work = nullptr;
    TRY(scr.get(&work, 64 * 64, s));
    chol_f64(H, ldq, q, work, err, s);
    launch_leaf_inverse(H, ldq, q, Md, ldq, s);
    launch_l_to_f32(H, ldq, q, Lf, ldq, s);
  }
  CK(cudaGetLastError());
  phase("cholesky");
  // ---- M = L^{-1} (FP32; already complete after the recursive factorization), packed tiles --
  if (!recursive) TRY(tri_inverse_f32(Lf, ldq, q, Md, ldq, wk, h->sp.chol_prec == POGS_CHOL_MIXED, err, s));
  if (h->sp.chol_prec == POGS_CHOL_MIXED && q >= 1024) {
    // S = M^T M = (I + G)^{-1}, lower tiles on the tensor cores (TF32x3); each iteration then
    // applies it in one pass over its packed triangle instead of M and M^T in two.  From q = 1024
    // on, where the inverse's own products are TF32x3 already; below, M v and M^T z in FP32 keep
    // the iterates closest to the FP64 trajectory and cost little.
    float* S = nullptr;
    TRY(scr.get(&S, (size_t)(ldq * ldq), s));
    size_t need = 0;
    // X = Y = M^T, zero for k < i (M lower triangular): each tile skips the K boxes before its rows
    if (tc_gemm_tf32x3(q, q, q, Md, ldq, true, Md, ldq, true, 1.0f, S, nullptr, ldq, TC_EPI_STORE, true, nullptr, 0,
                       &need, err, s, true) == 0) {
      char* ws = nullptr;
      TRY(scr.get(&ws, need, s));
      if (tc_gemm_tf32x3(q, q, q, Md, ldq, true, Md, ldq, true, 1.0f, S, nullptr, ldq, TC_EPI_STORE, true, ws, need,
                         nullptr, err, s, true) == 0) {
        TRY(dalloc(h, &h->St, (size_t)h->T * (h->T + 1) / 2 * kTile * kTile));
        TRY(dalloc(h, &h->part_sy, (size_t)h->T * h->T * kTile));
        launch_pack_tiles(S, ldq, q, h->T, h->St, s, true);
      }
    }
  }
  if (!h->St) {
    TRY(dalloc(h, &h->Mt, (size_t)h->T * (h->T + 1) / 2 * kTile * kTile));
    launch_pack_tiles(Md, ldq, q, h->T, h->Mt, s);
  }
  CK(cudaGetLastError());
  phase("inverse");
  release_kept_rows(h, s);
  CK(cudaStreamSynchronize(s));
  return 0;
}

int alloc_state(pogs_handle* h) {
  const size_t nv = (size_t)h->nv, mv = (size_t)h->mv;
  float** nvecs[] = {&h->x, &h->xt, &h->xh, &h->cx, &h->mu, &h->ox, &h->omu, &h->tn, &h->ga, &h->gb, &h->gc, &h->gd, &h->ge};
  for (auto p : nvecs) TRY(dalloc(h, p, nv));
  float** mvecs[] = {&h->y, &h->yt, &h->yh, &h->dy, &h->nu, &h->w, &h->oy, &h->onu, &h->fa, &h->fb, &h->fc, &h->fd, &h->fe};
  for (auto p : mvecs) TRY(dalloc(h, p, mv));
  // projection work vectors hold q-, m- or n-length data (tall refinement writes A x0 into v0):
  // max(nv, mv) covers m, lda and T*128 in both orientations
  const size_t qv = nv > mv ? nv : mv;
  float** qvecs[] = {&h->r, &h->z, &h->x0, &h->v0, &h->r2};
  for (auto p : qvecs) TRY(dalloc(h, p, qv));
  const size_t kmax = nv > mv ? nv : mv;
  float** rvecs[] = {&h->ra, &h->rb, &h->rc, &h->rd, &h->re};
  for (auto p : rvecs) TRY(dalloc(h, p, kmax));
  TRY(dalloc(h, &h->rh, kmax));
  TRY(dalloc(h, &h->fh, mv));
  TRY(dalloc(h, &h->gh, nv));
  TRY(dalloc(h, &h->D, mv));
  TRY(dalloc(h, &h->E, nv));
  const GemvGeom& g = h->geom;
  TRY(dalloc(h, &h->part_t, (size_t)g.t_nsplit * 3 * h->lda));
  TRY(dalloc(h, &h->cnt_t, (size_t)g.t_ncolblk));
  TRY(dalloc(h, &h->part_n, (size_t)g.n_ncolsplit * 2 * h->m));
  TRY(dalloc(h, &h->cnt_n, (size_t)g.n_nrowblk));
  TRY(dalloc(h, &h->part_tr, (size_t)h->T * (h->T + 1) / 2 * kTile));
  TRY(dalloc(h, &h->cnt_tr, (size_t)h->T));
  TRY(dalloc(h, &h->prox_part, (size_t)h->nprox * 6));
  TRY(dalloc(h, &h->pri_part, (size_t)g.n_nrowblk * 2));
  TRY(dalloc(h, &h->dual_part, (size_t)g.t_ncolblk * 2));
  {
    float** cgv[] = {&h->cg_rt, &h->cg_rb, &h->cg_s, &h->cg_p, &h->cg_q, &h->cg_z};
    for (auto p : cgv) TRY(dalloc(h, p, qv));
    const size_t np = (size_t)std::max(g.n_nrowblk, g.t_ncolblk) * 2;
    Df** cgp[] = {&h->cg_r0_part, &h->cg_s0_part, &h->cg_q_part, &h->cg_s_part};
    for (auto p : cgp) TRY(dalloc(h, p, np));
    h->cg_nblk = cg_blocks(std::max(h->mv, h->nv));
    TRY(dalloc(h, &h->cg_r_part, (size_t)h->cg_nblk * 2));
    TRY(dalloc(h, &h->cg_p_part, (size_t)h->cg_nblk * 2));
    TRY(dalloc(h, &h->cg_cnt, 1));
    TRY(dalloc(h, &h->cg, 1));
  }
  TRY(dalloc(h, &h->st, 1));
  TRY(dalloc(h, &h->cfg, 1));
  void* pin = pin_slot_get();
  if (!pin) return POGS_ERR_OOM;
  h->st_host = static_cast<DevState*>(pin);
  h->cfg_host = reinterpret_cast<DevCfg*>(static_cast<char*>(pin) + sizeof(DevState));
  h->cg_host = reinterpret_cast<CgState*>(static_cast<char*>(pin) + ((sizeof(DevState) + sizeof(DevCfg) + 15) & ~size_t(15)));
  return 0;
}

void release(pogs_handle* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  for (void* p : h->allocs) cudaFreeAsync(p, h->stream);
  if (h->ldl) {
    h->ldl->release(h->stream);
    delete h->ldl;
  }
  pin_slot_put(h->st_host);
  if (h->cap) cudaStreamDestroy(h->cap);
  for (cudaEvent_t e : h->ev)
    if (e) cudaEventDestroy(e);
  delete h;
}

// Copy a host or device source array into a device array (or return the device pointer).
template <class T>
int stage_in(const T* src, T* staging, int64_t k, cudaStream_t s, const T** out) {
  if (!src) {
    *out = nullptr;
    return 0;
  }
  if (is_device_ptr(src)) {
    *out = src;
    return 0;
  }
  CK(cudaMemcpyAsync(staging, src, (size_t)k * sizeof(T), cudaMemcpyHostToDevice, s));
  *out = staging;
  return 0;
}

int upload_fn(pogs_handle* h, const pogs_fn* fn, int64_t k, int is_f) {
  cudaStream_t s = h->stream;
  if (!fn || !fn->h) return POGS_ERR_ARG;
  FnDev raw{};
  TRY(stage_in(fn->h, h->rh, k, s, &raw.h));
  TRY(stage_in(fn->a, h->ra, k, s, &raw.a));
  TRY(stage_in(fn->b, h->rb, k, s, &raw.b));
  TRY(stage_in(fn->c, h->rc, k, s, &raw.c));
  TRY(stage_in(fn->d, h->rd, k, s, &raw.d));
  TRY(stage_in(fn->e, h->re, k, s, &raw.e));
  if (is_f) launch_fold(raw, k, h->D, 1, h->fh, h->fa, h->fb, h->fc, h->fd, h->fe, &h->st->err, s);
  else launch_fold(raw, k, h->E, 0, h->gh, h->ga, h->gb, h->gc, h->gd, h->ge, &h->st->err, s);
  CK(cudaGetLastError());
  return 0;
}

int reset_state(pogs_handle* h, const pogs_params* p) {
  cudaStream_t s = h->stream;
  // serialise against the previous use of the pinned staging
  CK(cudaStreamSynchronize(s));
  DevState init;
  memset(&init, 0, sizeof(init));
  init.rho = p->rho0;
  init.pend = 1.0;
  init.status = POGS_MAX_ITER;
  *h->st_host = init;
  DevCfg c;
  memset(&c, 0, sizeof(c));
  c.abs_tol = p->abs_tol; c.rel_tol = p->rel_tol; c.alpha = p->alpha; c.delta = p->delta; c.tau = p->tau;
  c.inv_delta = 1.0 / p->delta;
  c.max_iter = p->max_iter; c.gap_stop = p->gap_stop; c.adaptive = p->adaptive_rho;
  *h->cfg_host = c;
  CK(cudaMemcpyAsync(h->st, h->st_host, sizeof(DevState), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(h->cfg, h->cfg_host, sizeof(DevCfg), cudaMemcpyHostToDevice, s));
  {
    CgState cg;
    memset(&cg, 0, sizeof(cg));
    cg.max_steps = cg_steps_for(h, p);
    cg.tol = (float)p->cg_tol;
    *h->cg_host = cg;
    CK(cudaMemcpyAsync(h->cg, h->cg_host, sizeof(CgState), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(h->cg_z, 0, std::max(h->nv, h->mv) * sizeof(float), s));   // fat CGLS warm start
  }
  CK(cudaMemsetAsync(h->x, 0, h->nv * sizeof(float), s));
  CK(cudaMemsetAsync(h->xt, 0, h->nv * sizeof(float), s));
  CK(cudaMemsetAsync(h->y, 0, h->mv * sizeof(float), s));
  CK(cudaMemsetAsync(h->yt, 0, h->mv * sizeof(float), s));
  return 0;
}

int copy_out(const float* dsrc, float* dst, int64_t k, cudaStream_t s) {
  if (!dst) return 0;
  CK(cudaMemcpyAsync(dst, dsrc, (size_t)k * sizeof(float), is_device_ptr(dst) ? cudaMemcpyDeviceToDevice
                                                                                  : cudaMemcpyDeviceToHost, s));
  return 0;
}

}  // namespace

extern "C" {

void pogs_default_params(pogs_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->abs_tol = 1e-4;
  p->rel_tol = 1e-3;
  p->max_iter = 10000;
  p->rho0 = 1.0;
  p->alpha = 1.7;
  p->delta = 1.05;
  p->tau = 0.8;
  p->sk_sweeps = 10;
  p->gamma = 0.0;
  p->gram_prec = POGS_GRAM_BF16X3;
  p->refine_steps = 0;
  p->gap_stop = 1;
  p->adaptive_rho = 1;
  p->equil = 1;
  p->verbose = 0;
  p->loop_mode = 0;
  p->check_every = 10;
  p->chol_prec = POGS_CHOL_MIXED;
  p->proj_mode = POGS_PROJ_DIRECT;
  p->cg_max_iter = 30;
  p->cg_tol = 1e-4;
}

}  // extern "C"

// The part of pogs_setup and pogs_setup_csr after argument checks: handle, geometry, state,
// ingest, equilibration and (direct projection) the cached factor.
static int setup_common(const float* A, int64_t m, int64_t n, int64_t lda, char order, const CsrIn* csr,
                        int64_t nnz, const pogs_params* p, void* stream, pogs_handle** out) {
  const double t0 = now_ms();
  pogs_handle* h = new (std::nothrow) pogs_handle();
  if (!h) return POGS_ERR_OOM;
  h->m = m;
  h->n = n;
  h->tall = m >= n;
  h->q = h->tall ? n : m;
  h->lda = round_up(n, kLdaAlign);
  h->T = (int)cdiv(h->q, kTile);
  h->nv = round_up(std::max<int64_t>(h->lda, h->tall ? (int64_t)h->T * kTile : 0), kTile);
  h->mv = round_up(std::max<int64_t>(m, h->tall ? 0 : (int64_t)h->T * kTile), kTile);
  h->sp = *p;
  h->indirect = p->proj_mode == POGS_PROJ_CGLS;
  h->stream = static_cast<cudaStream_t>(stream);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return POGS_ERR_CUDA;
  }
  if (cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return POGS_ERR_CUDA;
  }
  for (cudaEvent_t& e : h->ev) {
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      release(h);
      return POGS_ERR_CUDA;
    }
  }
  h->sparse = csr != nullptr;
  h->nnz = nnz;
  if (h->sparse) csr_geometry(h->geom, m, n, nnz, h->num_sms);
  else h->geom = choose_geometry(m, n, h->lda, h->num_sms);
  h->nprox = (int)std::min<int64_t>(cdiv(m + n, 256), (int64_t)h->num_sms * 4);
  int rc = alloc_state(h);
  if (rc == 0) rc = setup_impl(h, A, lda, order, csr);
  if (rc == 0) {
    if (cudaMemcpyAsync(h->st_host, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
      rc = POGS_ERR_CUDA;
    else if (h->st_host->err != 0) rc = h->st_host->err;
  }
  if (rc != 0) {
    release(h);
    return rc;
  }
  h->setup_ms = now_ms() - t0;
  for (int k = 0; k < 5; ++k) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, h->ev[k], h->ev[k + 1]) != cudaSuccess) {
      cudaGetLastError();
      ms = -1.0f;
    }
    h->phase_ms[k] = ms;
  }
  *out = h;
  return 0;
}


extern "C" {

int pogs_setup(const float* A, int64_t m, int64_t n, int64_t lda, char order, const pogs_params* p, void* stream,
               pogs_handle** out) {
  if (!out) return POGS_ERR_ARG;
  *out = nullptr;
  if (!A || m < 1 || n < 1 || m > (1ll << 31) - 1 || n > (1ll << 31) - 1) return POGS_ERR_ARG;
  const bool colmajor = (order == 'C' || order == 'c');
  if (!(colmajor || order == 'R' || order == 'r')) return POGS_ERR_ARG;
  if ((!colmajor && lda < n) || (colmajor && lda < m)) return POGS_ERR_ARG;
  pogs_params def;
  pogs_default_params(&def);
  if (!p) p = &def;
  if (validate_params(p) != 0) return POGS_ERR_ARG;
  return setup_common(A, m, n, lda, order, nullptr, 0, p, stream, out);
}

int pogs_setup_csr(int64_t m, int64_t n, int64_t nnz, const int* rowptr, const int* colind, const float* val,
                   const pogs_params* p, void* stream, pogs_handle** out) {
  if (!out) return POGS_ERR_ARG;
  *out = nullptr;
  if (!rowptr || m < 1 || n < 1 || m > (1ll << 31) - 2 || n > (1ll << 31) - 2 || nnz < 0 ||
      nnz > (1ll << 31) - 1 || (nnz > 0 && (!colind || !val)))
    return POGS_ERR_ARG;
  pogs_params def;
  pogs_default_params(&def);
  if (!p) p = &def;
  if (validate_params(p) != 0) return POGS_ERR_ARG;
  const CsrIn in{rowptr, colind, val};
  return setup_common(nullptr, m, n, n, 'R', &in, nnz, p, stream, out);
}

// Warm start (Section 5): the graph point (x^0 / E, A^ x^0 / E) and the scaled duals
// y~ = -(nu^0 / D) / rho^0, x~ = -A^T y~ (Section 3.3 invariant); a part not given stays zero and
// the first prox step estimates it.
int warm_start(pogs_handle* h, const float* x0, const float* nu0, double rho0) {
  cudaStream_t s = h->stream;
  const GemvGeom& g = h->geom;
  const int m = (int)h->m, n = (int)h->n;
  if (x0) {
    const float* src = nullptr;
    TRY(stage_in(x0, h->tn, h->n, s, &src));
    launch_warm(src, h->E, h->n, 1.0f, h->x, nullptr, s);
    EpiArgs e = epi0();
    e.out1 = h->y;
    launch_gemv_n(1, false, EPN_RAW, h->A, h->lda, m, n, h->x, nullptr, g, h->part_n, h->cnt_n, e, nullptr, s);
  }
  if (nu0) {
    const float* src = nullptr;
    TRY(stage_in(nu0, h->oy, h->m, s, &src));
    launch_warm(src, h->D, h->m, (float)(1.0 / rho0), h->w, h->yt, s);
    EpiArgs e = epi0();
    e.out1 = h->xt;
    launch_gemv_t(1, false, EPT_RAW, h->A, h->lda, m, n, h->w, nullptr, nullptr, g, h->part_t, h->cnt_t, e, nullptr,
                  s);
  }
  CK(cudaGetLastError());
  return 0;
}

int pogs_solve_warm(pogs_handle* h, const pogs_fn* f, const pogs_fn* g, const pogs_params* p, const float* x0,
                    const float* nu0, float* x, float* y, float* mu, float* nu, pogs_info* info) {
  if (!h || !f || !g) return POGS_ERR_ARG;
  if (!p) p = &h->sp;
  if (validate_params(p) != 0) return POGS_ERR_ARG;
  const double t0 = now_ms();
  cudaStream_t s = h->stream;
  TRY(reset_state(h, p));
  TRY(upload_fn(h, f, h->m, 1));
  TRY(upload_fn(h, g, h->n, 0));
  if (x0 || nu0) TRY(warm_start(h, x0, nu0, p->rho0));
  const int refine = p->refine_steps;
  const int cg_steps = cg_steps_for(h, p);
  TRY(build_graph(h, refine, p->loop_mode, cg_steps));
  if (p->loop_mode == 0) {
    CK(cudaGraphLaunch(h->gexec, s));
  } else {
    const int every = p->check_every > 0 ? p->check_every : 10;
    int launched = 0;
    while (launched < p->max_iter) {
      for (int i = 0; i < every && launched < p->max_iter; ++i, ++launched) CK(cudaGraphLaunch(h->gexec, s));
      CK(cudaMemcpyAsync(h->st_host, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (h->st_host->done) break;
    }
  }
  release_kept_rows(h, s);
  launch_unscale((int)h->n, (int)h->m, h->xh, h->mu, h->yh, h->nu, h->D, h->E, x ? h->ox : nullptr,
                 mu ? h->omu : nullptr, y ? h->oy : nullptr, nu ? h->onu : nullptr, s);
  CK(cudaGetLastError());
  TRY(copy_out(h->ox, x, h->n, s));
  TRY(copy_out(h->omu, mu, h->n, s));
  TRY(copy_out(h->oy, y, h->m, s));
  TRY(copy_out(h->onu, nu, h->m, s));
  CK(cudaMemcpyAsync(h->st_host, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const DevState& st = *h->st_host;
  count_launch(st.k * kernels_per_iteration(h, refine, cg_steps));
  h->solved = true;
  int status = st.status;
  if (st.err != 0) status = st.err;
  if (info) {
    info->status = status;
    info->iters = st.k;
    info->rho = st.rho;
    info->r_pri = st.r_pri;
    info->r_dual = st.r_dual;
    info->eps_pri = st.eps_pri;
    info->eps_dual = st.eps_dual;
    info->gap = st.gap;
    info->obj = st.obj;
    info->r_pri_unscaled = st.r_pri_u;
    info->r_dual_unscaled = st.r_dual_u;
    info->setup_ms = h->setup_ms;
    info->solve_ms = now_ms() - t0;
  }
  return status;
}

int pogs_solve(pogs_handle* h, const pogs_fn* f, const pogs_fn* g, const pogs_params* p, float* x, float* y,
               float* mu, float* nu, pogs_info* info) {
  return pogs_solve_warm(h, f, g, p, nullptr, nullptr, x, y, mu, nu, info);
}

void pogs_free(pogs_handle* h) { release(h); }

int pogs_prox_eval(const pogs_fn* fn, int64_t k, const float* v, const float* rho_vec, float rho, float* out,
                   void* stream) {
  if (!fn || !fn->h || !v || !out || k < 0) return POGS_ERR_ARG;
  if (k == 0) return 0;
  FnDev d{fn->h, fn->a, fn->b, fn->c, fn->d, fn->e};
  // NULL parameter arrays take their defaults through a temporary filled array
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* tmp = nullptr;
  const bool need = !fn->a || !fn->b || !fn->c || !fn->d || !fn->e;
  if (need) {
    if (pool_alloc(reinterpret_cast<void**>(&tmp), (size_t)k * 2 * sizeof(float), s) != 0) return POGS_ERR_OOM;
    launch_fill(tmp, k, 1.0f, s);
    launch_fill(tmp + k, k, 0.0f, s);
    if (!d.a) d.a = tmp;
    if (!d.c) d.c = tmp;
    if (!d.b) d.b = tmp + k;
    if (!d.d) d.d = tmp + k;
    if (!d.e) d.e = tmp + k;
  }
  launch_prox_eval(d, k, v, rho_vec, rho, out, s);
  cudaError_t e = cudaGetLastError();
  if (tmp) cudaFreeAsync(tmp, s);
  return e == cudaSuccess ? 0 : POGS_ERR_CUDA;
}

int pogs_get_equil(const pogs_handle* h, float* D, float* E) {
  if (!h) return POGS_ERR_ARG;
  TRY(copy_out(h->D, D, h->m, h->stream));
  TRY(copy_out(h->E, E, h->n, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return 0;
}

int pogs_get_ahat(const pogs_handle* h, float* Ahat) {
  if (!h || !Ahat) return POGS_ERR_ARG;
  if (h->sparse) {
    // dense m x n copy of the CSR values
    const size_t bytes = (size_t)(h->m * h->n) * sizeof(float);
    void* q = nullptr;
    TRY(pool_alloc(&q, bytes, h->stream));
    float* tmp = static_cast<float*>(q);
    int rc = 0;
    if (cudaMemsetAsync(tmp, 0, bytes, h->stream) != cudaSuccess) rc = POGS_ERR_CUDA;
    if (rc == 0) {
      launch_csr_densify(h->csr_rp, h->csr_ci, h->csr_va, h->m, tmp, h->n, h->stream);
      if (cudaMemcpyAsync(Ahat, tmp, bytes, is_device_ptr(Ahat) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          h->stream) != cudaSuccess)
        rc = POGS_ERR_CUDA;
    }
    cudaFreeAsync(tmp, h->stream);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return POGS_ERR_CUDA;
    return rc;
  }
  CK(cudaMemcpy2DAsync(Ahat, h->n * sizeof(float), h->A, h->lda * sizeof(float), h->n * sizeof(float), h->m,
                       is_device_ptr(Ahat) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return 0;
}

int pogs_project(pogs_handle* h, const float* c, const float* d, float* x, float* y, const pogs_params* p) {
  if (!h || !c || !d) return POGS_ERR_ARG;
  if (!p) p = &h->sp;
  if (validate_params(p) != 0) return POGS_ERR_ARG;
  cudaStream_t s = h->stream;
  TRY(reset_state(h, p));
  CK(cudaMemcpyAsync(h->cx, c, h->n * sizeof(float), is_device_ptr(c) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(h->dy, d, h->m * sizeof(float), is_device_ptr(d) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(h->xh, 0, h->nv * sizeof(float), s));
  CK(cudaMemsetAsync(h->mu, 0, h->nv * sizeof(float), s));
  CK(cudaMemsetAsync(h->yh, 0, h->mv * sizeof(float), s));
  CK(cudaMemsetAsync(h->nu, 0, h->mv * sizeof(float), s));
  enqueue_projection(h, p->refine_steps, cg_steps_for(h, p), s);
  release_kept_rows(h, s);
  CK(cudaGetLastError());
  TRY(copy_out(h->x, x, h->n, s));
  TRY(copy_out(h->y, y, h->m, s));
  CK(cudaStreamSynchronize(s));
  return 0;
}

}  // extern "C"

extern "C" {

int pogs_get_setup_report(const pogs_handle* h, pogs_setup_report* r) {
  if (!h || !r) return POGS_ERR_ARG;
  r->ingest_ms = h->phase_ms[0];
  r->equil_ms = h->phase_ms[1];
  r->gram_ms = h->phase_ms[2];
  r->factor_ms = h->phase_ms[3];
  r->inverse_ms = h->phase_ms[4];
  r->gram_prec_used = h->gram_used;
  r->chol_prec_used = h->sp.chol_prec;
  r->device_bytes = h->device_bytes;
  return 0;
}

long long pogs_kernel_launches(void) { return g_launch_count.load(); }

long long pogs_device_allocations(void) { return g_alloc_count.load(); }

int pogs_time_kernels(pogs_handle* h, int reps, double* ms, double* bytes) {
  if (!h || reps < 1 || !h->solved || h->indirect) return POGS_ERR_ARG;   // times the direct projection
  cudaStream_t s = h->stream;
  const double m = (double)h->m, n = (double)h->n, q = (double)h->q;
  // one pass over A^: dense m x n FP32; sparse: values + column indices + row pointers of the
  // CSR of A^ (row dots) or of A^T (column sums)
  const double nz = (double)h->nnz;
  const double An = h->sparse ? 8.0 * nz + 4.0 * (m + 1) : 4.0 * m * n;
  const double At = h->sparse ? 8.0 * nz + 4.0 * (n + 1) : 4.0 * m * n;
  const double tri = 2.0 * q * (q + 1.0);
  double b[7];
  b[0] = 41.0 * (m + n);                                   // prox: x, x~, params in; x^, c, mu out
  if (h->tall) {
    b[1] = At + 12 * m + 20 * n;                            // A^T [d, nu, y~] ; c, mu, E in ; r, x~ out
    b[2] = tri + 8 * q;
    b[3] = tri + 20 * q;                                   // z, c, x~ in ; x, x~ out
    if (h->St) {
      b[2] = tri + 24 * q;                                 // S tiles; r, c, x~ in ; x, x~ out
      b[3] = 0.0;
    }
    b[4] = An + 8 * n + 24 * m;                            // A [x, x^] ; d, y^, D, y~ in ; y, y~ out
  } else {
    b[1] = An + 8 * n + 16 * m;                            // A [c, x^] ; d, y^, D in ; r out
    b[2] = tri + 8 * q;
    b[3] = tri + 24 * q;                                   // z, d, y~ in ; y, y~, w out
    if (h->St) {
      b[2] = tri + 28 * q;                                 // S tiles; r, d, y~ in ; y, y~, w out
      b[3] = 0.0;
    }
    b[4] = At + 12 * m + 20 * n;                           // A^T [w, nu, y~] ; c, mu, E in ; x, x~ out
  }
  if (h->ldl) {   // the factor read twice (forward, backward), the work vector, the in/out vectors
    const LdlFactor& F = *h->ldl;
    b[2] = 2.0 * (double)F.panel_entries * 8.0 + 4.0 * 8.0 * F.N + 24.0 * q;
    b[3] = 0.0;
  }
  b[5] = 0.0;
  b[6] = b[0] + b[1] + b[2] + b[3] + b[4];
  // keep the stopping test from ever firing: zero tolerances, no iteration cap
  {
    CK(cudaStreamSynchronize(s));
    DevCfg c = *h->cfg_host;
    c.abs_tol = 0.0;
    c.rel_tol = 0.0;
    c.max_iter = 0x7fffffff;
    *h->cfg_host = c;
    CK(cudaMemcpyAsync(h->cfg, h->cfg_host, sizeof(DevCfg), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(&h->st->done, 0, sizeof(int), s));
  }
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const GemvGeom& g = h->geom;
  const int M = (int)h->m, N = (int)h->n, Q = (int)h->q;
  auto run = [&](int k) {
    switch (k) {
      case 0:
        launch_prox_step(N, M, h->x, h->xt, h->xh, h->cx, h->mu, h->y, h->yt, h->yh, h->dy, h->nu, fn_g(h), fn_f(h),
                         h->st, h->cfg, h->prox_part, h->nprox, s);
        break;
      case 1: {
        EpiArgs e = epi0();
        if (h->tall) {
          e.r = h->r; e.cx = h->cx; e.mu = h->mu; e.E = h->E; e.xt = h->xt; e.res_part = h->dual_part;
          launch_gemv_t(3, false, EPT_TALL_R, h->A, h->lda, M, N, h->dy, h->nu, h->yt, g, h->part_t, h->cnt_t, e, h->st,
                        s);
        } else {
          e.r = h->r; e.dy = h->dy; e.yh = h->yh; e.D = h->D; e.res_part = h->pri_part;
          launch_gemv_n(2, false, EPN_FAT_R, h->A, h->lda, M, N, h->cx, h->xh, g, h->part_n, h->cnt_n, e, h->st, s);
        }
        break;
      }
      case 2: {
        EpiArgs e = epi0();
        if (h->ldl) {   // the sparse LDL^T solve (all its launches)
          if (h->tall) {
            e.x = h->x; e.xt = h->xt; e.cx = h->cx;
            ldl_apply(*h->ldl, true, h->r, EPR_TALL_X, e, s);
          } else {
            e.y = h->y; e.yt = h->yt; e.dy = h->dy; e.w = h->w;
            ldl_apply(*h->ldl, false, h->r, EPR_FAT_Y, e, s);
          }
          break;
        }
        if (h->St) {   // the whole inverse in one symmetric pass
          if (h->tall) {
            e.x = h->x; e.xt = h->xt; e.cx = h->cx;
            launch_symv(EPR_TALL_X, h->St, h->T, Q, h->r, h->part_sy, h->cnt_tr, e, h->st, s);
          } else {
            e.y = h->y; e.yt = h->yt; e.dy = h->dy; e.w = h->w;
            launch_symv(EPR_FAT_Y, h->St, h->T, Q, h->r, h->part_sy, h->cnt_tr, e, h->st, s);
          }
          break;
        }
        e.out1 = h->z;
        launch_trmv(false, EPR_RAW, h->Mt, h->T, Q, h->r, h->part_tr, h->cnt_tr, e, h->st, s);
        break;
      }
      case 3: {
        if (h->St || h->ldl) break;
        EpiArgs e = epi0();
        if (h->tall) {
          e.x = h->x; e.xt = h->xt; e.cx = h->cx;
          launch_trmv(true, EPR_TALL_X, h->Mt, h->T, Q, h->z, h->part_tr, h->cnt_tr, e, h->st, s);
        } else {
          e.y = h->y; e.yt = h->yt; e.dy = h->dy; e.w = h->w;
          launch_trmv(true, EPR_FAT_Y, h->Mt, h->T, Q, h->z, h->part_tr, h->cnt_tr, e, h->st, s);
        }
        break;
      }
      case 4: {
        EpiArgs e = epi0();
        if (h->tall) {
          e.y = h->y; e.yt = h->yt; e.dy = h->dy; e.yh = h->yh; e.D = h->D; e.res_part = h->pri_part;
          launch_gemv_n(2, false, EPN_TALL_Y, h->A, h->lda, M, N, h->x, h->xh, g, h->part_n, h->cnt_n, e, h->st, s);
        } else {
          e.x = h->x; e.xt = h->xt; e.cx = h->cx; e.mu = h->mu; e.E = h->E; e.res_part = h->dual_part;
          launch_gemv_t(3, false, EPT_FAT_X, h->A, h->lda, M, N, h->w, h->nu, h->yt, g, h->part_t, h->cnt_t, e, h->st,
                        s);
        }
        break;
      }
      case 5:
        launch_check(h->st, h->cfg, h->prox_part, h->nprox, h->pri_part, g.n_nrowblk, h->dual_part, g.t_ncolblk, 0ull,
                     0, s);
        break;
    }
  };
  double t[7];
  for (int k = 0; k <= 6; ++k) {
    if (k < 6) run(k);
    else for (int j = 0; j < 6; ++j) run(j);
    CK(cudaEventRecord(e0, s));
    for (int r = 0; r < reps; ++r) {
      if (k < 6) run(k);
      else for (int j = 0; j < 6; ++j) run(j);
    }
    CK(cudaEventRecord(e1, s));
    CK(cudaEventSynchronize(e1));
    float el = 0.0f;
    CK(cudaEventElapsedTime(&el, e0, e1));
    t[k] = (double)el / reps;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  release_kept_rows(h, s);
  CK(cudaGetLastError());
  h->solved = false;   // iterate state is no longer a solve result
  for (int k = 0; k < 7; ++k) {
    if (ms) ms[k] = t[k];
    if (bytes) bytes[k] = b[k];
  }
  return 0;
}

}  // extern "C"

extern "C" int pogs_check_bounded_wait(void* stream) {
  return pogs::bounded_wait_probe(static_cast<cudaStream_t>(stream));
}

extern "C" int pogs_gram(const float* A, int64_t m, int64_t n, int64_t lda, int gram_prec, float* G, void* stream) {
  if (!A || !G || m < 1 || n < 1 || lda < n || gram_prec < POGS_GRAM_BF16 || gram_prec > POGS_GRAM_FP32)
    return POGS_ERR_ARG;
  if (!is_device_ptr(A) || !is_device_ptr(G)) return POGS_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool tall = m >= n;
  const int64_t q = tall ? n : m;
  int* err = nullptr;
  if (pool_alloc(reinterpret_cast<void**>(&err), sizeof(int), s) != 0) return POGS_ERR_OOM;
  CK(cudaMemsetAsync(err, 0, sizeof(int), s));
  int rc = 0;
  if (gram_prec == POGS_GRAM_FP32) {
    if (tall) gemm_f32(true, false, q, q, m, 1.0f, A, lda, A, lda, 0.0f, G, q, true, s);
    else gemm_f32(false, true, q, q, n, 1.0f, A, lda, A, lda, 0.0f, G, q, true, s);
  } else {
    size_t need = 0;
    rc = gram_tensor(gram_prec, A, lda, m, n, tall, G, q, nullptr, 0, &need, err, s);
    void* ws = nullptr;
    if (rc == 0 && pool_alloc(&ws, need, s) != 0) rc = POGS_ERR_OOM;
    if (rc == 0 && gram_tensor(gram_prec, A, lda, m, n, tall, G, q, ws, need, &need, err, s) != 0) rc = POGS_ERR_CUDA;
    if (ws) cudaFreeAsync(ws, s);
  }
  int herr = 0;
  if (cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    rc = POGS_ERR_CUDA;
  cudaFreeAsync(err, s);
  if (rc == 0 && herr != 0) rc = herr;
  if (rc == 0 && cudaGetLastError() != cudaSuccess) rc = POGS_ERR_CUDA;
  return rc;
}
