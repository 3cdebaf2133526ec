// Continuous-batching server: requests are admitted against a device-memory budget, stay
// resident on the device (matrix, factor, scalings and ADMM state), and advance together.
//
// Requests with min(m, n) <= 512 use the batched engine: each step launches the persistent
// iteration kernel once over every resident request, advancing each by up to `iters`
// iterations from its saved loop state; requests admitted between steps join at the next one
// and finished ones retire (outputs copied, memory released) after it.  Larger requests run
// through the single-problem path on worker threads with their own streams.  The two kinds take
// turns on the device (GpuGate below).  A request's result does not depend on what else is
// resident: the batched engine's arithmetic is fixed per instance and exact across step
// boundaries.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "batch.h"
#include "gate.h"
#include "kernels.h"

using namespace pogs;

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}
size_t al(size_t x) { return (x + 255) & ~size_t(255); }
bool is_dev(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

constexpr int kSmallMaxQ = 512;

// A step's hold on the gate, released on every return path.
struct StepHold {
  GpuGate* g = nullptr;
  void take(GpuGate& gate) {
    gate.write_lock();
    g = &gate;
  }
  void release() {
    if (g) g->write_unlock();
    g = nullptr;
  }
  ~StepHold() { release(); }
};

struct SReq {
  int64_t tag = 0;
  pogs_problem prob{};
  float *x = nullptr, *y = nullptr, *mu = nullptr, *nu = nullptr;
  bool small = false;
  size_t bytes = 0;
  double t_submit = 0, t_admit = 0;
  int slot = -1;
  char* arena = nullptr;
  BInst inst{};
};

// Device bytes a request holds while resident.
size_t small_bytes(int64_t m, int64_t n) {
  // vectors at a pitch of a multiple of 4 floats (the iteration reads some of them as float4)
  const int64_t q = std::min(m, n), v = (std::max(m, n) + 3) / 4 * 4, lda4 = (n + 3) / 4 * 4;
  size_t b = al((size_t)m * lda4 * 4) + al((size_t)q * q * 4) + al((size_t)q * q * 8) + al((size_t)m * 4) +
             al((size_t)n * 4) + al((size_t)17 * v * 4);
  for (int t = 0; t < 24; ++t) b += al((size_t)((t % 12) < 6 ? m : n) * (((t % 6) == 0) ? 1 : 4));
  return b;
}
size_t large_bytes(int64_t m, int64_t n) {
  const int64_t q = std::min(m, n), p = std::max(m, n);
  const int64_t T = (q + 127) / 128;
  // matrix + tiles + vectors resident, plus the setup peak (Gram, FP64 factor, dense inverse,
  // packed tensor-core operands)
  return (size_t)m * ((n + 31) / 32 * 32) * 4 + (size_t)T * (T + 1) / 2 * 128 * 128 * 4 + (size_t)64 * (m + n) * 4 +
         (size_t)q * q * (4 + 8 + 4 + 2) + (size_t)((q + 127) / 128 * 128) * ((p + 63) / 64 * 64) * 4;
}

}  // namespace

struct pogs_server {
  size_t budget = 0, used = 0;
  pogs_params p{};
  BCfg cfg{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;           // internal highest-priority stream (caller passed none)
  cudaEvent_t ev_in = nullptr;       // orders the internal stream after the legacy stream
  int num_sms = 148;
  int cap = 0;                       // slots for resident small requests
  BOut* d_outs = nullptr;
  BLoop* d_loops = nullptr;
  BInst* d_active = nullptr;
  BInst* d_new = nullptr;
  int* d_queue = nullptr;
  std::vector<int> free_slots;
  std::deque<SReq*> waiting;         // small requests not yet admitted
  std::vector<SReq*> active;
  std::vector<pogs_server_done> done;
  std::vector<BOut> h_outs;
  std::vector<BLoop> h_loops;
  // large requests
  std::vector<std::thread> workers;
  std::deque<SReq*> large_q;         // large requests not yet started by a worker
  std::mutex mu;
  std::condition_variable cv;
  GpuGate gate;
  bool stop = false;
  int64_t submitted = 0, completed = 0;
  // staging of admitted requests' host inputs: packed into one pinned buffer, copied to the
  // device in one transfer, and scattered to their arenas by one kernel (grow-only buffers)
  char* h_stage = nullptr;
  size_t h_stage_bytes = 0;
  char* d_stage = nullptr;
  size_t d_stage_bytes = 0;
  struct Piece* d_pieces = nullptr;
  size_t d_pieces_cap = 0;
};

namespace {

void worker_main(pogs_server* S) {
  // large requests run on low-priority streams; they take turns with the batched steps (the
  // gate), so the priority only orders what is left pending at a turn's boundary
  cudaStream_t st;
  cudaEvent_t ev = nullptr;
  int lo = 0, hi = 0;
  cudaDeviceGetStreamPriorityRange(&lo, &hi);
  if (cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, lo) != cudaSuccess) {
    cudaGetLastError();
    st = nullptr;
  }
  if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    ev = nullptr;
  }
  while (true) {
    SReq* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      // a large request is charged to the budget when a worker starts it: queued, it holds
      // no device memory
      S->cv.wait(lk, [&] {
        return S->stop || (!S->large_q.empty() && S->used + S->large_q.front()->bytes <= S->budget);
      });
      if (S->stop) break;
      r = S->large_q.front();
      S->large_q.pop_front();
      S->used += r->bytes;
      r->t_admit = now_s();
    }
    pogs_server_done d;
    memset(&d, 0, sizeof(d));
    d.tag = r->tag;
    d.submit_s = r->t_submit;
    d.admit_s = r->t_admit;
    pogs_handle* h = nullptr;
    // device inputs written before the submission, on the server's stream (or the legacy
    // default stream when the server owns its stream), are ordered before their use here
    if (st && ev) {
      cudaEventRecord(ev, S->own_stream ? (cudaStream_t)0 : S->stream);
      cudaStreamWaitEvent(st, ev, 0);
    }
    S->gate.read_lock();
    int rc = pogs_setup(r->prob.A, r->prob.m, r->prob.n, r->prob.lda, 'R', &S->p, st, &h);
    if (rc == 0) {
      rc = pogs_solve(h, &r->prob.f, &r->prob.g, &S->p, r->x, r->y, r->mu, r->nu, &d.info);
      pogs_free(h);
    }
    S->gate.read_unlock();
    d.info.status = rc;
    d.done_s = now_s();
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->done.push_back(d);
      S->used -= r->bytes;
      ++S->completed;
    }
    S->cv.notify_all();
    delete r;
  }
  if (ev) cudaEventDestroy(ev);
  if (st) cudaStreamDestroy(st);
}

// Lay out a small request's arena and fill its descriptor (device pointers).
void layout_small(SReq* r, BOut* out, BLoop* loop) {
  const pogs_problem& pr = r->prob;
  BInst& I = r->inst;
  memset(&I, 0, sizeof(I));
  char* a = r->arena;
  size_t cur = 0;
  auto take = [&](size_t bytes) {
    char* p = a + cur;
    cur = al(cur + bytes);
    return p;
  };
  I.m = (int)pr.m;
  I.n = (int)pr.n;
  I.lda = (int)((pr.n + 3) / 4 * 4);
  I.q = (int)std::min(pr.m, pr.n);
  I.tall = pr.m >= pr.n;
  I.A = (float*)take((size_t)pr.m * I.lda * 4);
  I.M = (float*)take((size_t)I.q * I.q * 4);
  I.H = (double*)take((size_t)I.q * I.q * 8);
  I.D = (float*)take((size_t)pr.m * 4);
  I.E = (float*)take((size_t)pr.n * 4);
  void* raw[12];
  for (int t = 0; t < 12; ++t) raw[t] = take((size_t)(t < 6 ? pr.m : pr.n) * ((t % 6) == 0 ? 1 : 4));
  const void* src[12] = {pr.f.h, pr.f.a, pr.f.b, pr.f.c, pr.f.d, pr.f.e, pr.g.h, pr.g.a, pr.g.b, pr.g.c, pr.g.d, pr.g.e};
  auto in = [&](int t) -> void* { return src[t] ? raw[t] : nullptr; };
  I.fh0 = (const uint8_t*)in(0); I.fa0 = (const float*)in(1); I.fb0 = (const float*)in(2);
  I.fc0 = (const float*)in(3); I.fd0 = (const float*)in(4); I.fe0 = (const float*)in(5);
  I.gh0 = (const uint8_t*)in(6); I.ga0 = (const float*)in(7); I.gb0 = (const float*)in(8);
  I.gc0 = (const float*)in(9); I.gd0 = (const float*)in(10); I.ge0 = (const float*)in(11);
  void* fo[12];
  for (int t = 0; t < 12; ++t) fo[t] = take((size_t)(t < 6 ? pr.m : pr.n) * ((t % 6) == 0 ? 1 : 4));
  I.fh = (uint8_t*)fo[0]; I.fa = (float*)fo[1]; I.fb = (float*)fo[2]; I.fc = (float*)fo[3]; I.fd = (float*)fo[4];
  I.fe = (float*)fo[5];
  I.gh = (uint8_t*)fo[6]; I.ga = (float*)fo[7]; I.gb = (float*)fo[8]; I.gc = (float*)fo[9]; I.gd = (float*)fo[10];
  I.ge = (float*)fo[11];
  const int64_t v = (std::max(pr.m, pr.n) + 3) / 4 * 4;   // 16-byte aligned vectors (float4 reads)
  float* vec = (float*)take((size_t)17 * v * 4);
  float** vecs[] = {&I.x, &I.y, &I.xt, &I.yt, &I.xh, &I.yh, &I.cx, &I.dy, &I.mu, &I.nu, &I.r, &I.z, &I.w,
                    &I.ox, &I.oy, &I.omu, &I.onu};
  for (int t = 0; t < 17; ++t) *vecs[t] = vec + (size_t)t * v;
  I.out = out;
  I.loop = loop;
}

}  // namespace

// One staged input: `rows` rows of `row_bytes` bytes, contiguous at `src` in the device staging
// buffer, written `pitch` bytes apart at `dst` (an arena).
struct Piece {
  size_t src;
  char* dst;
  int64_t rows, row_bytes, pitch;
};

namespace {

// One block per piece; 16-byte words where the row is 16-byte sized and both ends aligned
// (the matrix rows when n is a multiple of 4), bytes otherwise.
__global__ void scatter_pieces_kernel(const char* __restrict__ stage, const Piece* __restrict__ pieces) {
  const Piece pc = pieces[blockIdx.x];
  const char* src = stage + pc.src;
  const bool wide = ((pc.row_bytes | pc.pitch | (int64_t)(uintptr_t)pc.dst | (int64_t)pc.src) & 15) == 0;
  for (int64_t r = 0; r < pc.rows; ++r) {
    const char* sr = src + r * pc.row_bytes;
    char* dr = pc.dst + r * pc.pitch;
    if (wide) {
      for (int64_t k = threadIdx.x; k < pc.row_bytes / 16; k += blockDim.x)
        reinterpret_cast<float4*>(dr)[k] = reinterpret_cast<const float4*>(sr)[k];
    } else {
      for (int64_t k = threadIdx.x; k < pc.row_bytes; k += blockDim.x) dr[k] = sr[k];
    }
  }
}

// The host inputs of the requests in `list` (all host-resident), in chunks of about kStageChunk
// bytes: each chunk is packed into the pinned staging buffer (several threads for large chunks),
// copied to the device in one transfer and scattered to the arenas by one launch; the stream is
// synchronised before the buffers are reused.
constexpr size_t kStageChunk = (size_t)1 << 30;

int stage_chunk(pogs_server* S, const std::vector<Piece>& pieces, const std::vector<const char*>& hsrc,
                size_t total, cudaStream_t s) {
  if (total > S->h_stage_bytes) {
    if (S->h_stage) cudaFreeHost(S->h_stage);
    S->h_stage = nullptr;
    S->h_stage_bytes = 0;
    if (cudaHostAlloc(reinterpret_cast<void**>(&S->h_stage), total, cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      return POGS_ERR_OOM;
    }
    S->h_stage_bytes = total;
  }
  if (total > S->d_stage_bytes) {
    if (S->d_stage) cudaFreeAsync(S->d_stage, s);
    S->d_stage = nullptr;
    S->d_stage_bytes = 0;
    count_alloc();
    if (cudaMallocAsync(reinterpret_cast<void**>(&S->d_stage), total, s) != cudaSuccess) {
      cudaGetLastError();
      return POGS_ERR_OOM;
    }
    S->d_stage_bytes = total;
  }
  if (pieces.size() > S->d_pieces_cap) {
    if (S->d_pieces) cudaFreeAsync(S->d_pieces, s);
    S->d_pieces = nullptr;
    S->d_pieces_cap = 0;
    count_alloc();
    if (cudaMallocAsync(reinterpret_cast<void**>(&S->d_pieces), pieces.size() * sizeof(Piece), s) != cudaSuccess) {
      cudaGetLastError();
      return POGS_ERR_OOM;
    }
    S->d_pieces_cap = pieces.size();
  }
  const int nth = total > ((size_t)64 << 20) ? 8 : 1;
  auto pack = [&](size_t lo, size_t hi) {
    for (size_t i = lo; i < hi; ++i)
      std::memcpy(S->h_stage + pieces[i].src, hsrc[i], (size_t)(pieces[i].rows * pieces[i].row_bytes));
  };
  if (nth == 1) {
    pack(0, pieces.size());
  } else {   // pieces split evenly by bytes
    std::vector<size_t> cut(nth + 1, pieces.size());
    cut[0] = 0;
    size_t i = 0;
    for (int t = 1; t < nth; ++t) {
      const size_t goal = total * t / nth;
      while (i < pieces.size() && pieces[i].src < goal) ++i;
      cut[t] = i;
    }
    std::vector<std::thread> th;
    for (int t = 0; t < nth; ++t) th.emplace_back(pack, cut[t], cut[t + 1]);
    for (auto& x : th) x.join();
  }
  if (cudaMemcpyAsync(S->d_stage, S->h_stage, total, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(S->d_pieces, pieces.data(), pieces.size() * sizeof(Piece), cudaMemcpyHostToDevice, s) !=
          cudaSuccess) {
    cudaGetLastError();
    return POGS_ERR_CUDA;
  }
  count_launch();
  scatter_pieces_kernel<<<(unsigned)pieces.size(), 256, 0, s>>>(S->d_stage, S->d_pieces);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return POGS_ERR_CUDA;
  }
  return 0;
}

int stage_host_inputs(pogs_server* S, const std::vector<SReq*>& list, cudaStream_t s) {
  std::vector<Piece> pieces;
  std::vector<const char*> hsrc;
  size_t total = 0;
  auto add = [&](const void* src, void* dst, int64_t rows, int64_t row_bytes, int64_t pitch, int64_t src_pitch) {
    // rows of a strided host source are packed contiguously, one piece per row
    const bool contiguous = src_pitch == row_bytes;
    for (int64_t r = 0; r < (contiguous ? 1 : rows); ++r) {
      Piece pc;
      pc.src = total;
      pc.dst = static_cast<char*>(dst) + r * pitch;
      pc.rows = contiguous ? rows : 1;
      pc.row_bytes = row_bytes;
      pc.pitch = pitch;
      pieces.push_back(pc);
      hsrc.push_back(static_cast<const char*>(src) + r * src_pitch);
      total += (size_t)((pc.rows * row_bytes + 15) & ~int64_t(15));
    }
  };
  for (SReq* r : list) {
    const pogs_problem& pr = r->prob;
    const BInst& I = r->inst;
    add(pr.A, I.A, pr.m, pr.n * 4, (int64_t)I.lda * 4, pr.lda * 4);
    const void* src[12] = {pr.f.h, pr.f.a, pr.f.b, pr.f.c, pr.f.d, pr.f.e, pr.g.h, pr.g.a, pr.g.b, pr.g.c, pr.g.d, pr.g.e};
    const void* dst[12] = {I.fh0, I.fa0, I.fb0, I.fc0, I.fd0, I.fe0, I.gh0, I.ga0, I.gb0, I.gc0, I.gd0, I.ge0};
    for (int t = 0; t < 12; ++t) {
      if (!src[t]) continue;
      const int64_t bytes = (t < 6 ? pr.m : pr.n) * ((t % 6) == 0 ? 1 : 4);
      add(src[t], const_cast<void*>(dst[t]), 1, bytes, bytes, bytes);
    }
    if (total >= kStageChunk) {
      const int rc = stage_chunk(S, pieces, hsrc, total, s);
      if (rc != 0) return rc;
      pieces.clear();
      hsrc.clear();
      total = 0;
    }
  }
  return pieces.empty() ? 0 : stage_chunk(S, pieces, hsrc, total, s);
}

int copy_inputs(SReq* r, cudaStream_t s) {
  const pogs_problem& pr = r->prob;
  const BInst& I = r->inst;
  const cudaMemcpyKind kA = is_dev(pr.A) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (cudaMemcpy2DAsync(I.A, (size_t)I.lda * 4, pr.A, (size_t)pr.lda * 4, (size_t)pr.n * 4, pr.m, kA, s) !=
      cudaSuccess)
    return POGS_ERR_CUDA;
  const void* src[12] = {pr.f.h, pr.f.a, pr.f.b, pr.f.c, pr.f.d, pr.f.e, pr.g.h, pr.g.a, pr.g.b, pr.g.c, pr.g.d, pr.g.e};
  const void* dst[12] = {I.fh0, I.fa0, I.fb0, I.fc0, I.fd0, I.fe0, I.gh0, I.ga0, I.gb0, I.gc0, I.gd0, I.ge0};
  for (int t = 0; t < 12; ++t) {
    if (!src[t]) continue;
    const size_t bytes = (size_t)(t < 6 ? pr.m : pr.n) * ((t % 6) == 0 ? 1 : 4);
    if (cudaMemcpyAsync(const_cast<void*>(dst[t]), src[t], bytes,
                        is_dev(src[t]) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s) != cudaSuccess)
      return POGS_ERR_CUDA;
  }
  return 0;
}

}  // namespace

extern "C" {

int pogs_server_create(size_t hbm_budget, int large_workers, int max_resident, const pogs_params* p, void* stream,
                       pogs_server** out) {
  if (!out || hbm_budget == 0 || large_workers < 0 || max_resident < 1) return POGS_ERR_ARG;
  *out = nullptr;
  pogs_server* S = new pogs_server();
  pogs_default_params(&S->p);
  if (p) S->p = *p;
  S->budget = hbm_budget;
  S->stream = static_cast<cudaStream_t>(stream);
  if (!S->stream) {
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (cudaStreamCreateWithPriority(&S->stream, cudaStreamNonBlocking, hi) != cudaSuccess ||
        cudaEventCreateWithFlags(&S->ev_in, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      if (S->stream) cudaStreamDestroy(S->stream);
      delete S;
      return POGS_ERR_CUDA;
    }
    S->own_stream = true;
  }
  S->cap = max_resident;
  BCfg& c = S->cfg;
  memset(&c, 0, sizeof(c));
  c.abs_tol = S->p.abs_tol; c.rel_tol = S->p.rel_tol; c.rho0 = S->p.rho0; c.alpha = S->p.alpha; c.delta = S->p.delta;
  c.tau = S->p.tau; c.gamma_scale = S->p.gamma; c.max_iter = S->p.max_iter; c.gap_stop = S->p.gap_stop;
  c.adaptive = S->p.adaptive_rho; c.sk_sweeps = S->p.sk_sweeps; c.equil = S->p.equil;
  c.mixed_chol = S->p.chol_prec == POGS_CHOL_MIXED;
  int dev = 0;
  count_alloc(5);
  bool ok = cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&S->num_sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
            cudaMalloc(&S->d_outs, sizeof(BOut) * S->cap) == cudaSuccess &&
            cudaMalloc(&S->d_loops, sizeof(BLoop) * S->cap) == cudaSuccess &&
            cudaMalloc(&S->d_active, sizeof(BInst) * S->cap) == cudaSuccess &&
            cudaMalloc(&S->d_new, sizeof(BInst) * S->cap) == cudaSuccess &&
            cudaMalloc(&S->d_queue, sizeof(int)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    pogs_server_destroy(S);
    return POGS_ERR_OOM;
  }
  {
    // keep freed request memory in the stream-ordered pool for the next admissions
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t keep = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
  }
  for (int i = S->cap - 1; i >= 0; --i) S->free_slots.push_back(i);
  S->h_outs.resize(S->cap);
  S->h_loops.resize(S->cap);
  for (int i = 0; i < large_workers; ++i) S->workers.emplace_back(worker_main, S);
  *out = S;
  return 0;
}

int pogs_server_submit(pogs_server* S, const pogs_problem* prob, float* x, float* y, float* mu, float* nu,
                       int64_t tag) {
  if (!S || !prob || !prob->A || prob->m < 1 || prob->n < 1 || prob->lda < prob->n || !prob->f.h || !prob->g.h)
    return POGS_ERR_ARG;
  // no CUDA call here: with the workers busy in the driver, each one could wait milliseconds,
  // and submission is on the caller's critical path.  The stream ordering of device inputs is
  // set up when a request is admitted (pogs_server_step, worker_main).
  SReq* r = new SReq();
  r->tag = tag;
  r->prob = *prob;
  r->x = x; r->y = y; r->mu = mu; r->nu = nu;
  r->small = std::min(prob->m, prob->n) <= kSmallMaxQ;
  r->bytes = r->small ? small_bytes(prob->m, prob->n) : large_bytes(prob->m, prob->n);
  if (r->bytes > S->budget) {
    delete r;
    return POGS_ERR_CAPACITY;
  }
  r->t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    (r->small ? S->waiting : S->large_q).push_back(r);
    ++S->submitted;
  }
  if (!r->small) S->cv.notify_all();
  return 0;
}

int pogs_server_step(pogs_server* S, int iters) {
  if (!S || iters < 1) return POGS_ERR_ARG;
  cudaStream_t s = S->stream;
  // ---- admission of small requests: first come first served, within the memory budget and
  // the slot count (large requests are admitted by the workers, in their own order) ----------
  std::vector<SReq*> fresh;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    while (!S->waiting.empty()) {
      SReq* r = S->waiting.front();
      if (S->used + r->bytes > S->budget || S->free_slots.empty()) break;
      S->waiting.pop_front();
      S->used += r->bytes;
      r->t_admit = now_s();
      r->slot = S->free_slots.back();
      S->free_slots.pop_back();
      fresh.push_back(r);
    }
  }
  if (fresh.empty() && S->active.empty()) return 0;
  if (!fresh.empty() && S->own_stream) {
    // device inputs written on the legacy default stream before their submission are ordered
    // before their use on the server's internal (non-blocking) stream
    if (cudaEventRecord(S->ev_in, 0) != cudaSuccess || cudaStreamWaitEvent(s, S->ev_in, 0) != cudaSuccess) {
      cudaGetLastError();
      return POGS_ERR_CUDA;
    }
  }
  StepHold hold;
  hold.take(S->gate);
  std::vector<SReq*> host_in;
  for (SReq* r : fresh) {
    count_alloc();
    if (cudaMallocAsync((void**)&r->arena, r->bytes, s) != cudaSuccess) {
      cudaGetLastError();
      return POGS_ERR_OOM;
    }
    layout_small(r, S->d_outs + r->slot, S->d_loops + r->slot);
    // requests whose inputs all live in host memory are staged together below
    const pogs_problem& pr = r->prob;
    const void* ins[13] = {pr.A, pr.f.h, pr.f.a, pr.f.b, pr.f.c, pr.f.d, pr.f.e,
                           pr.g.h, pr.g.a, pr.g.b, pr.g.c, pr.g.d, pr.g.e};
    bool any_dev = false;
    for (const void* p : ins) any_dev = any_dev || is_dev(p);
    if (any_dev) {
      if (copy_inputs(r, s) != 0) return POGS_ERR_CUDA;
    } else {
      host_in.push_back(r);
    }
    if (cudaMemsetAsync(S->d_outs + r->slot, 0, sizeof(BOut), s) != cudaSuccess ||
        cudaMemsetAsync(S->d_loops + r->slot, 0, sizeof(BLoop), s) != cudaSuccess)
      return POGS_ERR_CUDA;
    S->active.push_back(r);
  }
  if (!host_in.empty()) {
    const int rc = stage_host_inputs(S, host_in, s);
    if (rc != 0) return rc;
  }
  if (!fresh.empty()) {
    std::vector<BInst> hn;
    for (SReq* r : fresh) hn.push_back(r->inst);
    if (cudaMemcpyAsync(S->d_new, hn.data(), sizeof(BInst) * hn.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
      return POGS_ERR_CUDA;
    int rc = batch_setup(S->d_new, (int)hn.size(), S->cfg, s);
    if (rc != 0) return rc;
  }
  // ---- one launch advances every resident request ------------------------------------------
  std::vector<BInst> ha;
  for (SReq* r : S->active) ha.push_back(r->inst);
  const int na = (int)ha.size();
  if (cudaMemcpyAsync(S->d_active, ha.data(), sizeof(BInst) * na, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(S->d_queue, 0, sizeof(int), s) != cudaSuccess)
    return POGS_ERR_CUDA;
  int rc = batch_iterate(S->d_active, na, S->cfg, S->d_queue, nullptr, S->num_sms * 4, 0, iters, s);
  if (rc != 0) return rc;
  if (cudaMemcpyAsync(S->h_outs.data(), S->d_outs, sizeof(BOut) * S->cap, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(S->h_loops.data(), S->d_loops, sizeof(BLoop) * S->cap, cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return POGS_ERR_CUDA;
  }
  hold.release();
  // ---- retire finished requests ------------------------------------------------------------------
  std::vector<SReq*> keep;
  const double t = now_s();
  for (SReq* r : S->active) {
    const BOut& o = S->h_outs[r->slot];
    const BLoop& L = S->h_loops[r->slot];
    const bool setup_failed = o.status != 0 && o.iters == 0;
    if (!setup_failed && !L.done) {
      keep.push_back(r);
      continue;
    }
    const BInst& I = r->inst;
    const float* srcs[4] = {I.ox, I.oy, I.omu, I.onu};
    float* dsts[4] = {r->x, r->y, r->mu, r->nu};
    const int64_t lens[4] = {I.n, I.m, I.n, I.m};
    if (!setup_failed)
      for (int k = 0; k < 4; ++k)
        if (dsts[k])
          cudaMemcpyAsync(dsts[k], srcs[k], (size_t)lens[k] * 4,
                          is_dev(dsts[k]) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(r->arena, s);
    pogs_server_done d;
    memset(&d, 0, sizeof(d));
    d.tag = r->tag;
    d.submit_s = r->t_submit;
    d.admit_s = r->t_admit;
    d.done_s = t;
    d.info.status = o.status;
    d.info.iters = o.iters;
    d.info.rho = o.rho;
    d.info.r_pri = o.r_pri;
    d.info.r_dual = o.r_dual;
    d.info.eps_pri = o.eps_pri;
    d.info.eps_dual = o.eps_dual;
    d.info.gap = o.gap;
    d.info.obj = o.obj;
    d.info.r_pri_unscaled = o.r_pri_u;
    d.info.r_dual_unscaled = o.r_dual_u;
    std::lock_guard<std::mutex> lk(S->mu);
    S->done.push_back(d);
    S->used -= r->bytes;
    S->free_slots.push_back(r->slot);
    ++S->completed;
    delete r;
  }
  S->active.swap(keep);
  S->cv.notify_all();   // budget returned: a worker may start a large request
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return POGS_ERR_CUDA;
  }
  return 0;
}

int pogs_server_poll(pogs_server* S, pogs_server_done* out, int max) {
  if (!S || (max > 0 && !out)) return POGS_ERR_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  const int k = std::min<int>(max, (int)S->done.size());
  for (int i = 0; i < k; ++i) out[i] = S->done[i];
  S->done.erase(S->done.begin(), S->done.begin() + k);
  return k;
}

int pogs_server_pending(pogs_server* S) {
  if (!S) return POGS_ERR_ARG;
  std::lock_guard<std::mutex> lk(S->mu);
  return (int)(S->submitted - S->completed);
}

void pogs_server_destroy(pogs_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  for (auto& t : S->workers) t.join();
  if (S->stream) cudaStreamSynchronize(S->stream);
  for (SReq* r : S->active) {
    cudaFree(r->arena);
    delete r;
  }
  for (SReq* r : S->waiting) delete r;
  for (SReq* r : S->large_q) delete r;
  cudaFree(S->d_outs);
  cudaFree(S->d_loops);
  cudaFree(S->d_active);
  cudaFree(S->d_new);
  cudaFree(S->d_queue);
  if (S->d_stage) cudaFree(S->d_stage);
  if (S->d_pieces) cudaFree(S->d_pieces);
  if (S->h_stage) cudaFreeHost(S->h_stage);
  if (S->ev_in) cudaEventDestroy(S->ev_in);
  if (S->own_stream) cudaStreamDestroy(S->stream);
  delete S;
}

}  // extern "C"
