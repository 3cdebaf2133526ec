// pogs_solve_batch: host side of the batched solver (arena layout, ingest, launch-configuration
// autotuning, CUDA-graph launch of the persistent kernel, results).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <thread>
#include <tuple>
#include <vector>

#include "batch.h"
#include "kernels.h"

using namespace pogs;

namespace {

constexpr int kMaxBatchQ = 512;   // batched setup keeps a q x 32 FP32 panel in shared memory

bool is_dev(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

size_t al(size_t x) { return (x + 255) & ~size_t(255); }

// Pinned host memory for staging host inputs and outputs, kept between calls and grown on demand
// (up to kPinnedMax); one call holds it at a time, and a call that finds it taken, or needs more,
// stages in pageable memory instead.
constexpr size_t kPinnedMax = size_t(4) << 30;
struct PinnedStage {
  std::mutex mu;
  char* p = nullptr;
  size_t cap = 0;
};
PinnedStage g_pin;

// The pinned buffer with at least `bytes`, locked by `lk`, or nullptr.
char* pinned(std::unique_lock<std::mutex>& lk, size_t bytes) {
  if (bytes > kPinnedMax) return nullptr;
  lk = std::unique_lock<std::mutex>(g_pin.mu, std::try_to_lock);
  if (!lk.owns_lock()) return nullptr;
  if (g_pin.cap < bytes) {
    if (g_pin.p) cudaFreeHost(g_pin.p);
    g_pin.p = nullptr;
    g_pin.cap = 0;
    if (cudaHostAlloc(reinterpret_cast<void**>(&g_pin.p), bytes, cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      g_pin.p = nullptr;
      lk.unlock();
      return nullptr;
    }
    g_pin.cap = bytes;
  }
  return g_pin.p;
}

// f(k) for k < n on up to eight host threads.
template <class F>
void parallel_for(int n, F f) {
  const int nt = std::max(1, std::min({8, n, (int)std::thread::hardware_concurrency()}));
  if (nt == 1) {
    for (int k = 0; k < n; ++k) f(k);
    return;
  }
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t)
    th.emplace_back([&, t] {
      for (int k = t; k < n; k += nt) f(k);
    });
  for (auto& x : th) x.join();
}

// One region copied between a caller's device array and an arena: `rows` rows of `row_bytes`
// bytes, `src_pitch` / `dst_pitch` bytes apart; each destination row is zero-filled from
// row_bytes to fill_bytes (an arena row's padding).
struct DevPiece {
  const char* src;
  char* dst;
  int64_t rows, row_bytes, src_pitch, dst_pitch, fill_bytes;
};

// All regions of one call in one launch: block b takes pieces b, b + grid, ...; 16-byte words
// where both rows and pitches allow, else 4-byte words, else bytes.
__global__ void __launch_bounds__(256) copy_pieces_kernel(const DevPiece* __restrict__ pcs, int count) {
  for (int p = blockIdx.x; p < count; p += gridDim.x) {
    const DevPiece pc = pcs[p];
    const uintptr_t al_bits = (uintptr_t)pc.src | (uintptr_t)pc.dst | (uintptr_t)pc.row_bytes |
                              (uintptr_t)pc.src_pitch | (uintptr_t)pc.dst_pitch | (uintptr_t)pc.fill_bytes;
    for (int64_t r = 0; r < pc.rows; ++r) {
      const char* sr = pc.src + r * pc.src_pitch;
      char* dr = pc.dst + r * pc.dst_pitch;
      if ((al_bits & 15) == 0) {
        for (int64_t k = threadIdx.x; k < pc.fill_bytes / 16; k += blockDim.x)
          reinterpret_cast<float4*>(dr)[k] = 16 * k < pc.row_bytes ? reinterpret_cast<const float4*>(sr)[k]
                                                                    : make_float4(0.f, 0.f, 0.f, 0.f);
      } else if ((al_bits & 3) == 0) {
        for (int64_t k = threadIdx.x; k < pc.fill_bytes / 4; k += blockDim.x)
          reinterpret_cast<float*>(dr)[k] = 4 * k < pc.row_bytes ? reinterpret_cast<const float*>(sr)[k] : 0.0f;
      } else {
        for (int64_t k = threadIdx.x; k < pc.fill_bytes; k += blockDim.x) dr[k] = k < pc.row_bytes ? sr[k] : 0;
      }
    }
  }
}

// Launches copy_pieces_kernel over `pcs` (host vector) through a pool-allocated device table,
// freed in stream order.
int copy_pieces(const std::vector<DevPiece>& pcs, cudaStream_t s) {
  if (pcs.empty()) return 0;
  DevPiece* d = nullptr;
  if (pool_alloc(reinterpret_cast<void**>(&d), sizeof(DevPiece) * pcs.size(), s) != 0) return POGS_ERR_OOM;
  int rc = 0;
  if (cudaMemcpyAsync(d, pcs.data(), sizeof(DevPiece) * pcs.size(), cudaMemcpyHostToDevice, s) != cudaSuccess) {
    rc = POGS_ERR_CUDA;
  } else {
    count_launch();
    const int grid = (int)std::min<size_t>(pcs.size(), 148 * 16);
    copy_pieces_kernel<<<grid, 256, 0, s>>>(d, (int)pcs.size());
    if (cudaGetLastError() != cudaSuccess) rc = POGS_ERR_CUDA;
  }
  cudaGetLastError();
  cudaFreeAsync(d, s);
  return rc;
}

// Returned tuples of all instances into one device buffer (x, y, mu, nu of instance k at
// out_off[k]), one CTA per instance, for a single copy to the host.
__global__ void gather_out_kernel(const BInst* __restrict__ insts, const size_t* __restrict__ out_off, float* dst) {
  const BInst& I = insts[blockIdx.x];
  float* d = dst + out_off[blockIdx.x];
  const float* src[4] = {I.ox, I.oy, I.omu, I.onu};
  const int len[4] = {I.n, I.m, I.n, I.m};
  for (int t = 0; t < 4; ++t) {
    for (int i = threadIdx.x; i < len[t]; i += blockDim.x) d[i] = src[t][i];
    d += len[t];
  }
}

// Launch configurations the tuner chooses between; none changes per-instance arithmetic.
struct LaunchCfg {
  int grid_mult;     // resident CTAs per SM
  int smem;          // shared-memory budget for staging an instance's matrix (0: stream from L2)
  int largest_first; // schedule order
};
// (CTAs per SM, shared-memory budget for the matrix, largest first).  Each CTA also holds 24 KB of
// staged vectors and 13 KB of reduction buffers, so the candidates fill the SM's 228 KB.
const LaunchCfg kCandidates[] = {{1, 184 * 1024, 1}, {2, 76 * 1024, 1}, {2, 0, 1},
                                 {4, 0, 1},          {3, 36 * 1024, 1}, {2, 76 * 1024, 0}};
std::map<std::tuple<int, int, int>, LaunchCfg> g_tuned;
std::mutex g_tuned_mu;

#define BCK(call)                                   \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) {                        \
      cudaGetLastError();                           \
      rc = (e_ == cudaErrorMemoryAllocation) ? POGS_ERR_OOM : POGS_ERR_CUDA; \
      goto done;                                    \
    }                                               \
  } while (0)

}  // namespace

extern "C" int pogs_solve_batch(int count, const pogs_problem* probs, const pogs_params* p, pogs_result* out,
                                void* stream) {
  if (count < 0 || (count > 0 && (!probs || !out))) return POGS_ERR_ARG;
  pogs_params def;
  pogs_default_params(&def);
  if (!p) p = &def;
  for (int i = 0; i < count; ++i) {
    const pogs_problem& pr = probs[i];
    if (!pr.A || pr.m < 1 || pr.n < 1 || pr.lda < pr.n || !pr.f.h || !pr.g.h) return POGS_ERR_ARG;
    memset(&out[i].info, 0, sizeof(pogs_info));
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<int> small, large;
  for (int i = 0; i < count; ++i) (std::min(probs[i].m, probs[i].n) <= kMaxBatchQ ? small : large).push_back(i);
  int worst = 0;
  // ---- large problems: the single-problem path -------------------------------------------
  for (int i : large) {
    pogs_handle* h = nullptr;
    const pogs_problem& pr = probs[i];
    int rc = pogs_setup(pr.A, pr.m, pr.n, pr.lda, 'R', p, stream, &h);
    if (rc == 0) {
      rc = pogs_solve(h, &pr.f, &pr.g, p, out[i].x, out[i].y, out[i].mu, out[i].nu, &out[i].info);
      pogs_free(h);
    }
    out[i].info.status = rc;
    if (rc == POGS_MAX_ITER) worst = std::max(worst, 1);
    if (rc < 0 && rc != POGS_ERR_ARG && rc != POGS_ERR_NONFINITE && rc != POGS_ERR_NUMERIC) return rc;
  }
  if (small.empty()) return worst;

  // ---- small problems: arena layout (inputs first, contiguous, so host inputs go in one copy)
  const int ns = (int)small.size();
  std::vector<BInst> inst(ns);
  std::vector<size_t> offA(ns), offM(ns), offH(ns), offD(ns), offE(ns), offIn(ns * 12), offF(ns * 12), offV(ns);
  size_t cur = 0;
  for (int k = 0; k < ns; ++k) {
    const pogs_problem& pr = probs[small[k]];
    const int lda4 = (int)round_up(pr.n, 4);
    offA[k] = cur;
    cur = al(cur + (size_t)pr.m * lda4 * 4);
    for (int t = 0; t < 12; ++t) {   // raw f: h,a..e (m) then g: h,a..e (n)
      const int64_t len = t < 6 ? pr.m : pr.n;
      offIn[k * 12 + t] = cur;
      cur = al(cur + (size_t)len * ((t % 6) == 0 ? 1 : 4));
    }
  }
  const size_t in_end = cur;
  for (int k = 0; k < ns; ++k) {
    const pogs_problem& pr = probs[small[k]];
    const int64_t q = std::min(pr.m, pr.n), vlen = round_up(std::max(pr.m, pr.n), 4);   // 16-byte vectors
    offM[k] = cur;
    cur = al(cur + (size_t)q * q * 4);
    offH[k] = cur;
    cur = al(cur + (size_t)q * q * 8);
    offD[k] = cur;
    cur = al(cur + (size_t)pr.m * 4);
    offE[k] = cur;
    cur = al(cur + (size_t)pr.n * 4);
    for (int t = 0; t < 12; ++t) {
      const int64_t len = t < 6 ? pr.m : pr.n;
      offF[k * 12 + t] = cur;
      cur = al(cur + (size_t)len * ((t % 6) == 0 ? 1 : 4));
    }
    offV[k] = cur;
    cur = al(cur + (size_t)17 * vlen * 4);
  }
  const size_t total = cur;

  int rc = 0;
  char* arena = nullptr;
  BInst* d_inst = nullptr;
  BOut* d_out = nullptr;
  int *d_queue = nullptr, *d_order = nullptr;
  std::vector<char> stage;
  std::unique_lock<std::mutex> pin_lock;
  char* hst = nullptr;                 // staging for host inputs and outputs (pinned or `stage`)
  std::vector<size_t> out_off(ns + 1, 0);
  size_t* d_outoff = nullptr;
  float* d_gather = nullptr;
  bool any_host_out = false;
  std::vector<BOut> hout(ns);
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaStream_t cap = nullptr;
  BCfg cfg;
  LaunchCfg lc = kCandidates[0];
  int num_sms = 148, dev = 0;
  std::vector<int> order_big(ns), order_in(ns);
  bool any_host_in = false;
  std::vector<char> dev_out((size_t)ns * 4);   // per output array: on the device (1) or the host (0)
  // stream-ordered allocations from the library's pool (no device-wide synchronisation)
  if (pool_alloc(reinterpret_cast<void**>(&arena), total, s) != 0 ||
      pool_alloc(reinterpret_cast<void**>(&d_inst), sizeof(BInst) * ns, s) != 0 ||
      pool_alloc(reinterpret_cast<void**>(&d_out), sizeof(BOut) * ns, s) != 0 ||
      pool_alloc(reinterpret_cast<void**>(&d_queue), sizeof(int), s) != 0 ||
      pool_alloc(reinterpret_cast<void**>(&d_order), sizeof(int) * ns, s) != 0) {
    rc = POGS_ERR_OOM;
    goto done;
  }
  BCK(cudaMemsetAsync(d_out, 0, sizeof(BOut) * ns, s));
  // ---- ingest -------------------------------------------------------------------------------
  // Device inputs are copied device to device; host inputs are packed (row pitch padded to four
  // floats) into one staging buffer by several host threads and copied in one transfer when every
  // input is on the host, else region by region.
  {
    std::vector<char> dev_A(ns);
    std::vector<char> dev_in((size_t)ns * 12);
    bool all_host = true;
    for (int k = 0; k < ns; ++k) {
      const pogs_problem& pr = probs[small[k]];
      const void* src[12] = {pr.f.h, pr.f.a, pr.f.b, pr.f.c, pr.f.d, pr.f.e, pr.g.h, pr.g.a, pr.g.b, pr.g.c, pr.g.d, pr.g.e};
      dev_A[k] = is_dev(pr.A);
      any_host_in |= !dev_A[k];
      all_host &= !dev_A[k];
      for (int t = 0; t < 12; ++t) {
        dev_in[(size_t)k * 12 + t] = src[t] ? is_dev(src[t]) : 0;
        any_host_in |= src[t] && !dev_in[(size_t)k * 12 + t];
        all_host &= !src[t] || !dev_in[(size_t)k * 12 + t];
      }
    }
    for (int k = 0; k < ns; ++k) {
      const pogs_problem& pr = probs[small[k]];
      out_off[k + 1] = out_off[k] + 2 * (size_t)(pr.n + pr.m);
      const pogs_result& r = out[small[k]];
      const float* dsts[4] = {r.x, r.y, r.mu, r.nu};
      for (int t = 0; t < 4; ++t) {
        dev_out[(size_t)k * 4 + t] = dsts[t] ? is_dev(dsts[t]) : 0;
        any_host_out |= dsts[t] && !dev_out[(size_t)k * 4 + t];
      }
    }
    const size_t need = std::max(any_host_in ? in_end : 0, any_host_out ? out_off[ns] * 4 : 0);
    if (need > 0) {
      hst = pinned(pin_lock, need);
      if (!hst) {
        stage.resize(need);
        hst = stage.data();
      }
    }
    if (any_host_in) {
      parallel_for(ns, [&](int k) {
        const pogs_problem& pr = probs[small[k]];
        const int lda4 = (int)round_up(pr.n, 4);
        if (!dev_A[k])
          for (int64_t i = 0; i < pr.m; ++i) {
            char* row = hst + offA[k] + (size_t)i * lda4 * 4;
            memcpy(row, pr.A + i * pr.lda, (size_t)pr.n * 4);
            if (lda4 > pr.n) memset(row + (size_t)pr.n * 4, 0, (size_t)(lda4 - pr.n) * 4);
          }
        const void* src[12] = {pr.f.h, pr.f.a, pr.f.b, pr.f.c, pr.f.d, pr.f.e, pr.g.h, pr.g.a, pr.g.b, pr.g.c, pr.g.d, pr.g.e};
        for (int t = 0; t < 12; ++t)
          if (src[t] && !dev_in[(size_t)k * 12 + t])
            memcpy(hst + offIn[k * 12 + t], src[t], (size_t)(t < 6 ? pr.m : pr.n) * ((t % 6) == 0 ? 1 : 4));
      });
    }
    // host regions: the whole packed input region in one transfer (the parts that belong to device
    // inputs carry nothing and are overwritten next, in stream order); device regions: one launch
    if (any_host_in) BCK(cudaMemcpyAsync(arena, hst, in_end, cudaMemcpyHostToDevice, s));
    if (!all_host) {
      std::vector<DevPiece> pcs;
      pcs.reserve((size_t)ns * 13);
      for (int k = 0; k < ns; ++k) {
        const pogs_problem& pr = probs[small[k]];
        const int lda4 = (int)round_up(pr.n, 4);
        if (dev_A[k])
          pcs.push_back(DevPiece{reinterpret_cast<const char*>(pr.A), arena + offA[k], pr.m, pr.n * 4, pr.lda * 4,
                                 (int64_t)lda4 * 4, (int64_t)lda4 * 4});
        const void* src[12] = {pr.f.h, pr.f.a, pr.f.b, pr.f.c, pr.f.d, pr.f.e, pr.g.h, pr.g.a, pr.g.b, pr.g.c, pr.g.d, pr.g.e};
        for (int t = 0; t < 12; ++t) {
          if (!src[t] || !dev_in[(size_t)k * 12 + t]) continue;
          const int64_t bytes = (t < 6 ? pr.m : pr.n) * ((t % 6) == 0 ? 1 : 4);
          pcs.push_back(DevPiece{static_cast<const char*>(src[t]), arena + offIn[k * 12 + t], 1, bytes, bytes, bytes, bytes});
        }
      }
      rc = copy_pieces(pcs, s);
      if (rc != 0) goto done;
    }
  }
  for (int k = 0; k < ns; ++k) {
    const pogs_problem& pr = probs[small[k]];
    BInst& I = inst[k];
    memset(&I, 0, sizeof(I));
    I.m = (int)pr.m;
    I.n = (int)pr.n;
    I.lda = (int)round_up(pr.n, 4);
    I.q = (int)std::min(pr.m, pr.n);
    I.tall = pr.m >= pr.n;
    I.A = reinterpret_cast<float*>(arena + offA[k]);
    I.M = reinterpret_cast<float*>(arena + offM[k]);
    I.H = reinterpret_cast<double*>(arena + offH[k]);
    I.D = reinterpret_cast<float*>(arena + offD[k]);
    I.E = reinterpret_cast<float*>(arena + offE[k]);
    const void* src[12] = {pr.f.h, pr.f.a, pr.f.b, pr.f.c, pr.f.d, pr.f.e, pr.g.h, pr.g.a, pr.g.b, pr.g.c, pr.g.d, pr.g.e};
    auto in = [&](int t) -> void* { return src[t] ? (void*)(arena + offIn[k * 12 + t]) : nullptr; };
    I.fh0 = (const uint8_t*)in(0); I.fa0 = (const float*)in(1); I.fb0 = (const float*)in(2);
    I.fc0 = (const float*)in(3); I.fd0 = (const float*)in(4); I.fe0 = (const float*)in(5);
    I.gh0 = (const uint8_t*)in(6); I.ga0 = (const float*)in(7); I.gb0 = (const float*)in(8);
    I.gc0 = (const float*)in(9); I.gd0 = (const float*)in(10); I.ge0 = (const float*)in(11);
    auto fo = [&](int t) { return arena + offF[k * 12 + t]; };
    I.fh = (uint8_t*)fo(0); I.fa = (float*)fo(1); I.fb = (float*)fo(2); I.fc = (float*)fo(3); I.fd = (float*)fo(4);
    I.fe = (float*)fo(5);
    I.gh = (uint8_t*)fo(6); I.ga = (float*)fo(7); I.gb = (float*)fo(8); I.gc = (float*)fo(9); I.gd = (float*)fo(10);
    I.ge = (float*)fo(11);
    const int64_t vlen = round_up(std::max(pr.m, pr.n), 4);   // the iteration reads some vectors as float4
    float* v = reinterpret_cast<float*>(arena + offV[k]);
    float** vecs[] = {&I.x, &I.y, &I.xt, &I.yt, &I.xh, &I.yh, &I.cx, &I.dy, &I.mu, &I.nu, &I.r, &I.z, &I.w,
                      &I.ox, &I.oy, &I.omu, &I.onu};
    for (int t = 0; t < 17; ++t) *vecs[t] = v + (size_t)t * vlen;
    I.out = d_out + k;
    I.loop = nullptr;
  }
  // ---- configuration ------------------------------------------------------------------------
  memset(&cfg, 0, sizeof(cfg));
  cfg.abs_tol = p->abs_tol;
  cfg.rel_tol = p->rel_tol;
  cfg.rho0 = p->rho0;
  cfg.alpha = p->alpha;
  cfg.delta = p->delta;
  cfg.tau = p->tau;
  cfg.gamma_scale = p->gamma;
  cfg.max_iter = p->max_iter;
  cfg.gap_stop = p->gap_stop;
  cfg.adaptive = p->adaptive_rho;
  cfg.sk_sweeps = p->sk_sweeps;
  cfg.equil = p->equil;
  cfg.mixed_chol = p->chol_prec == POGS_CHOL_MIXED;
  BCK(cudaGetDevice(&dev));
  BCK(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
  std::iota(order_in.begin(), order_in.end(), 0);
  order_big = order_in;
  std::stable_sort(order_big.begin(), order_big.end(), [&](int a, int b) {
    return (int64_t)inst[a].m * inst[a].n > (int64_t)inst[b].m * inst[b].n;
  });
  BCK(cudaMemcpyAsync(d_inst, inst.data(), sizeof(BInst) * ns, cudaMemcpyHostToDevice, s));
  rc = batch_setup(d_inst, ns, cfg, s);
  if (rc != 0) goto done;
  {
    // size class of this batch: log2 of the count, of the largest q and of the mean m n
    double mn = 0;
    int qmax = 0;
    for (auto& I : inst) {
      mn += (double)I.m * I.n;
      qmax = std::max(qmax, I.q);
    }
    const auto key = std::make_tuple((int)std::log2(ns + 1.0), (int)std::log2(qmax + 1.0), (int)std::log2(mn / ns + 1.0));
    bool have = false;
    {
      std::lock_guard<std::mutex> g(g_tuned_mu);
      auto it = g_tuned.find(key);
      if (it != g_tuned.end()) {
        lc = it->second;
        have = true;
      }
    }
    if (!have && ns >= 32) {
      // time each candidate on this batch: 20 iterations of every instance, stopping disabled
      BCfg tc = cfg;
      tc.max_iter = std::min(20, cfg.max_iter);
      tc.abs_tol = 0.0;
      tc.rel_tol = 0.0;
      cudaEvent_t e0, e1;
      BCK(cudaEventCreate(&e0));
      BCK(cudaEventCreate(&e1));
      float best = 1e30f;
      for (const LaunchCfg& c : kCandidates) {
        for (auto& I : inst) I.stage_smem = c.smem > 0 && (int64_t)I.m * I.lda * 4 <= c.smem;
        BCK(cudaMemcpyAsync(d_inst, inst.data(), sizeof(BInst) * ns, cudaMemcpyHostToDevice, s));
        BCK(cudaMemcpyAsync(d_order, (c.largest_first ? order_big : order_in).data(), sizeof(int) * ns,
                            cudaMemcpyHostToDevice, s));
        BCK(cudaMemsetAsync(d_queue, 0, sizeof(int), s));
        BCK(cudaEventRecord(e0, s));
        rc = batch_iterate(d_inst, ns, tc, d_queue, d_order, num_sms * c.grid_mult, c.smem, 0, s);
        if (rc != 0) goto done;
        BCK(cudaEventRecord(e1, s));
        BCK(cudaEventSynchronize(e1));
        float ms = 0;
        BCK(cudaEventElapsedTime(&ms, e0, e1));
        if (p->verbose > 1)
          fprintf(stderr, "pogs batch tune: grid %dx%d smem %d order %d: %.3f ms\n", c.grid_mult, num_sms, c.smem,
                  c.largest_first, ms);
        if (ms < best) {
          best = ms;
          lc = c;
        }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      std::lock_guard<std::mutex> g(g_tuned_mu);
      g_tuned[key] = lc;
    }
  }
  for (auto& I : inst) I.stage_smem = lc.smem > 0 && (int64_t)I.m * I.lda * 4 <= lc.smem;
  BCK(cudaMemcpyAsync(d_inst, inst.data(), sizeof(BInst) * ns, cudaMemcpyHostToDevice, s));
  BCK(cudaMemcpyAsync(d_order, (lc.largest_first ? order_big : order_in).data(), sizeof(int) * ns,
                      cudaMemcpyHostToDevice, s));
  // the persistent launch (with its queue reset) runs as one captured CUDA graph
  BCK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  BCK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
  ++g_capture_depth;
  cudaMemsetAsync(d_queue, 0, sizeof(int), cap);
  rc = batch_iterate(d_inst, ns, cfg, d_queue, d_order, num_sms * lc.grid_mult, lc.smem, 0, cap);
  --g_capture_depth;
  BCK(cudaStreamEndCapture(cap, &graph));
  if (rc != 0) goto done;
  BCK(cudaGraphInstantiate(&gexec, graph, 0));
  BCK(cudaGraphLaunch(gexec, s));
  count_launch(1);
  // ---- results ------------------------------------------------------------------------------
  BCK(cudaMemcpyAsync(hout.data(), d_out, sizeof(BOut) * ns, cudaMemcpyDeviceToHost, s));
  // device destinations directly; host ones gathered on the device, copied in one transfer and
  // scattered by several host threads
  {
    std::vector<DevPiece> pcs;
    for (int k = 0; k < ns; ++k) {
      pogs_result& r = out[small[k]];
      const BInst& I = inst[k];
      const float* srcs[4] = {I.ox, I.oy, I.omu, I.onu};
      float* dsts[4] = {r.x, r.y, r.mu, r.nu};
      const int64_t bytes[4] = {(int64_t)I.n * 4, (int64_t)I.m * 4, (int64_t)I.n * 4, (int64_t)I.m * 4};
      for (int t = 0; t < 4; ++t)
        if (dsts[t] && dev_out[(size_t)k * 4 + t])
          pcs.push_back(DevPiece{reinterpret_cast<const char*>(srcs[t]), reinterpret_cast<char*>(dsts[t]), 1,
                                 bytes[t], bytes[t], bytes[t], bytes[t]});
    }
    rc = copy_pieces(pcs, s);
    if (rc != 0) goto done;
  }
  if (any_host_out) {
    if (pool_alloc(reinterpret_cast<void**>(&d_outoff), sizeof(size_t) * ns, s) != 0 ||
        pool_alloc(reinterpret_cast<void**>(&d_gather), out_off[ns] * 4, s) != 0) {
      rc = POGS_ERR_OOM;
      goto done;
    }
    BCK(cudaMemcpyAsync(d_outoff, out_off.data(), sizeof(size_t) * ns, cudaMemcpyHostToDevice, s));
    count_launch();
    gather_out_kernel<<<ns, 256, 0, s>>>(d_inst, d_outoff, d_gather);
    BCK(cudaGetLastError());
    BCK(cudaMemcpyAsync(hst, d_gather, out_off[ns] * 4, cudaMemcpyDeviceToHost, s));
  }
  BCK(cudaStreamSynchronize(s));
  if (any_host_out)
    parallel_for(ns, [&](int k) {
      pogs_result& r = out[small[k]];
      const pogs_problem& pr = probs[small[k]];
      const float* src = reinterpret_cast<const float*>(hst) + out_off[k];
      float* dsts[4] = {r.x, r.y, r.mu, r.nu};
      const int64_t lens[4] = {pr.n, pr.m, pr.n, pr.m};
      for (int t = 0; t < 4; ++t) {
        if (dsts[t] && !dev_out[(size_t)k * 4 + t]) memcpy(dsts[t], src, (size_t)lens[t] * 4);
        src += lens[t];
      }
    });
  for (int k = 0; k < ns; ++k) {
    pogs_info& info = out[small[k]].info;
    const BOut& o = hout[k];
    info.status = o.status;
    info.iters = o.iters;
    info.rho = o.rho;
    info.r_pri = o.r_pri;
    info.r_dual = o.r_dual;
    info.eps_pri = o.eps_pri;
    info.eps_dual = o.eps_dual;
    info.gap = o.gap;
    info.obj = o.obj;
    info.r_pri_unscaled = o.r_pri_u;
    info.r_dual_unscaled = o.r_dual_u;
    if (o.status == POGS_MAX_ITER) worst = std::max(worst, 1);
  }
  rc = worst;
done:
  if (gexec) cudaGraphExecDestroy(gexec);
  if (graph) cudaGraphDestroy(graph);
  if (cap) cudaStreamDestroy(cap);
  if (arena) cudaFreeAsync(arena, s);
  if (d_inst) cudaFreeAsync(d_inst, s);
  if (d_out) cudaFreeAsync(d_out, s);
  if (d_queue) cudaFreeAsync(d_queue, s);
  if (d_order) cudaFreeAsync(d_order, s);
  if (d_outoff) cudaFreeAsync(d_outoff, s);
  if (d_gather) cudaFreeAsync(d_gather, s);
  cudaStreamSynchronize(s);
  return rc;
}
