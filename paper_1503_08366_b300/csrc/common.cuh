// Shared device helpers, device-side solver state and launch constants.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>

#include "../../include/pogs.h"

#define POGS_DEV __device__ __forceinline__

namespace pogs {

constexpr int kWarp = 32;
constexpr int kTile = 128;          // packed-triangle tile edge (L^{-1} storage)
constexpr int kLdaAlign = 32;       // row pitch of A^ in floats (128 bytes)

// Scalars of the ADMM loop that live on the device (Algorithm 1 + Algorithm 3).
struct DevState {
  double rho;         // rho^k
  double pend;        // pending rescale factor rho^{k-1}/rho^k for x~, y~ (applied on read)
  double r_pri, r_dual, eps_pri, eps_dual, gap, obj;
  double r_pri_u, r_dual_u;
  int k;              // iteration counter
  int l, u;           // Algorithm 3 bookkeeping
  int done;           // 1 once converged / max_iter / error
  int status;         // POGS_OK, POGS_MAX_ITER, or negative error
  int err;            // device-side error flag (e.g. NUMERIC pivot, TIMEOUT)
  int pad_;
};

// Parameters read by the check kernel (copied by value into the launch).
struct LoopParams {
  double abs_tol, rel_tol, alpha, delta, tau;
  int max_iter, gap_stop, adaptive;
};

// Per-element function parameters (pre-conditioned), structure of arrays.
struct FnDev {
  const uint8_t* h;
  const float *a, *b, *c, *d, *e;
};

// ---- reductions -------------------------------------------------------------------------
POGS_DEV float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
POGS_DEV double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---- double-float accumulation -------------------------------------------------------------
// Sums that must keep more digits than FP32 (norms, gap terms, objective partials) are carried
// as an unevaluated pair hi + lo of FP32 numbers and updated with error-free transformations:
// Knuth's TwoSum for additions and the exact rounding error of a product recovered with one
// FMA.  That keeps about 48 significant bits using only the FP32 pipes (B300's FP64 rate is a
// small fraction of its FP32 rate); per-warp results are converted to FP64 once.
struct Df {
  float hi, lo;
};
POGS_DEV void df_add(Df& a, float x) {
  const float s = __fadd_rn(a.hi, x);
  const float bb = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
  a.hi = s;
  a.lo = __fadd_rn(a.lo, e);
}
POGS_DEV void df_add(Df& a, const Df& b) {
  df_add(a, b.hi);
  a.lo = __fadd_rn(a.lo, b.lo);
}
POGS_DEV void df_add_prod(Df& a, float x, float y) {   // a += x y
  const float p = __fmul_rn(x, y);
  const float pe = __fmaf_rn(x, y, -p);   // exact: x y - p
  df_add(a, p);
  a.lo = __fadd_rn(a.lo, pe);
}
POGS_DEV double df_value(const Df& a) { return (double)a.hi + (double)a.lo; }
// (hi, lo) <- (hi, lo) - x exactly up to the final rounding of the pair: TwoSum of hi and -x
// (the rounding error e of s = hi - x is recovered exactly), then Fast2Sum of s and lo + e.
POGS_DEV void df_sub(float& hi, float& lo, float x) {
  const float s = __fsub_rn(hi, x);
  const float bb = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(-x, bb));
  const float t = __fadd_rn(lo, e);
  hi = __fadd_rn(s, t);
  lo = __fsub_rn(t, __fsub_rn(hi, s));
}

// Block-wide sum of NV double-float values per thread: a fixed xor-shuffle tree on the FP32
// pipes inside each warp, then the same across the per-warp results in warp 0 (no serial FP64
// chain); `out` valid in thread 0; `sh` holds NV * (blockDim/32) doubles (used as double-float
// pairs).  Deterministic.
template <int NV>
POGS_DEV void block_sum_df(Df (&v)[NV], double (&out)[NV], double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  Df* sd = reinterpret_cast<Df*>(sh);
#pragma unroll
  for (int t = 0; t < NV; ++t) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const Df b{__shfl_xor_sync(0xffffffffu, v[t].hi, o), __shfl_xor_sync(0xffffffffu, v[t].lo, o)};
      df_add(v[t], b);
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int t = 0; t < NV; ++t) sd[t * nw + wid] = v[t];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int t = 0; t < NV; ++t) {
      Df a = lane < nw ? sd[t * nw + lane] : Df{0.0f, 0.0f};
      for (int o = 1; o < nw; o <<= 1) {
        const Df b{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
        df_add(a, b);
      }
      out[t] = df_value(a);
    }
  }
  __syncthreads();
}

// Block-wide FP64 sum of NV values per thread; result valid in thread 0. `sh` holds
// NV * (blockDim/32) doubles. Deterministic (fixed shuffle tree + fixed warp order).
template <int NV>
POGS_DEV void block_sum(double (&v)[NV], double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int t = 0; t < NV; ++t) v[t] = warp_sum(v[t]);
  if (lane == 0) {
#pragma unroll
    for (int t = 0; t < NV; ++t) sh[t * nw + wid] = v[t];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int t = 0; t < NV; ++t) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += sh[t * nw + w];
      v[t] = s;
    }
  }
  __syncthreads();
}

// L2 policy marking lines as the first to evict: for matrices streamed once per pass (far
// larger than L2), so that what a pass writes for its next launch (split partial sums) and the
// vectors it reads stay in L2 instead of being pushed out by the stream.
POGS_DEV uint64_t l2_evict_first() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

// L2 policy marking lines as the last to evict: for the leading rows of a matrix that every
// pass reads, so that they stay in L2 from one pass to the next while the rest streams.
POGS_DEV uint64_t l2_evict_last() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

// Streamed load (no L1 allocation) under an L2 policy from l2_evict_first() or l2_evict_last().
POGS_DEV float4 ldg_stream(const float4* p, uint64_t pol) {
  float4 r;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
               : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
               : "l"(p), "l"(pol));
  return r;
}

POGS_DEV float4 ldg_stream(const float4* p) {
  float4 r;
  asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
               : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
               : "l"(p));
  return r;
}

// "Last block done" protocol: every block of a group publishes its partial results,
// fences, and bumps the group's counter; the block that brings the counter to `total`
// reduces the partials in a fixed order and resets the counter for the next launch.
POGS_DEV bool arrive_last(unsigned* counter, unsigned total) {
  __shared__ unsigned s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned prev = atomicAdd(counter, 1u);
    s_last = (prev == total - 1) ? 1u : 0u;
    if (s_last) *counter = 0u;   // reset for the next use (no other block touches it now)
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last != 0;
}

// Process-wide count of kernel launches issued by this library (graph replays are added by
// the caller from the number of iterations executed; launches recorded during stream capture
// are not counted).
extern std::atomic<long long> g_launch_count;
extern thread_local int g_capture_depth;
inline void count_launch(int k = 1) {
  if (g_capture_depth == 0) g_launch_count.fetch_add(k, std::memory_order_relaxed);
}

// Process-wide count of device memory allocations requested by this library (pool
// allocations and cudaMalloc / cudaMallocAsync calls).
extern std::atomic<long long> g_alloc_count;
inline void count_alloc(int k = 1) { g_alloc_count.fetch_add(k, std::memory_order_relaxed); }

// Runs a set-up step (a cudaFuncSetAttribute call, say) once per device: function attributes
// belong to a device's context, so a process that uses several devices needs the call on each.
// Thread-safe; a step that fails is retried on the next call.
struct PerDeviceOnce {
  static constexpr int kMaxDevices = 64;
  std::mutex mu;
  bool done[kMaxDevices] = {};
  template <class Fn>
  int run(Fn fn) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
      cudaGetLastError();
      return -1;
    }
    std::lock_guard<std::mutex> lk(mu);
    if (done[dev]) return 0;
    const int rc = fn();
    if (rc == 0) done[dev] = true;
    return rc;
  }
};

inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }
inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace pogs
