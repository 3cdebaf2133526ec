// Tensor-core Gram formation (Section 3.5: forming A^T A or A A^T dominates the setup) and a
// general K-major tcgen05 GEMM used by it.
//
//   G = X X^T,  X = A^T (q = n, m >= n) or X = A (q = m, m < n),  lower 128 x 128 tiles only.
//
// Operands are packed once into K-major, zero-padded buffers (rows to 128, K to one TMA box):
//   BF16:    X_hi = bf16(X)                                  one MMA per K step
//   BF16x3:  X_hi = bf16(X), X_lo = bf16(X - X_hi)           hi.hi + hi.lo + lo.hi per K step
//   TF32:    X rounded to TF32 (kept in 32-bit words)        one kind::tf32 MMA per K step
//   TF32x3:  X_hi = tf32(X), X_lo = tf32(X - X_hi)           hi.hi + hi.lo + lo.hi per K step
//            (about 21 significant bits per product; the triangular inverse's GEMMs)
// FP32 accumulation in tensor memory, drained in K chunks.  One CTA computes one 128 x 128
// output tile: one thread streams X tiles with TMA through a multi-stage shared-memory ring
// (128-byte swizzle), one thread issues tcgen05.mma, four warps read the accumulator back with
// tcgen05.ld.
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <cstdio>
#include <cstring>

#include "kernels.h"
#include "tc.cuh"

namespace pogs {

namespace {

constexpr int kTileRows = 128;   // M = N = 128 per CTA
constexpr int kTileBytes = kTileRows * 128;   // one operand tile: 128 rows x 128 bytes

enum TcMode : int { TC_BF16 = 0, TC_BF16X3 = 1, TC_TF32 = 2, TC_TF32X3 = 3 };

template <int MODE>
struct TcCfg {
  static constexpr bool kSplit = MODE == TC_BF16X3 || MODE == TC_TF32X3;   // hi/lo operand pairs
  static constexpr bool kTf32 = MODE == TC_TF32 || MODE == TC_TF32X3;
  static constexpr int kOps = kSplit ? 4 : 2;                        // operand tiles per stage
  static constexpr int kStages = kSplit ? 3 : 6;
  static constexpr int kStageBytes = kOps * kTileBytes;
  static constexpr int kElemsPerBox = kTf32 ? 32 : 64;               // K elements per 128-byte row
  static constexpr int kMmaPerBox = 4;                              // 32 bytes of K per MMA
  static constexpr size_t kSmem = (size_t)kStages * kStageBytes + 1024 + 256;
};

struct TcArgs {
  int nkb;                 // K boxes
  int tiles;               // tiles along M (and N, lower_only)
  int tiles_n;             // tiles along N (full grid)
  int lower_only;          // enumerate the lower triangle of tiles
  int kskip;               // X, Y are lower triangular in K (X[i][k] = 0 for k < i): tile (ti, tj) starts
                           // its K loop at 128 max(ti, tj)
  int64_t M, N;            // valid output extent
  float* C;                // FP32 output (epi 0), hi part of the pair (epi 2)
  float* Clo;              // lo part of the double-float pair (epi 2)
  double* C64;             // FP64 output (epi 1: C64 += alpha * acc, lower triangle)
  int64_t ldc;
  double alpha;            // epi 0: C = alpha * acc; epi 1: C64 += alpha * acc; epi 2: (C, Clo) -= acc
  int epi;
  int* err;
};

// Warp roles (192 threads): warp 0 lane 0 -- TMA producer; warp 1 lane 0 -- MMA issuer;
// warps 2..5 -- epilogue, warp w reading TMEM lanes 32 (w % 4) .. 32 (w % 4) + 31 (rows of the
// tile).  The tensor-core accumulator is double-buffered in TMEM (2 x 128 columns) and
// restarted every kChunk K boxes: the epilogue warps drain each finished chunk into FP32
// registers with round-to-nearest adds while the next chunk accumulates.  The accumulator
// adds inside the tensor core are not round-to-nearest, so an undrained sum over K carries
// a bias that grows linearly with K; chunking bounds it to the chunk length.
constexpr int kChunkBoxes = 8;   // 512 BF16 / 256 TF32 elements of K per accumulator chunk

template <int MODE>
__global__ void __launch_bounds__(192, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mxh, const __grid_constant__ CUtensorMap mxl,
                   const __grid_constant__ CUtensorMap myh, const __grid_constant__ CUtensorMap myl, TcArgs a) {
  using Cfg = TcCfg<MODE>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + Cfg::kStages * Cfg::kStageBytes);
  uint64_t* empty = full + Cfg::kStages;
  uint64_t* acc_full = empty + Cfg::kStages;   // [2]: chunk in buffer b complete (MMA -> epilogue)
  uint64_t* acc_empty = acc_full + 2;          // [2]: buffer b drained (epilogue -> MMA)
  uint64_t* drain = acc_empty + 2;             // all MMAs of this CTA complete (teardown)
  uint32_t* tslot = reinterpret_cast<uint32_t*>(drain + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  int ti, tj;
  if (a.lower_only) {
    const int b = blockIdx.x;
    int i = (int)((sqrtf(8.0f * (float)b + 1.0f) - 1.0f) * 0.5f);
    while ((i + 1) * (i + 2) / 2 <= b) ++i;
    while (i * (i + 1) / 2 > b) --i;
    ti = i;
    tj = b - i * (i + 1) / 2;
  } else {
    ti = blockIdx.x / a.tiles_n;
    tj = blockIdx.x % a.tiles_n;
  }
  // K boxes of this tile: [kb0, kb0 + nkb)
  const int kb0 = a.kskip ? (max(ti, tj) * kTileRows) / Cfg::kElemsPerBox : 0;
  const int nkb = a.nkb - kb0;
  const int nchunks = (nkb + kChunkBoxes - 1) / kChunkBoxes;

  if (threadIdx.x == 0) {
    for (int s = 0; s < Cfg::kStages; ++s) {
      tc::mbar_init(full + s, 1);
      tc::mbar_init(empty + s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(acc_full + b, 1);
      tc::mbar_init(acc_empty + b, 4);   // one arrival per epilogue warp
    }
    tc::mbar_init(drain, 1);
    tc::fence_mbar_init();
  }
  if (warp == 1) {
    tc::tmem_alloc(tslot, 256);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    if (lane == 0) {
      // ---- TMA producer ---------------------------------------------------------------------
      tc::prefetch_tmap(&mxh);
      tc::prefetch_tmap(&myh);
      if (Cfg::kSplit) {
        tc::prefetch_tmap(&mxl);
        tc::prefetch_tmap(&myl);
      }
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % Cfg::kStages;
        const uint32_t ph = (uint32_t)(kb / Cfg::kStages) & 1u;
        if (kb >= Cfg::kStages && !tc::mbar_wait(empty + s, ph ^ 1u)) {
          atomicCAS(a.err, 0, POGS_ERR_TIMEOUT);
          break;
        }
        uint8_t* st = smem + s * Cfg::kStageBytes;
        tc::mbar_arrive_expect_tx(full + s, Cfg::kStageBytes);
        const int x = (kb0 + kb) * Cfg::kElemsPerBox;
        tc::tma_load_2d(st, &mxh, x, ti * kTileRows, full + s);
        tc::tma_load_2d(st + kTileBytes, &myh, x, tj * kTileRows, full + s);
        if (Cfg::kSplit) {
          tc::tma_load_2d(st + 2 * kTileBytes, &mxl, x, ti * kTileRows, full + s);
          tc::tma_load_2d(st + 3 * kTileBytes, &myl, x, tj * kTileRows, full + s);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer ---------------------------------------------------------------------------
      bool ok = true;
      for (int c = 0; c < nchunks && ok; ++c) {
        const int buf = c & 1;
        const uint32_t d = tmem + (uint32_t)(buf * 128);
        if (c >= 2 && !tc::mbar_wait(acc_empty + buf, (uint32_t)((c >> 1) - 1) & 1u)) {
          ok = false;
          break;
        }
        tc::fence_after_sync();
        const int kb1 = min(nkb, (c + 1) * kChunkBoxes);
        for (int kb = c * kChunkBoxes; kb < kb1; ++kb) {
          const int s = kb % Cfg::kStages;
          const uint32_t ph = (uint32_t)(kb / Cfg::kStages) & 1u;
          if (!tc::mbar_wait(full + s, ph)) {
            ok = false;
            break;
          }
          tc::fence_after_sync();
          uint8_t* st = smem + s * Cfg::kStageBytes;
          const uint64_t ah = tc::desc_sw128(st), bh = tc::desc_sw128(st + kTileBytes);
#pragma unroll
          for (int k = 0; k < Cfg::kMmaPerBox; ++k) {
            const uint32_t acc = (kb > c * kChunkBoxes || k > 0) ? 1u : 0u;
            const uint64_t adv = 2ull * k;   // +32 bytes along K
            if (MODE == TC_TF32) {
              tc::mma_tf32(d, ah + adv, bh + adv, tc::kIdescTF32, acc);
            } else if (MODE == TC_TF32X3) {
              const uint64_t al = tc::desc_sw128(st + 2 * kTileBytes), bl = tc::desc_sw128(st + 3 * kTileBytes);
              tc::mma_tf32(d, ah + adv, bh + adv, tc::kIdescTF32, acc);
              tc::mma_tf32(d, ah + adv, bl + adv, tc::kIdescTF32, 1u);
              tc::mma_tf32(d, al + adv, bh + adv, tc::kIdescTF32, 1u);
            } else {
              tc::mma_bf16(d, ah + adv, bh + adv, tc::kIdescBF16, acc);
              if (MODE == TC_BF16X3) {
                const uint64_t al = tc::desc_sw128(st + 2 * kTileBytes), bl = tc::desc_sw128(st + 3 * kTileBytes);
                tc::mma_bf16(d, ah + adv, bl + adv, tc::kIdescBF16, 1u);
                tc::mma_bf16(d, al + adv, bh + adv, tc::kIdescBF16, 1u);
              }
            }
          }
          tc::mma_commit(empty + s);   // stage s free once these MMAs have read it
        }
        tc::mma_commit(acc_full + buf);  // chunk complete
      }
      if (!ok) atomicCAS(a.err, 0, POGS_ERR_TIMEOUT);
      // every MMA this thread issued has finished before the tensor memory is released
      tc::mma_commit(drain);
      if (!tc::mbar_wait(drain, 0)) atomicCAS(a.err, 0, POGS_ERR_TIMEOUT);
    }
  } else {
    // ---- epilogue warps: drain chunks, accumulate in FP32 (round to nearest), store -----------
    const int wq = warp & 3;                      // TMEM lane quarter this warp may access
    const int64_t row = (int64_t)ti * kTileRows + wq * 32 + lane;
    float acc[128];
#pragma unroll
    for (int i = 0; i < 128; ++i) acc[i] = 0.0f;
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
      const int buf = c & 1;
      if (!tc::mbar_wait(acc_full + buf, (uint32_t)(c >> 1) & 1u)) {
        ok = false;
        break;
      }
      tc::fence_after_sync();
      const uint32_t taddr = tmem + (static_cast<uint32_t>(wq * 32) << 16) + (uint32_t)(buf * 128);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float v[32];
        tc::tmem_ld32(taddr + q * 32, v);
#pragma unroll
        for (int i = 0; i < 32; ++i) acc[q * 32 + i] = __fadd_rn(acc[q * 32 + i], v[i]);
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(acc_empty + buf)) : "memory");
    }
    if (!ok) {
      if (lane == 0) atomicCAS(a.err, 0, POGS_ERR_TIMEOUT);
    } else if (row < a.M) {
      const int64_t col0 = (int64_t)tj * kTileRows;
      if (a.epi == 0) {
        const float al = (float)a.alpha;
        if (al != 1.0f) {
#pragma unroll
          for (int i = 0; i < 128; ++i) acc[i] *= al;
        }
        float* out = a.C + row * a.ldc + col0;
        if (col0 + 128 <= a.N && ((reinterpret_cast<uintptr_t>(out) & 15) == 0)) {
#pragma unroll
          for (int i = 0; i < 128; i += 4)
            *reinterpret_cast<float4*>(out + i) = make_float4(acc[i], acc[i + 1], acc[i + 2], acc[i + 3]);
        } else {
#pragma unroll
          for (int i = 0; i < 128; ++i)
            if (col0 + i < a.N) out[i] = acc[i];
        }
      } else if (a.epi == 1) {
        double* out = a.C64 + row * a.ldc + col0;
#pragma unroll
        for (int i = 0; i < 128; ++i)
          if (col0 + i < a.N && col0 + i <= row) out[i] += a.alpha * (double)acc[i];
      } else {
        // double-float Schur complement update, lower triangle
        float* oh = a.C + row * a.ldc + col0;
        float* ol = a.Clo + row * a.ldc + col0;
        if (tj < ti && col0 + 128 <= a.N && ((reinterpret_cast<uintptr_t>(oh) | reinterpret_cast<uintptr_t>(ol)) & 15) == 0) {
#pragma unroll
          for (int i = 0; i < 128; i += 4) {
            float4 h = *reinterpret_cast<float4*>(oh + i), l = *reinterpret_cast<float4*>(ol + i);
            df_sub(h.x, l.x, acc[i]);
            df_sub(h.y, l.y, acc[i + 1]);
            df_sub(h.z, l.z, acc[i + 2]);
            df_sub(h.w, l.w, acc[i + 3]);
            *reinterpret_cast<float4*>(oh + i) = h;
            *reinterpret_cast<float4*>(ol + i) = l;
          }
        } else {
#pragma unroll
          for (int i = 0; i < 128; ++i)
            if (col0 + i < a.N && col0 + i <= row) {
              float h = oh[i], l = ol[i];
              df_sub(h, l, acc[i]);
              oh[i] = h;
              ol[i] = l;
            }
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 1) tc::tmem_dealloc(tmem, 256);
}

// ---- operand packing ----------------------------------------------------------------------
// X (rows x K): element (r, k) = TRANS ? src[k*ld + r] : src[r*ld + k]; written K-major to a
// zero-padded [rp x Kp] buffer (BF16 hi/lo or TF32-rounded FP32).
template <bool TRANS, int MODE>
__global__ void pack_kernel(const float* __restrict__ src, int64_t ld, int64_t rows, int64_t K, int64_t Kp,
                            void* hi, void* lo) {
  __shared__ float t[32][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, k0 = (int64_t)blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    float v = 0.0f;
    if (TRANS) {
      const int64_t k = k0 + i, r = r0 + threadIdx.x;     // contiguous along r in the source
      if (r < rows && k < K) v = src[k * ld + r];
      t[i][threadIdx.x] = v;                               // t[k][r]
    } else {
      const int64_t r = r0 + i, k = k0 + threadIdx.x;
      if (r < rows && k < K) v = src[r * ld + k];
      t[threadIdx.x][i] = v;                               // t[k][r]
    }
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t r = r0 + i, k = k0 + threadIdx.x;
    const float v = t[threadIdx.x][i];
    const int64_t o = r * Kp + k;
    if (MODE == TC_TF32 || MODE == TC_TF32X3) {
      uint32_t u;
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(v));
      const float h = __uint_as_float(u);
      static_cast<float*>(hi)[o] = h;
      if (MODE == TC_TF32X3) {
        uint32_t w;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(w) : "f"(__fsub_rn(v, h)));
        static_cast<float*>(lo)[o] = __uint_as_float(w);
      }
    } else {
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      static_cast<__nv_bfloat16*>(hi)[o] = h;
      if (MODE == TC_BF16X3) static_cast<__nv_bfloat16*>(lo)[o] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

// Map over a K-major [rows x inner] buffer with 128-row x 128-byte boxes, 128-byte swizzle.
int make_map(CUtensorMap* map, const void* ptr, bool tf32, uint64_t inner, uint64_t rows) {
  auto enc = encode_fn();
  if (!enc) return -1;
  const uint32_t esize = tf32 ? 4 : 2;
  cuuint64_t gdim[2] = {inner, rows};
  cuuint64_t gstride[1] = {inner * esize};
  cuuint32_t box[2] = {128u / esize, (cuuint32_t)kTileRows};
  cuuint32_t es[2] = {1, 1};
  const CUresult r = enc(map, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                         const_cast<void*>(ptr), gdim, gstride, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -1;
}

template <int MODE>
int launch_tc(const CUtensorMap& xh, const CUtensorMap& xl, const CUtensorMap& yh, const CUtensorMap& yl,
              const TcArgs& a, int ntiles, cudaStream_t s) {
  using Cfg = TcCfg<MODE>;
  static PerDeviceOnce attr;
  if (attr.run([] {
        if (cudaFuncSetAttribute(tc_gemm_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)Cfg::kSmem) == cudaSuccess)
          return 0;
        cudaGetLastError();
        return -1;
      }) != 0)
    return -1;
  count_launch();
  tc_gemm_kernel<MODE><<<ntiles, 192, Cfg::kSmem, s>>>(xh, xl, yh, yl, a);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace

// G (q x q, row-major, ld ldg; lower 128-tiles written) = X X^T with X = A^T (tall) or A (fat).
int gram_tensor(int prec, const float* A, int64_t lda, int64_t m, int64_t n, bool tall, float* G, int64_t ldg,
                void* scratch, size_t scratch_bytes, size_t* need_bytes, int* err, cudaStream_t s) {
  int mode;
  if (prec == POGS_GRAM_BF16) mode = TC_BF16;
  else if (prec == POGS_GRAM_BF16X3) mode = TC_BF16X3;
  else if (prec == POGS_GRAM_TF32) mode = TC_TF32;
  else return -1;
  if (!encode_fn()) return -1;
  const int64_t q = tall ? n : m, K = tall ? m : n;
  const int64_t rp = round_up(q, kTileRows);
  const int64_t kbox = mode == TC_TF32 ? 32 : 64;
  const int64_t Kp = round_up(K, kbox);
  const size_t esize = mode == TC_TF32 ? 4 : 2;
  const size_t one = (size_t)rp * Kp * esize;
  const size_t need = one * (mode == TC_BF16X3 ? 2 : 1) + 256;
  if (need_bytes) *need_bytes = need;
  if (!scratch) return 0;
  if (scratch_bytes < need) return -1;
  char* base = static_cast<char*>(scratch);
  void* hi = base;
  void* lo = mode == TC_BF16X3 ? base + one : nullptr;
  dim3 pg((unsigned)(Kp / 32), (unsigned)(rp / 32)), pb(32, 8);
  count_launch();
  if (tall) {
    if (mode == TC_BF16) pack_kernel<true, TC_BF16><<<pg, pb, 0, s>>>(A, lda, q, K, Kp, hi, lo);
    else if (mode == TC_BF16X3) pack_kernel<true, TC_BF16X3><<<pg, pb, 0, s>>>(A, lda, q, K, Kp, hi, lo);
    else pack_kernel<true, TC_TF32><<<pg, pb, 0, s>>>(A, lda, q, K, Kp, hi, lo);
  } else {
    if (mode == TC_BF16) pack_kernel<false, TC_BF16><<<pg, pb, 0, s>>>(A, lda, q, K, Kp, hi, lo);
    else if (mode == TC_BF16X3) pack_kernel<false, TC_BF16X3><<<pg, pb, 0, s>>>(A, lda, q, K, Kp, hi, lo);
    else pack_kernel<false, TC_TF32><<<pg, pb, 0, s>>>(A, lda, q, K, Kp, hi, lo);
  }
  if (cudaGetLastError() != cudaSuccess) return -1;
  CUtensorMap mh, ml;
  memset(&ml, 0, sizeof(ml));
  if (make_map(&mh, hi, mode == TC_TF32, (uint64_t)Kp, (uint64_t)rp) != 0) return -1;
  if (mode == TC_BF16X3 && make_map(&ml, lo, false, (uint64_t)Kp, (uint64_t)rp) != 0) return -1;
  if (mode != TC_BF16X3) ml = mh;
  TcArgs a;
  memset(&a, 0, sizeof(a));
  a.nkb = (int)(Kp / kbox);
  a.tiles = (int)(rp / kTileRows);
  a.tiles_n = a.tiles;
  a.lower_only = 1;
  a.M = q;
  a.N = q;
  a.C = G;
  a.ldc = ldg;
  a.alpha = 1.0;
  a.epi = 0;
  a.err = err;
  const int ntiles = a.tiles * (a.tiles + 1) / 2;
  if (mode == TC_BF16) return launch_tc<TC_BF16>(mh, ml, mh, ml, a, ntiles, s);
  if (mode == TC_BF16X3) return launch_tc<TC_BF16X3>(mh, ml, mh, ml, a, ntiles, s);
  return launch_tc<TC_TF32>(mh, ml, mh, ml, a, ntiles, s);
}

// C (M x N, row-major, ld ldc) op= X Y^T on the tensor cores in TF32x3, with X (M x K) and Y (N x K)
// read from row-major A and B: X[i][k] = transA ? A[k*lda + i] : A[i*lda + k], likewise Y from B.
// X and Y are packed K-major as TF32 hi/lo pairs (zero padded to 128 rows and 32 columns of K);
// every 128 x 128 tile of C (the lower ones when `lower`) is one CTA.  epi TC_EPI_STORE:
// C = alpha X Y^T; TC_EPI_DF_SUB: the double-float pair (C, Clo) -= X Y^T on and below the
// diagonal.  When A == B with equal layout and M == N (a rank-K update), one packing serves both.
// scratch == nullptr: *need_bytes receives the scratch size only.
int tc_gemm_tf32x3(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda, bool transA, const float* B,
                   int64_t ldb, bool transB, float alpha, float* C, float* Clo, int64_t ldc, int epi, bool lower,
                   void* scratch, size_t scratch_bytes, size_t* need_bytes, int* err, cudaStream_t s, bool kskip) {
  if (!encode_fn()) return -1;
  const bool same = A == B && lda == ldb && transA == transB && M == N;
  const int64_t mp = round_up(M, kTileRows), np = round_up(N, kTileRows), Kp = round_up(K, 32);
  const int64_t xs = round_up(mp * Kp * 4, 256), ys = same ? 0 : round_up(np * Kp * 4, 256);
  const size_t need = (size_t)(2 * xs + 2 * ys);
  if (need_bytes) *need_bytes = need;
  if (!scratch) return 0;
  if (scratch_bytes < need) return -1;
  char* base = static_cast<char*>(scratch);
  void* xh = base;
  void* xl = base + xs;
  void* yh = same ? xh : base + 2 * xs;
  void* yl = same ? xl : base + 2 * xs + ys;
  auto pack = [&](const float* src, int64_t ld, bool trans, int64_t rows, int64_t rp, void* hi, void* lo) {
    const dim3 grid((unsigned)(Kp / 32), (unsigned)(rp / 32)), blk(32, 8);
    count_launch();
    if (trans) pack_kernel<true, TC_TF32X3><<<grid, blk, 0, s>>>(src, ld, rows, K, Kp, hi, lo);
    else pack_kernel<false, TC_TF32X3><<<grid, blk, 0, s>>>(src, ld, rows, K, Kp, hi, lo);
  };
  pack(A, lda, transA, M, mp, xh, xl);
  if (!same) pack(B, ldb, transB, N, np, yh, yl);
  if (cudaGetLastError() != cudaSuccess) return -1;
  CUtensorMap mxh, mxl, myh, myl;
  if (make_map(&mxh, xh, true, (uint64_t)Kp, (uint64_t)mp) != 0 || make_map(&mxl, xl, true, (uint64_t)Kp, (uint64_t)mp) != 0 ||
      make_map(&myh, yh, true, (uint64_t)Kp, (uint64_t)np) != 0 || make_map(&myl, yl, true, (uint64_t)Kp, (uint64_t)np) != 0)
    return -1;
  TcArgs a;
  memset(&a, 0, sizeof(a));
  a.nkb = (int)(Kp / 32);
  a.tiles = (int)(mp / kTileRows);
  a.tiles_n = (int)(np / kTileRows);
  a.lower_only = lower ? 1 : 0;
  a.kskip = kskip ? 1 : 0;
  if (lower && a.tiles != a.tiles_n) return -1;
  a.M = M;
  a.N = N;
  a.C = C;
  a.Clo = Clo;
  a.ldc = ldc;
  a.alpha = alpha;
  a.epi = epi;
  a.err = err;
  const int ntiles = lower ? a.tiles * (a.tiles + 1) / 2 : a.tiles * a.tiles_n;
  return launch_tc<TC_TF32X3>(mxh, mxl, myh, myl, a, ntiles, s);
}

int tc_gemm_nn_tf32x3(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda, const float* B, int64_t ldb,
                      float alpha, float* C, int64_t ldc, void* scratch, size_t scratch_bytes, size_t* need_bytes,
                      int* err, cudaStream_t s) {
  return tc_gemm_tf32x3(M, N, K, A, lda, false, B, ldb, true, alpha, C, nullptr, ldc, TC_EPI_STORE, false, scratch,
                        scratch_bytes, need_bytes, err, s);
}

namespace {
// One thread waits, with the bounded wait every tcgen05 kernel uses, on a barrier whose phase
// no thread completes; the wait gives up after its budget and the status says so.
__global__ void bounded_wait_probe_kernel(int* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_mbar_init();
    *status = tc::mbar_wait(&bar, 0) ? 0 : POGS_ERR_TIMEOUT;
  }
}
}  // namespace

int bounded_wait_probe(cudaStream_t s) {
  void* q = nullptr;
  if (pool_alloc(&q, sizeof(int), s) != 0) return POGS_ERR_OOM;
  int* d = static_cast<int*>(q);
  int h = POGS_ERR_CUDA;
  count_launch();
  bounded_wait_probe_kernel<<<1, 32, 0, s>>>(d);
  if (cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    h = POGS_ERR_CUDA;
  }
  cudaFreeAsync(d, s);
  return h;
}

}  // namespace pogs
