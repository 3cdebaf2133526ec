// Mixed-precision blocked Cholesky of I + G and the FP32 inverse factor M = L^{-1}
// (Section 3.5, factorization caching), built on one double-buffered SIMT SGEMM.
//
// Right-looking, 128-wide block columns (the tile edge of the packed inverse):
//   diag   one CTA factors the 128 x 128 diagonal block of the FP64 Schur complement in FP32
//          shared memory (32-wide sub-blocks) and inverts it; W_kk = L_kk^{-1} is also the
//          diagonal tile of M;
//   panel  L21 = H21 W_kk^T from the FP32-rounded Schur complement, stored FP32;
//   update H22 <- H22 - L21 L21^T: FP32 products accumulated over the 128-wide panel, then
//          subtracted from the Schur complement (lower tiles only).
// The Schur complement is held in extended precision as an unevaluated sum hi + lo of two
// FP32 numbers and every update is applied with error-free transformations (Knuth's TwoSum
// followed by Dekker's Fast2Sum renormalisation), which carries about 48 significant bits
// through the q/128 block steps using only the FP32 pipes -- B300's FP64 rate is a small
// fraction of its FP32 rate, and an FP64 subtraction per element and block step would cost
// as much as the products themselves.  Every O(q^3) product runs on the FP32 pipes.  I + G
// has all eigenvalues >= 1, so no pivot of the factorization suffers cancellation.
//
// The inverse uses the 2 x 2 block identity
//   inv([[L11, 0], [L21, L22]]) = [[M11, 0], [-M22 L21 M11, M22]]
// recursively, splitting at multiples of 128 so that the leaves are the W_kk above.
#include <algorithm>

#include <vector>

#include "kernels.h"

namespace pogs {
namespace {

constexpr int kBM = 128, kBN = 128, kBK = 16;
constexpr int kLDS = kBM + 4;   // shared k-row pitch (floats): 16-byte aligned rows

enum { OUT_F32 = 0, OUT_SUB_DF = 1 };

// Four consecutive elements r[0 .. 3] of a row whose remaining length is `left` (zero past
// it).  The caller guarantees 16-byte alignment of r (ld % 4 == 0, k % 4 == 0).
__device__ __forceinline__ float4 ld4(const float* __restrict__ r, int64_t left) {
  if (left >= 4) return *reinterpret_cast<const float4*>(r);
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (left > 0) v.x = r[0];
  if (left > 1) v.y = r[1];
  if (left > 2) v.z = r[2];
  return v;
}
// C = op(A) op(B) on 128 x 128 tiles, 256 threads, 8 x 8 outputs per thread (two 4-row by
// two 4-column groups, 64 apart, so shared reads are float4 and conflict-free).
//   A: M x K row-major.
//   B: BT ? N x K row-major (C = A B^T) : K x N row-major (C = A B).
//   OUT_F32:    Cf = alpha * (A op(B))
//   OUT_SUB_DF: (Cf, Clo) -= A op(B) on the double-float pair, elements on or below the
//               diagonal only when `lower`.
// MINB: resident CTAs per SM the register budget is sized for.
// `lower`: blockIdx.x enumerates the lower-triangular tiles (row of tiles by row of tiles).
// `tri`: bit 0 -- op(B) lower triangular (rows k < j of column j are zero): skip k < col0;
//        bit 1 -- A lower triangular (A[i][k] = 0 for k > i): stop at row0 + 128.
// Global tiles are prefetched into registers while the previous shared tile is consumed.
template <bool BT, int OUT, int MINB>
__global__ void __launch_bounds__(256, MINB)
    sgemm128_kernel(int M, int N, int K, const float* __restrict__ A, int64_t lda, const float* __restrict__ B,
                    int64_t ldb, float alpha, float* __restrict__ Cf, float* __restrict__ Clo, int64_t ldc,
                    int lower, int tri) {
  __shared__ __align__(16) float As[2][kBK][kLDS];
  __shared__ __align__(16) float Bs[2][kBK][kLDS];
  int bi, bj;
  if (lower) {
    const int b = blockIdx.x;
    int I = (int)((sqrtf(8.0f * (float)b + 1.0f) - 1.0f) * 0.5f);
    while ((I + 1) * (I + 2) / 2 <= b) ++I;
    while (I * (I + 1) / 2 > b) --I;
    bi = I;
    bj = b - I * (I + 1) / 2;
  } else {
    bi = blockIdx.y;
    bj = blockIdx.x;
  }
  const int row0 = bi * kBM, col0 = bj * kBN;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  int kbeg = 0, kend = K;
  if (tri & 1) kbeg = col0 < K ? col0 : K;
  if (tri & 2) kend = row0 + kBM < K ? row0 + kBM : K;

  // per-thread global sources: A rows r = tid/4 (+64), K offset 4*(tid%4); B likewise when
  // BT, else K row tid/32 (+8) and columns 4*(tid%32)
  const int r_ld = tid >> 2, kq = (tid & 3) * 4;
  const float* ap[2];
  const float* bp[2];
  bool aok[2], bok[2];
#pragma unroll
  for (int l = 0; l < 2; ++l) {
    const int ar = row0 + r_ld + 64 * l;
    aok[l] = ar < M;
    ap[l] = A + (int64_t)(aok[l] ? ar : 0) * lda + kq;
    if (BT) {
      const int br = col0 + r_ld + 64 * l;
      bok[l] = br < N;
      bp[l] = B + (int64_t)(bok[l] ? br : 0) * ldb + kq;
    } else {
      const int bc = col0 + (tid & 31) * 4;
      bok[l] = bc < N;
      bp[l] = B + (int64_t)((tid >> 5) + 8 * l) * ldb + (bok[l] ? bc : 0);
    }
  }
  const int bc_left = N - (col0 + (tid & 31) * 4);

  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  float4 ra[2], rb[2];
  auto gload = [&](int k0) {
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      ra[l] = aok[l] ? ld4(ap[l] + k0, K - (k0 + kq)) : make_float4(0.f, 0.f, 0.f, 0.f);
      if (BT) {
        rb[l] = bok[l] ? ld4(bp[l] + k0, K - (k0 + kq)) : make_float4(0.f, 0.f, 0.f, 0.f);
      } else {
        const int kr = k0 + (tid >> 5) + 8 * l;
        rb[l] = (bok[l] && kr < K) ? ld4(bp[l] + (int64_t)k0 * ldb, bc_left) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
  };
  auto sstore = [&](int buf) {
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      const int r = r_ld + 64 * l;
      As[buf][kq + 0][r] = ra[l].x;
      As[buf][kq + 1][r] = ra[l].y;
      As[buf][kq + 2][r] = ra[l].z;
      As[buf][kq + 3][r] = ra[l].w;
      if (BT) {
        Bs[buf][kq + 0][r] = rb[l].x;
        Bs[buf][kq + 1][r] = rb[l].y;
        Bs[buf][kq + 2][r] = rb[l].z;
        Bs[buf][kq + 3][r] = rb[l].w;
      } else {
        *reinterpret_cast<float4*>(&Bs[buf][(tid >> 5) + 8 * l][(tid & 31) * 4]) = rb[l];
      }
    }
  };

  if (kbeg < kend) {
    gload(kbeg);
    sstore(0);
    __syncthreads();
    int buf = 0;
    for (int k0 = kbeg; k0 < kend; k0 += kBK) {
      const bool more = k0 + kBK < kend;
      if (more) gload(k0 + kBK);
#pragma unroll
      for (int k = 0; k < kBK; ++k) {
        const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][k][ty * 4]);
        const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][k][ty * 4 + 64]);
        const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][k][tx * 4]);
        const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][k][tx * 4 + 64]);
        const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
      }
      if (more) sstore(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }

#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int gi = row0 + ty * 4 + (i & 3) + (i >> 2) * 64;
    if (gi >= M) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int gj0 = col0 + tx * 4 + h * 64;
      if (gj0 >= N) continue;
      const float v0 = acc[i][h * 4 + 0], v1 = acc[i][h * 4 + 1], v2 = acc[i][h * 4 + 2], v3 = acc[i][h * 4 + 3];
      if (OUT == OUT_F32) {
        float* c = Cf + (int64_t)gi * ldc + gj0;
        if (gj0 + 3 < N) {
          *reinterpret_cast<float4*>(c) = make_float4(alpha * v0, alpha * v1, alpha * v2, alpha * v3);
        } else {
          c[0] = alpha * v0;
          if (gj0 + 1 < N) c[1] = alpha * v1;
          if (gj0 + 2 < N) c[2] = alpha * v2;
        }
      } else {
        float* ch = Cf + (int64_t)gi * ldc + gj0;
        float* cl = Clo + (int64_t)gi * ldc + gj0;
        const int lim = min(N, lower ? gi + 1 : N) - gj0;   // elements of this group to update
        if (lim >= 4) {
          float4 h = *reinterpret_cast<float4*>(ch);
          float4 l = *reinterpret_cast<float4*>(cl);
          df_sub(h.x, l.x, v0);
          df_sub(h.y, l.y, v1);
          df_sub(h.z, l.z, v2);
          df_sub(h.w, l.w, v3);
          *reinterpret_cast<float4*>(ch) = h;
          *reinterpret_cast<float4*>(cl) = l;
        } else if (lim > 0) {
          df_sub(ch[0], cl[0], v0);
          if (lim > 1) df_sub(ch[1], cl[1], v1);
          if (lim > 2) df_sub(ch[2], cl[2], v2);
        }
      }
    }
  }
}

// ---- small tiles ---------------------------------------------------------------------------
// The same products on 32 x 32 tiles, 64 threads, 4 x 4 outputs per thread, for shapes whose
// 128 x 128 grid would leave most SMs idle (the lookahead panels and the small levels of the
// recursion): 16 times the CTAs for the same work.  Every output accumulates the same terms
// in the same k order as the 128-tile kernel (the skipped leading and trailing k of triangular
// operands are exact zeros in both), so both kernels give the same bits.
constexpr int kSB = 32, kSK = 32;   // tile edge, K step
constexpr int kSLD = kSB + 4;       // shared k-row pitch (floats): 16-byte aligned rows
constexpr int64_t kSmallTileGrid = 64;   // 128-tile grids below this size take the 32-tile kernel
template <bool BT, int OUT>
__global__ void __launch_bounds__(64)
    sgemm32_kernel(int M, int N, int K, const float* __restrict__ A, int64_t lda, const float* __restrict__ B,
                   int64_t ldb, float alpha, float* __restrict__ Cf, float* __restrict__ Clo, int64_t ldc,
                   int lower, int tri) {
  __shared__ __align__(16) float As[2][kSK][kSLD];
  __shared__ __align__(16) float Bs[2][kSK][kSLD];
  int bi, bj;
  if (lower) {
    const int b = blockIdx.x;
    int I = (int)((sqrtf(8.0f * (float)b + 1.0f) - 1.0f) * 0.5f);
    while ((I + 1) * (I + 2) / 2 <= b) ++I;
    while (I * (I + 1) / 2 > b) --I;
    bi = I;
    bj = b - I * (I + 1) / 2;
  } else {
    bi = blockIdx.y;
    bj = blockIdx.x;
  }
  const int row0 = bi * kSB, col0 = bj * kSB;
  const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3;
  int kbeg = 0, kend = K;
  if (tri & 1) kbeg = col0 < K ? col0 : K;
  if (tri & 2) kend = row0 + kSB < K ? row0 + kSB : K;
  // per-thread global sources: A rows tid/8 (+8, +16, +24), K offset 4*(tid%8); B likewise
  // when BT, else K rows tid/8 (+8, ...) and columns 4*(tid%8)
  const int r_ld = tid >> 3, kq = (tid & 7) * 4;
  const float* ap[4];
  const float* bp[4];
  bool aok[4], bok[4];
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    const int ar = row0 + r_ld + 8 * l;
    aok[l] = ar < M;
    ap[l] = A + (int64_t)(aok[l] ? ar : 0) * lda + kq;
    if (BT) {
      const int br = col0 + r_ld + 8 * l;
      bok[l] = br < N;
      bp[l] = B + (int64_t)(bok[l] ? br : 0) * ldb + kq;
    } else {
      const int bc = col0 + kq;
      bok[l] = bc < N;
      bp[l] = B + (int64_t)(r_ld + 8 * l) * ldb + (bok[l] ? bc : 0);
    }
  }
  const int bc_left = N - (col0 + kq);
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  float4 ra[4], rb[4];
  auto gload = [&](int k0) {
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      ra[l] = aok[l] ? ld4(ap[l] + k0, K - (k0 + kq)) : make_float4(0.f, 0.f, 0.f, 0.f);
      if (BT) {
        rb[l] = bok[l] ? ld4(bp[l] + k0, K - (k0 + kq)) : make_float4(0.f, 0.f, 0.f, 0.f);
      } else {
        const int kr = k0 + r_ld + 8 * l;
        rb[l] = (bok[l] && kr < K) ? ld4(bp[l] + (int64_t)k0 * ldb, bc_left) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
  };
  auto sstore = [&](int buf) {
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int r = r_ld + 8 * l;
      As[buf][kq + 0][r] = ra[l].x;
      As[buf][kq + 1][r] = ra[l].y;
      As[buf][kq + 2][r] = ra[l].z;
      As[buf][kq + 3][r] = ra[l].w;
      if (BT) {
        Bs[buf][kq + 0][r] = rb[l].x;
        Bs[buf][kq + 1][r] = rb[l].y;
        Bs[buf][kq + 2][r] = rb[l].z;
        Bs[buf][kq + 3][r] = rb[l].w;
      } else {
        *reinterpret_cast<float4*>(&Bs[buf][r][kq]) = rb[l];
      }
    }
  };
  if (kbeg < kend) {
    gload(kbeg);
    sstore(0);
    __syncthreads();
    int buf = 0;
    for (int k0 = kbeg; k0 < kend; k0 += kSK) {
      const bool more = k0 + kSK < kend;
      if (more) gload(k0 + kSK);
#pragma unroll
      for (int k = 0; k < kSK; ++k) {
        const float4 a4 = *reinterpret_cast<const float4*>(&As[buf][k][ty * 4]);
        const float4 b4 = *reinterpret_cast<const float4*>(&Bs[buf][k][tx * 4]);
        const float a[4] = {a4.x, a4.y, a4.z, a4.w};
        const float b[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
      }
      if (more) sstore(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }
  const int gj0 = col0 + tx * 4;
  if (gj0 >= N) return;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gi = row0 + ty * 4 + i;
    if (gi >= M) continue;
    const float v0 = acc[i][0], v1 = acc[i][1], v2 = acc[i][2], v3 = acc[i][3];
    if (OUT == OUT_F32) {
      float* c = Cf + (int64_t)gi * ldc + gj0;
      if (gj0 + 3 < N) {
        *reinterpret_cast<float4*>(c) = make_float4(alpha * v0, alpha * v1, alpha * v2, alpha * v3);
      } else {
        c[0] = alpha * v0;
        if (gj0 + 1 < N) c[1] = alpha * v1;
        if (gj0 + 2 < N) c[2] = alpha * v2;
      }
    } else {
      float* ch = Cf + (int64_t)gi * ldc + gj0;
      float* cl = Clo + (int64_t)gi * ldc + gj0;
      const int lim = min(N, lower ? gi + 1 : N) - gj0;
      if (lim >= 4) {
        float4 h = *reinterpret_cast<float4*>(ch);
        float4 l = *reinterpret_cast<float4*>(cl);
        df_sub(h.x, l.x, v0);
        df_sub(h.y, l.y, v1);
        df_sub(h.z, l.z, v2);
        df_sub(h.w, l.w, v3);
        *reinterpret_cast<float4*>(ch) = h;
        *reinterpret_cast<float4*>(cl) = l;
      } else if (lim > 0) {
        df_sub(ch[0], cl[0], v0);
        if (lim > 1) df_sub(ch[1], cl[1], v1);
        if (lim > 2) df_sub(ch[2], cl[2], v2);
      }
    }
  }
}

template <bool BT, int OUT, int MINB>
void sgemm_launch(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda, const float* B, int64_t ldb,
                  float alpha, float* Cf, float* Clo, int64_t ldc, bool lower, int tri, cudaStream_t s) {
  if (M <= 0 || N <= 0) return;
  count_launch();   // sizes fit int: q <= 2^31 / 128 rows of 128-tiles
  const int64_t T = cdiv(M, kBM);
  const int64_t tiles = lower ? T * (T + 1) / 2 : cdiv(N, kBN) * T;
  if (tiles < kSmallTileGrid) {
    if (lower) {
      const int64_t Ts = cdiv(M, kSB);
      sgemm32_kernel<BT, OUT><<<(unsigned)(Ts * (Ts + 1) / 2), 64, 0, s>>>((int)M, (int)N, (int)K, A, lda, B, ldb,
                                                                         alpha, Cf, Clo, ldc, 1, tri);
    } else {
      dim3 grid((unsigned)cdiv(N, kSB), (unsigned)cdiv(M, kSB));
      sgemm32_kernel<BT, OUT><<<grid, 64, 0, s>>>((int)M, (int)N, (int)K, A, lda, B, ldb, alpha, Cf, Clo, ldc, 0,
                                                  tri);
    }
    return;
  }
  if (lower) {
    sgemm128_kernel<BT, OUT, MINB><<<(unsigned)(T * (T + 1) / 2), 256, 0, s>>>(
        (int)M, (int)N, (int)K, A, lda, B, ldb, alpha, Cf, Clo, ldc, 1, tri);
  } else {
    dim3 grid((unsigned)cdiv(N, kBN), (unsigned)cdiv(M, kBM));
    sgemm128_kernel<BT, OUT, MINB><<<grid, 256, 0, s>>>((int)M, (int)N, (int)K, A, lda, B, ldb, alpha, Cf, Clo,
                                                         ldc, 0, tri);
  }
}

// ---- diagonal block ------------------------------------------------------------------------
constexpr int kDB = 128;        // block edge
constexpr int kDS = kDB + 1;    // shared row pitch (conflict-free column walks)
constexpr int kDiagThreads = 512;   // 16 warps: one 128-block per CTA, latency-bound phases

constexpr int kPT = 100;   // pitch of the transposed panel (at most 96 rows), 16-byte rows
constexpr int kLB = 36;    // pitch of the aligned copy of the 32 x 32 diagonal factor

// One CTA factors the nb x nb diagonal block Hkk (hi part, lower triangle read) in FP32 and
// writes W = L_kk^{-1} (lower triangular, zero above the diagonal) to W (ld ldw).  Rows and
// columns nb..127 are padded with the identity.  Four 32-wide sub-block steps: warp 0 factors
// the 32 x 32 diagonal sub-block in registers (lane = row; each pivot column is published in
// shared memory and read back as float4 broadcasts) and inverts it (lane = column, forward
// substitution on e_c over an aligned copy of the factor); all warps then form the panel below
// it, P = S_panel V^T (kept transposed), and update the trailing rows from it.  The
// off-diagonal blocks of W follow by block forward substitution,
// W_ij = -W_ii sum_{k=j}^{i-1} L_ik W_kj.
__global__ void __launch_bounds__(kDiagThreads) chol_diag_kernel(const float* __restrict__ Hkk, int64_t ldh, int nb,
                                                        float* __restrict__ W, int64_t ldw, int* err) {
  extern __shared__ __align__(16) float sm[];
  float* S = sm;                 // [128][129]: Schur block, then L
  float* V = S + kDB * kDS;      // [128][129]: W in the lower triangle; T scratch
  float* Dv = V + kDB * kDS;     // [128]: 1 / L_jj
  float* Lb = Dv + kDB;          // [32][kLB]: the current 32 x 32 diagonal factor
  float* cb = Lb + 32 * kLB;     // [2][32]: column broadcast of the 32 x 32 factorization
  float* PT = cb + 64;           // [32][kPT]: the current panel, transposed
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (nb == kDB) {
    float4 ld[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int e = tid + t * kDiagThreads, i = e >> 5, k = (e & 31) * 4;
      ld[t] = k <= i ? *reinterpret_cast<const float4*>(Hkk + (int64_t)i * ldh + k) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int e = tid + t * kDiagThreads, i = e >> 5, k = (e & 31) * 4;
      float* s = S + i * kDS + k;
      float* v = V + i * kDS + k;
      s[0] = ld[t].x;
      s[1] = k + 1 <= i ? ld[t].y : 0.0f;
      s[2] = k + 2 <= i ? ld[t].z : 0.0f;
      s[3] = k + 3 <= i ? ld[t].w : 0.0f;
      v[0] = v[1] = v[2] = v[3] = 0.0f;
    }
  } else {
    constexpr int kPer = kDB * kDB / kDiagThreads;
    float ld[kPer];
#pragma unroll
    for (int t = 0; t < kPer; ++t) {
      const int e = tid + t * kDiagThreads, i = e >> 7, k = e & 127;
      ld[t] = (i < nb && k <= i) ? Hkk[(int64_t)i * ldh + k] : (i == k ? 1.0f : 0.0f);
    }
#pragma unroll
    for (int t = 0; t < kPer; ++t) {
      const int e = tid + t * kDiagThreads, i = e >> 7, k = e & 127;
      S[i * kDS + k] = ld[t];
      V[i * kDS + k] = 0.0f;
    }
  }
  __syncthreads();
  bool bad = false;
  for (int jb = 0; jb < 4; ++jb) {
    const int o = jb * 32;
    if (warp == 0) {
      // 32 x 32 sub-block, lane = row.  Step j scales column j by 1/L_jj (rsqrt of the pivot)
      // and publishes it in shared memory; every lane then subtracts L_lane,j L_k,j from its
      // entries k > j.  Entries above the diagonal are computed too (no predicates) and never
      // stored.
      float* Sd = S + o * kDS + o;
      float r[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) r[k] = Sd[lane * kDS + k];
      float dinv = 1.0f;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        float piv = __shfl_sync(0xffffffffu, r[j], j);
        if (!(piv > 0.0f) || !isfinite(piv)) {
          bad = true;
          piv = 1.0f;
        }
        const float rs = rsqrtf(piv);
        if (lane == j) {
          r[j] = piv * rs;
          dinv = rs;
        } else {
          r[j] *= rs;
        }
        if (j < 31) {
          float* c = cb + (j & 1) * 32;
          c[lane] = r[j];
          __syncwarp();
#pragma unroll
          for (int k4 = (j + 1) & ~3; k4 < 32; k4 += 4) {
            const float4 l4 = *reinterpret_cast<const float4*>(c + k4);
            const float lk[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (k4 + u > j) r[k4 + u] = fmaf(-r[j], lk[u], r[k4 + u]);
          }
        }
      }
#pragma unroll
      for (int k = 0; k < 32; ++k)
        if (k <= lane) Sd[lane * kDS + k] = r[k];
#pragma unroll
      for (int k4 = 0; k4 < 32; k4 += 4)
        *reinterpret_cast<float4*>(Lb + lane * kLB + k4) =
            make_float4(k4 <= lane ? r[k4] : 0.0f, k4 + 1 <= lane ? r[k4 + 1] : 0.0f,
                        k4 + 2 <= lane ? r[k4 + 2] : 0.0f, k4 + 3 <= lane ? r[k4 + 3] : 0.0f);
      Dv[o + lane] = dinv;
      __syncwarp();
      // inverse of the 32 x 32 factor, lane = column c: v_i = -(sum_{k<i} L_ik v_k) / L_ii,
      // four partial sums per row
      float v[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
#pragma unroll
        for (int k4 = 0; k4 < i; k4 += 4) {
          const float4 l4 = *reinterpret_cast<const float4*>(Lb + i * kLB + k4);
          a0 = fmaf(l4.x, v[k4], a0);
          if (k4 + 1 < i) a1 = fmaf(l4.y, v[k4 + 1], a1);
          if (k4 + 2 < i) a2 = fmaf(l4.z, v[k4 + 2], a2);
          if (k4 + 3 < i) a3 = fmaf(l4.w, v[k4 + 3], a3);
        }
        const float di = Dv[o + i];
        v[i] = i < lane ? 0.0f : (i == lane ? di : -((a0 + a1) + (a2 + a3)) * di);
      }
      float* Vd = V + o * kDS + o;
#pragma unroll
      for (int i = 0; i < 32; ++i) Vd[i * kDS + lane] = v[i];
    }
    __syncthreads();
    const int rows = kDB - o - 32;   // 96, 64, 32, 0: whole warps
    // panel P = S_panel V_jj^T, transposed into PT; task = one element
    for (int t = tid; t < rows * 32; t += kDiagThreads) {
      const int rr = t % rows, cc = t / rows;
      const float* Sr = S + (o + 32 + rr) * kDS + o;
      const float* Vc = V + (o + cc) * kDS + o;
      float a0 = 0.0f, a1 = 0.0f;
      int k = 0;
      for (; k + 1 <= cc; k += 2) {
        a0 = fmaf(Sr[k], Vc[k], a0);
        a1 = fmaf(Sr[k + 1], Vc[k + 1], a1);
      }
      if (k <= cc) a0 = fmaf(Sr[k], Vc[k], a0);
      PT[cc * kPT + rr] = a0 + a1;
    }
    __syncthreads();
    if (rows > 0) {
      // P into S (the factor's panel), and S[i][k] -= sum_c P[i][c] P[k][c] for
      // o+32 <= k <= i < 128 in 4 x 4 register blocks, lower blocks only
      for (int e = tid; e < rows * 32; e += kDiagThreads) {
        const int rr = e % rows, cc = e / rows;
        S[(o + 32 + rr) * kDS + o + cc] = PT[cc * kPT + rr];
      }
      const int nbk = rows >> 2, nblk = nbk * (nbk + 1) / 2;
      for (int b = tid; b < nblk; b += kDiagThreads) {
        int bi = (int)((sqrtf(8.0f * (float)b + 1.0f) - 1.0f) * 0.5f);
        while ((bi + 1) * (bi + 2) / 2 <= b) ++bi;
        while (bi * (bi + 1) / 2 > b) --bi;
        const int bk = b - bi * (bi + 1) / 2;
        float a[4][4];
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
          for (int u = 0; u < 4; ++u) a[t][u] = 0.0f;
#pragma unroll 8
        for (int cc = 0; cc < 32; ++cc) {
          const float4 p4 = *reinterpret_cast<const float4*>(PT + cc * kPT + bi * 4);
          const float4 q4 = *reinterpret_cast<const float4*>(PT + cc * kPT + bk * 4);
          const float pi[4] = {p4.x, p4.y, p4.z, p4.w}, pk[4] = {q4.x, q4.y, q4.z, q4.w};
#pragma unroll
          for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int u = 0; u < 4; ++u) a[t][u] = fmaf(pi[t], pk[u], a[t][u]);
        }
        const int i0 = o + 32 + bi * 4, k0 = o + 32 + bk * 4;
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (k0 + u <= i0 + t) S[(i0 + t) * kDS + k0 + u] -= a[t][u];
      }
    }
    __syncthreads();
  }
  // Off-diagonal 32-blocks of W, block row by block row.  T_j = sum_k L_{bi,k} W_{k,j} goes to
  // the (j, bi) block of V (strictly above the block diagonal, never part of W), then
  // W_{bi,j} = -V_{bi} T_j.  Task = 4 x 4 outputs.
  for (int bi = 1; bi < 4; ++bi) {
    for (int t = tid; t < bi * 64; t += kDiagThreads) {
      const int j = t >> 6, r0 = ((t >> 3) & 7) * 4, c0 = (t & 7) * 4;
      float a[4][4];
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) a[x][y] = 0.0f;
      for (int kk = j * 32; kk < bi * 32; ++kk) {
        float l[4], w[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) l[x] = S[(bi * 32 + r0 + x) * kDS + kk];
#pragma unroll
        for (int y = 0; y < 4; ++y) w[y] = V[kk * kDS + j * 32 + c0 + y];
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) a[x][y] = fmaf(l[x], w[y], a[x][y]);
      }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) V[(j * 32 + r0 + x) * kDS + bi * 32 + c0 + y] = a[x][y];
    }
    __syncthreads();
    for (int t = tid; t < bi * 64; t += kDiagThreads) {
      const int j = t >> 6, r0 = ((t >> 3) & 7) * 4, c0 = (t & 7) * 4;
      float a[4][4];
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) a[x][y] = 0.0f;
      for (int tt = 0; tt < r0 + 4; ++tt) {   // V_bi is lower triangular: rows r0..r0+3 need tt <= r0+3
        float vv[4], tv[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) vv[x] = V[(bi * 32 + r0 + x) * kDS + bi * 32 + tt];
#pragma unroll
        for (int y = 0; y < 4; ++y) tv[y] = V[(j * 32 + tt) * kDS + bi * 32 + c0 + y];
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) a[x][y] = fmaf(vv[x], tv[y], a[x][y]);
      }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) V[(bi * 32 + r0 + x) * kDS + j * 32 + c0 + y] = -a[x][y];
    }
    __syncthreads();
  }
  if (nb == kDB) {
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int e = tid + t * kDiagThreads, i = e >> 5, k = (e & 31) * 4;
      const float* v = V + i * kDS + k;
      *reinterpret_cast<float4*>(W + (int64_t)i * ldw + k) =
          make_float4(k <= i ? v[0] : 0.0f, k + 1 <= i ? v[1] : 0.0f, k + 2 <= i ? v[2] : 0.0f, k + 3 <= i ? v[3] : 0.0f);
    }
  } else {
    for (int e = tid; e < nb * nb; e += kDiagThreads) {
      const int i = e / nb, k = e - (e / nb) * nb;
      W[(int64_t)i * ldw + k] = k <= i ? V[i * kDS + k] : 0.0f;
    }
  }
  if (bad && lane == 0) atomicCAS(err, 0, POGS_ERR_NUMERIC);
}
constexpr size_t kDiagSmem = (size_t)(2 * kDB * kDS + kDB + 32 * kLB + 64 + 32 * kPT) * sizeof(float);

// Recursive 2 x 2 block inverse on the FP32 factor (leaves already in M).
// Tensor-core scratch of the inverse (nullptr: SIMT GEMMs only).
struct TcScratch {
  void* p;
  size_t bytes;
  int* err;
};
constexpr int64_t kTcInvMin = 512;   // blocks from this size on use the tensor cores

void inv_rec(const float* L, int64_t ldl, float* M, int64_t ldm, int64_t r0, int64_t nsz, float* work,
             const TcScratch& tc, cudaStream_t s) {
  if (nsz <= kTile) return;
  const int64_t nblk = cdiv(nsz, kTile);
  const int64_t n1 = (nblk / 2) * kTile, n2 = nsz - n1;
  inv_rec(L, ldl, M, ldm, r0, n1, work, tc, s);
  inv_rec(L, ldl, M, ldm, r0 + n1, n2, work, tc, s);
  // T = L21 M11 (M11 lower triangular), then M21 = -M22 T (M22 lower triangular).  The blocks
  // above the diagonal of M11 and M22 hold zeros, so the tensor-core products over the full K
  // equal the SIMT kernel's triangular ones.
  const float* L21 = L + (r0 + n1) * ldl + r0;
  const float* M11 = M + r0 * ldm + r0;
  const float* M22 = M + (r0 + n1) * ldm + r0 + n1;
  float* M21 = M + (r0 + n1) * ldm + r0;
  if (tc.p && std::min(n1, n2) >= kTcInvMin &&
      tc_gemm_nn_tf32x3(n2, n1, n1, L21, ldl, M11, ldm, 1.0f, work, n1, tc.p, tc.bytes, nullptr, tc.err, s) == 0 &&
      tc_gemm_nn_tf32x3(n2, n1, n2, M22, ldm, work, n1, -1.0f, M21, ldm, tc.p, tc.bytes, nullptr, tc.err, s) == 0)
    return;
  sgemm_launch<false, OUT_F32, 1>(n2, n1, n1, L21, ldl, M11, ldm, 1.0f, work, nullptr, n1, false, 1, s);
  sgemm_launch<false, OUT_F32, 1>(n2, n1, n2, M22, ldm, work, n1, -1.0f, M21, nullptr, ldm, false, 2, s);
}

// I + G as the double-float pair (G in place becomes hi; lo receives the rounding error of the
// diagonal 1 + G_ii), lower triangle, zero above.
__global__ void gram_to_df_kernel(float* G, int64_t ld, int64_t q, float* lo) {
  const int64_t total = q * q;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / q, j = e - i * q;
    float h = 0.0f, l = 0.0f;
    if (j < i) {
      h = G[i * ld + j];
    } else if (j == i) {
      const float g = G[i * ld + j];
      h = __fadd_rn(g, 1.0f);
      const float bb = __fsub_rn(h, g);
      l = __fadd_rn(__fsub_rn(g, __fsub_rn(h, bb)), __fsub_rn(1.0f, bb));   // TwoSum error, exact
    }
    G[i * ld + j] = h;
    lo[i * ld + j] = l;
  }
}

}  // namespace

int chol_mixed(float* G, float* Hlo, int64_t ldh, int64_t q, float* Lf, int64_t ldf, float* Md, int64_t ldm,
               int* err, cudaStream_t s) {
  if ((ldh | ldf | ldm) & 3) return POGS_ERR_ARG;   // 16-byte rows for the vector loads
  if (cudaFuncSetAttribute(chol_diag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDiagSmem) !=
      cudaSuccess)
    return POGS_ERR_CUDA;
  count_launch();
  gram_to_df_kernel<<<(int)std::min<int64_t>(cdiv(q * q, 256), 148 * 16), 256, 0, s>>>(G, ldh, q, Hlo);
  float* Hhi = G;
  // Lookahead: stream `ca` (highest priority) runs the critical chain -- diagonal block k,
  // panel k, and the update of block column k+1 by panel k; stream `cb` (lowest priority)
  // updates the remaining columns (>= k+2) by panel k, overlapping the next diagonal block and
  // panel.  Both write block column k+1 (cb with panel k-1, ca with panel k), so the critical
  // update of step k waits for cb's update of step k-1; every other pair touches disjoint
  // blocks or is ordered within one stream.
  int lo = 0, hi = 0;
  cudaDeviceGetStreamPriorityRange(&lo, &hi);
  cudaStream_t ca = nullptr, cb = nullptr;
  cudaEvent_t e_fork = nullptr, e_panel = nullptr, e_rest = nullptr, e_a = nullptr, e_b = nullptr;
  int rc = 0;
  if (cudaStreamCreateWithPriority(&ca, cudaStreamNonBlocking, hi) != cudaSuccess ||
      cudaStreamCreateWithPriority(&cb, cudaStreamNonBlocking, lo) != cudaSuccess ||
      cudaEventCreateWithFlags(&e_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&e_panel, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&e_rest, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&e_a, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&e_b, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    rc = POGS_ERR_CUDA;
  }
  if (rc == 0) {
    cudaEventRecord(e_fork, s);
    cudaStreamWaitEvent(ca, e_fork, 0);
    cudaStreamWaitEvent(cb, e_fork, 0);
    bool rest_pending = false;
    for (int64_t k0 = 0; k0 < q; k0 += kDB) {
      const int nb = (int)std::min<int64_t>(kDB, q - k0);
      count_launch();
      chol_diag_kernel<<<1, kDiagThreads, kDiagSmem, ca>>>(Hhi + k0 * ldh + k0, ldh, nb, Md + k0 * ldm + k0, ldm, err);
      const int64_t rest = q - k0 - nb;
      if (rest <= 0) break;
      // L21 = H21 W_kk^T (from the hi part: the pair rounds to hi)
      sgemm_launch<true, OUT_F32, 2>(rest, kDB, kDB, Hhi + (k0 + kDB) * ldh + k0, ldh, Md + k0 * ldm + k0, ldm,
                                     1.0f, Lf + (k0 + kDB) * ldf + k0, nullptr, ldf, false, 0, ca);
      cudaEventRecord(e_panel, ca);
      const float* P = Lf + (k0 + kDB) * ldf + k0;
      const int64_t nb1 = std::min<int64_t>(kDB, rest);
      // critical: block column k+1 (all rows below k) by panel k, after cb's update by panel k-1
      if (rest_pending) cudaStreamWaitEvent(ca, e_rest, 0);
      sgemm_launch<true, OUT_SUB_DF, 2>(rest, nb1, kDB, P, ldf, P, ldf, 1.0f, Hhi + (k0 + kDB) * ldh + k0 + kDB,
                                        Hlo + (k0 + kDB) * ldh + k0 + kDB, ldh, false, 0, ca);
      // the rest: columns >= k+2 (lower tiles) by panel k, overlapped
      const int64_t rest2 = rest - nb1;
      if (rest2 > 0) {
        cudaStreamWaitEvent(cb, e_panel, 0);
        const float* P2 = P + nb1 * ldf;
        sgemm_launch<true, OUT_SUB_DF, 2>(rest2, rest2, kDB, P2, ldf, P2, ldf, 1.0f,
                                          Hhi + (k0 + kDB + nb1) * ldh + k0 + kDB + nb1,
                                          Hlo + (k0 + kDB + nb1) * ldh + k0 + kDB + nb1, ldh, true, 0, cb);
        cudaEventRecord(e_rest, cb);
        rest_pending = true;
      } else {
        rest_pending = false;
      }
    }
    // join both streams back into the caller's stream
    cudaEventRecord(e_a, ca);
    cudaEventRecord(e_b, cb);
    cudaStreamWaitEvent(s, e_a, 0);
    cudaStreamWaitEvent(s, e_b, 0);
    if (cudaGetLastError() != cudaSuccess) rc = POGS_ERR_CUDA;
  }
  for (cudaEvent_t e : {e_fork, e_panel, e_rest, e_a, e_b})
    if (e) cudaEventDestroy(e);
  if (ca) cudaStreamDestroy(ca);
  if (cb) cudaStreamDestroy(cb);
  return rc;
}

namespace {

// Recursive factorization and inversion of the Schur block [r0, r0 + n) (see chol_inv_mixed).
// The critical chain (leaves, L21, the Schur update, the right half, M21) runs on `s`; the
// product T = L21 M11 of each level needs only the left half and L21, so it runs on the side
// stream `s2` (its own tensor-core scratch) while the right half is factored, and M21 = -M22 T
// waits for it.  Each active level keeps its T in the work area, stacked: a level's T at `T`,
// its right half's levels above it.
struct RecCtx {
  float *Hhi, *Hlo;
  int64_t ldh;
  float* Lf;
  int64_t ldf;
  float* Md;
  int64_t ldm;
  TcScratch tc, tc2;
  cudaStream_t s, s2;
  std::vector<cudaEvent_t>* events;
};

cudaEvent_t rec_event(const RecCtx& c) {
  cudaEvent_t e = nullptr;
  if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  c.events->push_back(e);
  return e;
}

void chol_inv_rec(const RecCtx& c, int64_t r0, int64_t n, float* T) {
  if (n <= kDB) {
    count_launch();
    chol_diag_kernel<<<1, kDiagThreads, kDiagSmem, c.s>>>(c.Hhi + r0 * c.ldh + r0, c.ldh, (int)n, c.Md + r0 * c.ldm + r0,
                                                 c.ldm, c.tc.err);
    return;
  }
  const int64_t n1 = (cdiv(n, kDB) / 2) * kDB, n2 = n - n1, r1 = r0 + n1;
  chol_inv_rec(c, r0, n1, T);
  const bool tc = c.tc.p && std::min(n1, n2) >= kTcInvMin;
  const float* H21 = c.Hhi + r1 * c.ldh + r0;
  const float* M11 = c.Md + r0 * c.ldm + r0;
  float* L21 = c.Lf + r1 * c.ldf + r0;
  // L21 = H21 M11^T (from the hi part: the pair rounds to hi)
  if (!(tc && tc_gemm_tf32x3(n2, n1, n1, H21, c.ldh, false, M11, c.ldm, false, 1.0f, L21, nullptr, c.ldf,
                             TC_EPI_STORE, false, c.tc.p, c.tc.bytes, nullptr, c.tc.err, c.s) == 0))
    sgemm_launch<true, OUT_F32, 2>(n2, n1, n1, H21, c.ldh, M11, c.ldm, 1.0f, L21, nullptr, c.ldf, false, 0, c.s);
  // T = L21 M11 on the side stream, overlapping everything below until M21
  cudaEvent_t e_l21 = rec_event(c), e_t = rec_event(c);
  const bool side = c.s2 && e_l21 && e_t;
  cudaStream_t st = side ? c.s2 : c.s;
  if (side) {
    cudaEventRecord(e_l21, c.s);
    cudaStreamWaitEvent(c.s2, e_l21, 0);
  }
  const bool tc_side = tc && (side ? c.tc2.p != nullptr : true);
  const TcScratch& ts = side ? c.tc2 : c.tc;
  if (!(tc_side && tc_gemm_nn_tf32x3(n2, n1, n1, L21, c.ldf, M11, c.ldm, 1.0f, T, n1, ts.p, ts.bytes, nullptr,
                                     ts.err, st) == 0))
    sgemm_launch<false, OUT_F32, 1>(n2, n1, n1, L21, c.ldf, M11, c.ldm, 1.0f, T, nullptr, n1, false, 1, st);
  if (side) cudaEventRecord(e_t, c.s2);
  // H22 -= L21 L21^T on the double-float pair (lower triangle)
  float* H22 = c.Hhi + r1 * c.ldh + r1;
  float* H22lo = c.Hlo + r1 * c.ldh + r1;
  if (!(tc && tc_gemm_tf32x3(n2, n2, n1, L21, c.ldf, false, L21, c.ldf, false, 1.0f, H22, H22lo, c.ldh,
                             TC_EPI_DF_SUB, true, c.tc.p, c.tc.bytes, nullptr, c.tc.err, c.s) == 0))
    sgemm_launch<true, OUT_SUB_DF, 2>(n2, n2, n1, L21, c.ldf, L21, c.ldf, 1.0f, H22, H22lo, c.ldh, true, 0, c.s);
  chol_inv_rec(c, r1, n2, T + n2 * n1);
  // M21 = -M22 T: the off-diagonal block of the inverse
  if (side) cudaStreamWaitEvent(c.s, e_t, 0);
  const float* M22 = c.Md + r1 * c.ldm + r1;
  float* M21 = c.Md + r1 * c.ldm + r0;
  if (tc && tc_gemm_nn_tf32x3(n2, n1, n2, M22, c.ldm, T, n1, -1.0f, M21, c.ldm, c.tc.p, c.tc.bytes, nullptr,
                              c.tc.err, c.s) == 0)
    return;
  sgemm_launch<false, OUT_F32, 1>(n2, n1, n2, M22, c.ldm, T, n1, -1.0f, M21, nullptr, c.ldm, false, 2, c.s);
}

}  // namespace

int chol_inv_mixed(float* G, float* Hlo, int64_t ldh, int64_t q, float* Lf, int64_t ldf, float* Md, int64_t ldm,
                   float* work, int* err, cudaStream_t s) {
  if ((ldh | ldf | ldm) & 3) return POGS_ERR_ARG;   // 16-byte rows for the vector loads
  if (cudaFuncSetAttribute(chol_diag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDiagSmem) !=
      cudaSuccess)
    return POGS_ERR_CUDA;
  count_launch();
  gram_to_df_kernel<<<(int)std::min<int64_t>(cdiv(q * q, 256), 148 * 16), 256, 0, s>>>(G, ldh, q, Hlo);
  std::vector<cudaEvent_t> events;
  RecCtx c{G, Hlo, ldh, Lf, ldf, Md, ldm, TcScratch{nullptr, 0, err}, TcScratch{nullptr, 0, err}, s, nullptr, &events};
  const int64_t n1 = (cdiv(q, kDB) / 2) * kDB, n2 = q - n1;
  if (std::min(n1, n2) >= kTcInvMin) {
    // the top level's products are the largest; every lower level fits in their scratch
    size_t need[4] = {0, 0, 0, 0};
    int rc = tc_gemm_tf32x3(n2, n1, n1, G, ldh, false, Md, ldm, false, 1.0f, Lf, nullptr, ldf, TC_EPI_STORE, false,
                            nullptr, 0, &need[0], err, s);
    rc |= tc_gemm_tf32x3(n2, n2, n1, Lf, ldf, false, Lf, ldf, false, 1.0f, G, Hlo, ldh, TC_EPI_DF_SUB, true,
                         nullptr, 0, &need[1], err, s);
    rc |= tc_gemm_nn_tf32x3(n2, n1, n1, Lf, ldf, Md, ldm, 1.0f, work, n1, nullptr, 0, &need[2], err, s);
    rc |= tc_gemm_nn_tf32x3(n2, n1, n2, Md, ldm, work, n1, -1.0f, Md, ldm, nullptr, 0, &need[3], err, s);
    if (rc == 0) {
      c.tc.bytes = std::max(std::max(need[0], need[1]), std::max(need[2], need[3]));
      if (pool_alloc(&c.tc.p, c.tc.bytes, s) != 0) c.tc.p = nullptr;
      c.tc2.bytes = need[2];
      if (pool_alloc(&c.tc2.p, c.tc2.bytes, s) != 0) c.tc2.p = nullptr;
    }
  }
  // side stream for the T products (lowest priority: the critical chain goes first)
  int lo = 0, hi = 0;
  cudaDeviceGetStreamPriorityRange(&lo, &hi);
  cudaStream_t s2 = nullptr;
  cudaEvent_t e_fork = nullptr, e_join = nullptr;
  if (cudaStreamCreateWithPriority(&s2, cudaStreamNonBlocking, lo) == cudaSuccess &&
      cudaEventCreateWithFlags(&e_fork, cudaEventDisableTiming) == cudaSuccess &&
      cudaEventCreateWithFlags(&e_join, cudaEventDisableTiming) == cudaSuccess) {
    cudaEventRecord(e_fork, s);   // the side stream starts after everything before this call
    cudaStreamWaitEvent(s2, e_fork, 0);
    c.s2 = s2;
  } else {
    cudaGetLastError();
  }
  chol_inv_rec(c, 0, q, work);
  if (c.s2) {   // join: the caller's stream continues after the side stream's last product
    cudaEventRecord(e_join, s2);
    cudaStreamWaitEvent(s, e_join, 0);
  }
  if (c.tc.p) cudaFreeAsync(c.tc.p, s);
  if (c.tc2.p) cudaFreeAsync(c.tc2.p, s);
  for (cudaEvent_t e : events)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : {e_fork, e_join})
    if (e) cudaEventDestroy(e);
  if (s2) cudaStreamDestroy(s2);
  return cudaGetLastError() == cudaSuccess ? 0 : POGS_ERR_CUDA;
}

int tri_inverse_f32(const float* L, int64_t ldl, int64_t q, float* M, int64_t ldm, float* work, bool tensor,
                    int* err, cudaStream_t s) {
  TcScratch tc{nullptr, 0, err};
  if (tensor && q > kTile) {
    // the top level's two products are the largest; every lower level fits in their scratch
    const int64_t n1 = (cdiv(q, kTile) / 2) * kTile, n2 = q - n1;
    size_t need1 = 0, need2 = 0;
    if (std::min(n1, n2) >= kTcInvMin &&
        tc_gemm_nn_tf32x3(n2, n1, n1, L, ldl, M, ldm, 1.0f, work, n1, nullptr, 0, &need1, err, s) == 0 &&
        tc_gemm_nn_tf32x3(n2, n1, n2, M, ldm, work, n1, -1.0f, M, ldm, nullptr, 0, &need2, err, s) == 0) {
      tc.bytes = std::max(need1, need2);
      if (pool_alloc(&tc.p, tc.bytes, s) != 0) tc.p = nullptr;
    }
  }
  inv_rec(L, ldl, M, ldm, 0, q, work, tc, s);
  if (tc.p) cudaFreeAsync(tc.p, s);
  return cudaGetLastError() == cudaSuccess ? 0 : POGS_ERR_CUDA;
}

}  // namespace pogs
