// One-time setup kernels: ingest of A, Sinkhorn-Knopp finish + Frobenius rescale
// (Algorithm 2, Section 4.1.2), the dense SIMT GEMM used for the FP32 Gram mode, the all-FP64
// blocked Cholesky of I + G (Section 3.5, factorization caching; the mixed-precision default
// is in chol.cu), the FP64 leaf inverses it needs, and the packing of M = L^{-1} into
// 128 x 128 tiles.
#include <algorithm>
#include <cstdio>

#include "kernels.h"

namespace pogs {

// ---- ingest --------------------------------------------------------------------------------
// Row-major (or column-major) source -> padded row-major A (pitch lda, zero padding),
// flagging non-finite entries.
// Block b takes rows b, b + grid, ...; a row moves as float4 words (four per thread in flight)
// when the source rows are 16-byte aligned, else one float at a time.  The destination pitch lda
// is a multiple of 4 floats and A is 16-byte aligned (the handle lays it out so); the same
// kernel also runs in place (src == A) to zero the padding and check a row-by-row host copy.
__global__ void __launch_bounds__(256) copy_rowmajor_kernel(const float* __restrict__ src, int64_t m, int64_t n,
                                                            int64_t lds, float* __restrict__ A, int64_t lda,
                                                            int* err) {
  const bool v4 = ((reinterpret_cast<uintptr_t>(src) | (uintptr_t)(lds * sizeof(float))) & 15) == 0;
  const int64_t nv = lda >> 2, nfull = n >> 2;   // float4 words per destination row; words wholly inside n
  int bad = 0;
  for (int64_t i = blockIdx.x; i < m; i += gridDim.x) {
    const float* sr = src + i * lds;
    float4* dr = reinterpret_cast<float4*>(A + i * lda);
    int64_t c = threadIdx.x;
    if (v4) {
      const float4* s4 = reinterpret_cast<const float4*>(sr);
      for (; c + 768 < nfull; c += 1024) {
        float4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = s4[c + 256 * u];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          bad |= !isfinite(v[u].x) | !isfinite(v[u].y) | !isfinite(v[u].z) | !isfinite(v[u].w);
          dr[c + 256 * u] = v[u];
        }
      }
      for (; c < nfull; c += 256) {
        const float4 v = s4[c];
        bad |= !isfinite(v.x) | !isfinite(v.y) | !isfinite(v.z) | !isfinite(v.w);
        dr[c] = v;
      }
    }
    for (; c < nv; c += 256) {   // the rest of the row one float at a time, zeros past n
      float w[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t j = 4 * c + u;
        w[u] = j < n ? sr[j] : 0.0f;
        if (j < n && !isfinite(w[u])) bad = 1;
      }
      dr[c] = make_float4(w[0], w[1], w[2], w[3]);
    }
  }
  if (bad) atomicCAS(err, 0, POGS_ERR_NONFINITE);   // first error wins
}

__global__ void copy_colmajor_kernel(const float* __restrict__ src, int64_t m, int64_t n, int64_t lds,
                                     float* __restrict__ A, int64_t lda, int* err) {
  __shared__ float t[32][33];
  const int64_t i0 = (int64_t)blockIdx.y * 32, j0 = (int64_t)blockIdx.x * 32;
  int bad = 0;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t j = j0 + r, i = i0 + threadIdx.x;   // read along i (contiguous in column-major)
    float v = 0.0f;
    if (i < m && j < n) {
      v = src[j * lds + i];
      if (!isfinite(v)) bad = 1;
    }
    t[r][threadIdx.x] = v;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t i = i0 + r, j = j0 + threadIdx.x;
    if (i < m && j < lda) A[i * lda + j] = (j < n) ? t[threadIdx.x][r] : 0.0f;
  }
  if (bad) atomicCAS(err, 0, POGS_ERR_NONFINITE);   // first error wins
}

void launch_copy_in(const float* src, int64_t m, int64_t n, int64_t lds, bool colmajor, float* A, int64_t lda,
                    int* err, cudaStream_t s) {
  if (!colmajor) {
    const int64_t g = std::min<int64_t>(m, 148 * 8);
    count_launch();
    copy_rowmajor_kernel<<<(int)g, 256, 0, s>>>(src, m, n, lds, A, lda, err);
  } else {
    dim3 grid((unsigned)cdiv(lda, 32), (unsigned)cdiv(m, 32));
    count_launch();
    copy_colmajor_kernel<<<grid, dim3(32, 8), 0, s>>>(src, m, n, lds, A, lda, err);
  }
}

// A^ = D A E in place (Section 4.1).  Block b takes rows b, b + grid, ...; float4 words of the
// row (pitch lda a multiple of 4 floats, A 16-byte aligned), each element times D_i E_j; the
// zero padding past n stays zero.
__global__ void __launch_bounds__(256) scale_kernel(float* __restrict__ A, int64_t lda, int64_t m, int64_t n,
                                                    const float* __restrict__ D, const float* __restrict__ E) {
  const int64_t nw = (n + 3) >> 2;   // words holding columns < n
  for (int64_t i = blockIdx.x; i < m; i += gridDim.x) {
    float4* r = reinterpret_cast<float4*>(A + i * lda);
    const float di = D[i];
    int64_t c = threadIdx.x;
    for (; c + 256 < nw; c += 512) {
      float4 v[2];
      float e[2][4];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        v[u] = r[c + 256 * u];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int64_t j = 4 * (c + 256 * u) + t;
          e[u][t] = j < n ? E[j] : 0.0f;
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        v[u].x *= di * e[u][0]; v[u].y *= di * e[u][1]; v[u].z *= di * e[u][2]; v[u].w *= di * e[u][3];
        r[c + 256 * u] = v[u];
      }
    }
    for (; c < nw; c += 256) {
      float4 v = r[c];
      float e[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int64_t j = 4 * c + t;
        e[t] = j < n ? E[j] : 0.0f;
      }
      v.x *= di * e[0]; v.y *= di * e[1]; v.z *= di * e[2]; v.w *= di * e[3];
      r[c] = v;
    }
  }
}

void launch_scale(float* A, int64_t lda, int64_t m, int64_t n, const float* D, const float* E, cudaStream_t s) {
  const int64_t g = std::min<int64_t>(m, 148 * 8);
  count_launch();
  scale_kernel<<<(int)g, 256, 0, s>>>(A, lda, m, n, D, E);
}

// D = sqrt(d / s), E = sqrt(e / s) with s = ||diag(d)^{1/2} A diag(e)^{1/2}||_F / sqrt(q):
// Algorithm 2's D = diag(d)^{1/p}, E = diag(e)^{1/p} (p = 2) rescaled evenly (Section 4.1.2).
__global__ void sk_finish_kernel(const float* dvec, const float* evec, int64_t m, int64_t n, const Df* frob_part,
                                 int nfrob, int64_t q, float* D, float* E) {
  __shared__ double sh[32];
  __shared__ double s_inv;
  double v[1] = {0.0};
  for (int i = threadIdx.x; i < nfrob; i += blockDim.x) v[0] += df_value(frob_part[2 * i]);
  block_sum<1>(v, sh);
  // A = 0: there is no norm to rescale to (the rescale is skipped)
  if (threadIdx.x == 0) s_inv = v[0] > 0.0 ? 1.0 / sqrt(v[0] / (double)q) : 1.0;
  __syncthreads();
  const double si = s_inv;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) D[i] = (float)sqrt((double)dvec[i] * si);
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) E[j] = (float)sqrt((double)evec[j] * si);
}

void launch_sk_finish(const float* dvec, const float* evec, int64_t m, int64_t n, const Df* frob_part, int nfrob,
                      int64_t q, float* D, float* E, cudaStream_t s) {
  count_launch();
  sk_finish_kernel<<<1, 1024, 0, s>>>(dvec, evec, m, n, frob_part, nfrob, q, D, E);
}

// ---- one Sinkhorn-Knopp sweep in one pass over A^ (Algorithm 2, p = 2) ----------------------
// For a row-major A (pitch lda, zero padding, lda <= 1024 kSkGroups floats): block b takes the
// rows [b R, b R + R) four at a time.  Two warps per row form the row sum of A_ij^2 e_j over
// their halves of the row (e staged in shared memory) and d_i = num_r / (sum + reg_r), which
// is written out; then every thread adds A_ij^2 d_i of the four rows into its columns'
// accumulators (lane-contiguous float4 groups, rows re-read from L2, where the first read left
// them).  That is Algorithm 2's d update followed by the column sums of its e update, with A
// streamed from HBM once per sweep instead of twice.  The block's column sums go to
// part[b][0, lda); sk_sweep_finish_kernel adds the blocks in order and forms e.
constexpr int kSkGroups = 12;   // float4 column groups per thread: lda <= 12288
constexpr int kSkBlocks = 296;  // two 256-thread blocks per SM

__global__ void __launch_bounds__(256, 2) sk_sweep_kernel(const float* __restrict__ A, int64_t lda, int m,
                                                          int rows_per_blk, const float* __restrict__ e_in,
                                                          float* __restrict__ d_out, float num_r, float reg_r,
                                                          float* __restrict__ part) {
  extern __shared__ float4 se4[];   // e over the padded row, lda / 4 groups
  __shared__ float psum[8];
  __shared__ float dsh[4];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ng = (int)(lda >> 2), half = (ng + 1) >> 1;
  for (int g = tid; g < ng; g += 256) se4[g] = reinterpret_cast<const float4*>(e_in)[g];
  __syncthreads();
  float4 acc[kSkGroups];
#pragma unroll
  for (int u = 0; u < kSkGroups; ++u) acc[u] = make_float4(0.f, 0.f, 0.f, 0.f);
  const int r0 = blockIdx.x * rows_per_blk, r1 = min(m, r0 + rows_per_blk);
  const uint64_t ps = l2_evict_first();
  for (int c = r0; c < r1; c += 4) {
    // row sums: warp w takes row c + w / 2, column groups [h half, h half + half), h = w % 2
    const int row = c + (warp >> 1);
    float sum = 0.0f;
    if (row < r1) {
      const float4* ar = reinterpret_cast<const float4*>(A + (int64_t)row * lda);
      const int g0 = (warp & 1) * half, g1 = min(ng, g0 + half);
      int g = g0 + lane;
      for (; g + 224 < g1; g += 256) {
        float4 a[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) a[u] = ar[g + 32 * u];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const float4 e = se4[g + 32 * u];
          sum = fmaf(a[u].x * a[u].x, e.x, sum); sum = fmaf(a[u].y * a[u].y, e.y, sum);
          sum = fmaf(a[u].z * a[u].z, e.z, sum); sum = fmaf(a[u].w * a[u].w, e.w, sum);
        }
      }
      for (; g < g1; g += 32) {
        const float4 a = ar[g], e = se4[g];
        sum = fmaf(a.x * a.x, e.x, sum); sum = fmaf(a.y * a.y, e.y, sum);
        sum = fmaf(a.z * a.z, e.z, sum); sum = fmaf(a.w * a.w, e.w, sum);
      }
    }
    sum = warp_sum(sum);
    if (lane == 0) psum[warp] = sum;
    __syncthreads();
    if (tid < 4 && c + tid < r1) {
      const float d = num_r / ((psum[2 * tid] + psum[2 * tid + 1]) + reg_r);
      dsh[tid] = d;
      d_out[c + tid] = d;
    }
    __syncthreads();
    // column sums of A_ij^2 d_i over the four rows, in row order
    const int nr = min(4, r1 - c);
    for (int k = 0; k < nr; ++k) {
      const float d = dsh[k];
      const float4* ar = reinterpret_cast<const float4*>(A + (int64_t)(c + k) * lda);
#pragma unroll
      for (int u = 0; u < kSkGroups; ++u) {
        const int g = tid + 256 * u;
        if (g < ng) {
          const float4 a = ldg_stream(ar + g, ps);
          acc[u].x = fmaf(a.x * a.x, d, acc[u].x); acc[u].y = fmaf(a.y * a.y, d, acc[u].y);
          acc[u].z = fmaf(a.z * a.z, d, acc[u].z); acc[u].w = fmaf(a.w * a.w, d, acc[u].w);
        }
      }
    }
  }
  float4* pb = reinterpret_cast<float4*>(part + (int64_t)blockIdx.x * lda);
#pragma unroll
  for (int u = 0; u < kSkGroups; ++u) {
    const int g = tid + 256 * u;
    if (g < ng) pb[g] = acc[u];
  }
}

// e_j = num_c / (sum_b part[b][j] + reg_c) for j < n (blocks added in order: warp w adds the
// blocks b = w, w + 8, ... for the block's 32 columns, then the eight warp sums in warp order)
// and the Frobenius partial sum_j e_j t_j = ||D A E||_F^2 of the block's columns into
// frob_part[2 blockIdx.x] (the second entry of the pair is 0).
__global__ void __launch_bounds__(256) sk_sweep_finish_kernel(const float* __restrict__ part, int nblk, int64_t lda,
                                                              int64_t n, float num_c, float reg_c,
                                                              float* __restrict__ e_out, Df* __restrict__ frob_part) {
  __shared__ float ws[8][32];
  __shared__ double sh[2 * 8];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t j = (int64_t)blockIdx.x * 32 + lane;
  float t = 0.0f;
  if (j < lda) {
    int b = warp;
    for (; b + 56 < nblk; b += 64) {
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = __ldcg(part + (int64_t)(b + 8 * u) * lda + j);
#pragma unroll
      for (int u = 0; u < 8; ++u) t += v[u];
    }
    for (; b < nblk; b += 8) t += __ldcg(part + (int64_t)b * lda + j);
  }
  ws[warp][lane] = t;
  __syncthreads();
  Df res[2] = {};
  if (warp == 0 && j < n) {
    float tj = 0.0f;
#pragma unroll
    for (int w = 0; w < 8; ++w) tj += ws[w][lane];
    const float ej = num_c / (tj + reg_c);
    e_out[j] = ej;
    df_add_prod(res[0], ej, tj);
  }
  double tot[2];
  block_sum_df<2>(res, tot, sh);
  if (tid == 0) {
    const float hi = (float)tot[0];
    frob_part[2 * blockIdx.x] = Df{hi, (float)(tot[0] - (double)hi)};
    frob_part[2 * blockIdx.x + 1] = Df{0.0f, 0.0f};
  }
}

bool sk_sweep_fits(int64_t m, int64_t lda) { return lda <= 1024 * kSkGroups && m >= 8 * kSkBlocks; }
int sk_sweep_blocks() { return kSkBlocks; }
int sk_sweep_finish_blocks(int64_t lda) { return (int)cdiv(lda, 32); }

int launch_sk_sweep(const float* A, int64_t lda, int64_t m, int64_t n, float* dvec, float* evec, double gamma,
                    float* part, Df* frob_part, cudaStream_t s) {
  const int rows = (int)round_up(cdiv(m, kSkBlocks), 4);
  const int smem = (int)(lda * sizeof(float));
  static PerDeviceOnce attr;
  if (attr.run([&] {
        return cudaFuncSetAttribute(sk_sweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    1024 * kSkGroups * (int)sizeof(float)) == cudaSuccess
                   ? 0
                   : -1;
      }) != 0) {
    cudaGetLastError();
    return POGS_ERR_CUDA;
  }
  count_launch(2);
  sk_sweep_kernel<<<kSkBlocks, 256, smem, s>>>(A, lda, (int)m, rows, evec, dvec, (float)n, (float)(gamma / (double)m),
                                              part);
  sk_sweep_finish_kernel<<<sk_sweep_finish_blocks(lda), 256, 0, s>>>(part, kSkBlocks, lda, n, (float)m,
                                                                     (float)(gamma / (double)n), evec, frob_part);
  return cudaGetLastError() == cudaSuccess ? 0 : POGS_ERR_CUDA;
}

// ---- dense SIMT GEMM -----------------------------------------------------------------------
// C = alpha op(A) op(B) + beta C, row-major, storage type TI, products and accumulation in
// TC (TI = double with TC = float gives FP32 products of FP32-rounded inputs added to an FP64
// C).  op(A)[i][k] = TA ? A[k*lda+i] : A[i*lda+k], op(B)[k][j] = TB ? B[j*ldb+k] : B[k*ldb+j].
// 256 threads, (BM/TM) x (BN/TN) = 16 x 16 thread grid, interleaved register tiles
// (conflict-free shared reads).  `tri` skips structurally zero K ranges: bit 0 -- op(B) lower
// triangular (op(B)[k][j] = 0 for k < j); bit 1 -- op(A) lower triangular (0 for k > i).
template <typename TI, typename TC, int BM, int BN, int BK, int TM, int TN, bool TA, bool TB>
__global__ void __launch_bounds__(256) gemm_kernel(int64_t M, int64_t N, int64_t K, TI alpha, const TI* A,
                                                   int64_t lda, const TI* B, int64_t ldb, TI beta, TI* C,
                                                   int64_t ldc, int lower_only, int tri) {
  // A and C may alias (in-place panel update): each block reads its own rows of A fully
  // before it writes C, and no other block touches those rows.
  constexpr int GX = BN / TN, GY = BM / TM;
  static_assert(GX * GY == 256, "thread grid");
  const int64_t bm = blockIdx.y, bn = blockIdx.x;
  const int64_t row0 = (int64_t)bm * BM, col0 = (int64_t)bn * BN;
  if (lower_only && col0 > row0 + BM - 1) return;
  __shared__ TC As[BK][BM + 1];
  __shared__ TC Bs[BK][BN + 1];
  const int tx = threadIdx.x % GX, ty = threadIdx.x / GX;
  TC acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = TC(0);
  const int64_t kbeg = (tri & 1) ? (col0 / BK) * BK : 0;
  const int64_t kend = (tri & 2) ? (row0 + BM < K ? row0 + BM : K) : K;
  for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
    for (int e = threadIdx.x; e < BM * BK; e += 256) {
      int i, k;
      if (TA) { k = e / BM; i = e % BM; } else { i = e / BK; k = e % BK; }
      const int64_t gi = row0 + i, gk = k0 + k;
      TC v = TC(0);
      if (gi < M && gk < K) v = (TC)(TA ? A[gk * lda + gi] : A[gi * lda + gk]);
      As[k][i] = v;
    }
    for (int e = threadIdx.x; e < BN * BK; e += 256) {
      int j, k;
      if (TB) { j = e / BK; k = e % BK; } else { k = e / BN; j = e % BN; }
      const int64_t gj = col0 + j, gk = k0 + k;
      TC v = TC(0);
      if (gj < N && gk < K) v = (TC)(TB ? B[gj * ldb + gk] : B[gk * ldb + gj]);
      Bs[k][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      TC a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[k][ty + i * GY];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[k][tx + j * GX];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int64_t gi = row0 + ty + i * GY;
    if (gi >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int64_t gj = col0 + tx + j * GX;
      if (gj >= N) continue;
      TI c = alpha * (TI)acc[i][j];
      if (beta != TI(0)) c = fma(beta, C[gi * ldc + gj], c);
      C[gi * ldc + gj] = c;
    }
  }
}

template <typename TI, typename TC, int BM, int BN, int BK, int TM, int TN>
static void gemm_launch(bool ta, bool tb, int64_t M, int64_t N, int64_t K, TI alpha, const TI* A, int64_t lda,
                        const TI* B, int64_t ldb, TI beta, TI* C, int64_t ldc, bool lower_only, int tri,
                        cudaStream_t s) {
  if (M <= 0 || N <= 0) return;
  count_launch();
  dim3 grid((unsigned)cdiv(N, BN), (unsigned)cdiv(M, BM));
  const int lo = lower_only ? 1 : 0;
#define POGS_G(a, b) gemm_kernel<TI, TC, BM, BN, BK, TM, TN, a, b><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, lo, tri)
  if (!ta && !tb) POGS_G(false, false);
  else if (!ta && tb) POGS_G(false, true);
  else if (ta && !tb) POGS_G(true, false);
  else POGS_G(true, true);
#undef POGS_G
}

void gemm_f32(bool ta, bool tb, int64_t M, int64_t N, int64_t K, float alpha, const float* A, int64_t lda,
              const float* B, int64_t ldb, float beta, float* C, int64_t ldc, bool lower_only, cudaStream_t s,
              int tri) {
  gemm_launch<float, float, 128, 128, 8, 8, 8>(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, lower_only,
                                               tri, s);
}
void gemm_f64(bool ta, bool tb, int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t lda,
              const double* B, int64_t ldb, double beta, double* C, int64_t ldc, bool lower_only, cudaStream_t s) {
  gemm_launch<double, double, 64, 64, 8, 4, 4>(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, lower_only, 0,
                                               s);
}

// H = I + G (lower triangle, FP64), zero above the diagonal.
__global__ void gram_to_f64_kernel(const float* G, int64_t ldg, int64_t q, double* H, int64_t ldh) {
  const int64_t total = q * q;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / q, j = e - i * q;
    double v = 0.0;
    if (j <= i) v = (double)G[i * ldg + j] + (i == j ? 1.0 : 0.0);
    H[i * ldh + j] = v;
  }
}
void launch_gram_to_f64(const float* G, int64_t ldg, int64_t q, double* H, int64_t ldh, cudaStream_t s) {
  int64_t g = std::min<int64_t>((q * q + 255) / 256, 148 * 16);
  count_launch();
  gram_to_f64_kernel<<<(int)g, 256, 0, s>>>(G, ldg, q, H, ldh);
}

// ---- FP64 blocked Cholesky (right-looking) ------------------------------------------------
constexpr int kNB = 64;

// Factor the nb x nb diagonal block in place and write its inverse factor to Linv (ld kNB).
// The inverse is built column by column (forward substitution on e_c, one column per
// thread) and kept transposed in the strict upper triangle of the same shared tile.
__global__ void __launch_bounds__(256) potrf_diag_kernel(double* Hk, int64_t ldh, int nb, double* Linv, int* err) {
  __shared__ double s[kNB][kNB + 1];
  __shared__ double dl[kNB], dx[kNB];
  const int tid = threadIdx.x;
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e % nb;
    s[i][j] = (j <= i) ? Hk[(int64_t)i * ldh + j] : 0.0;
  }
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (tid == 0) {
      double djj = s[j][j];
      if (!(djj > 0.0) || !isfinite(djj)) {
        atomicCAS(err, 0, POGS_ERR_NUMERIC);
        djj = 1.0;
      }
      s[j][j] = sqrt(djj);
    }
    __syncthreads();
    const double ljj = s[j][j];
    for (int i = j + 1 + tid; i < nb; i += blockDim.x) s[i][j] /= ljj;
    __syncthreads();
    const int rem = nb - j - 1;
    for (int e = tid; e < rem * rem; e += blockDim.x) {
      const int i = j + 1 + e / rem, k = j + 1 + e % rem;
      if (k <= i) s[i][k] -= s[i][j] * s[k][j];
    }
    __syncthreads();
  }
  if (tid < nb) dl[tid] = s[tid][tid];
  __syncthreads();
  if (tid < nb) {
    const int c = tid;
    const double xcc = 1.0 / dl[c];
    dx[c] = xcc;
    for (int i = c + 1; i < nb; ++i) {
      double acc = -s[i][c] * xcc;
      for (int k = c + 1; k < i; ++k) acc -= s[i][k] * s[c][k];   // X[k][c] lives at s[c][k]
      s[c][i] = acc / dl[i];
    }
  }
  __syncthreads();
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e % nb;
    Hk[(int64_t)i * ldh + j] = (j < i) ? s[i][j] : (j == i ? dl[i] : 0.0);
    Linv[i * kNB + j] = (j < i) ? s[j][i] : (j == i ? dx[i] : 0.0);
  }
}

int chol_f64(double* H, int64_t ldh, int64_t q, double* work, int* err, cudaStream_t s) {
  for (int64_t k0 = 0; k0 < q; k0 += kNB) {
    const int nb = (int)std::min<int64_t>(kNB, q - k0);
    count_launch();
    potrf_diag_kernel<<<1, 256, 0, s>>>(H + k0 * ldh + k0, ldh, nb, work, err);
    const int64_t rest = q - k0 - nb;
    if (rest > 0) {
      double* P = H + (k0 + nb) * ldh + k0;
      // panel: P <- P L_kk^{-T} (in place: one block column covers all nb <= 64 columns)
      gemm_f64(false, true, rest, nb, nb, 1.0, P, ldh, work, kNB, 0.0, P, ldh, false, s);
      // trailing update: H22 <- H22 - P P^T (lower tiles), all in FP64
      gemm_f64(false, true, rest, rest, nb, -1.0, P, ldh, P, ldh, 1.0, H + (k0 + nb) * ldh + (k0 + nb), ldh, true, s);
    }
  }
  return 0;
}

// ---- FP32 inverse factor M = L^{-1} ---------------------------------------------------------
// Diagonal 128 x 128 blocks of M inverted in FP64 from the FP64 factor (one block per CTA,
// one column per thread, forward substitution on e_c), written as FP32.  Column c of the
// inverse is kept transposed in the strict upper triangle of the shared tile.
__global__ void __launch_bounds__(128) leaf_inverse_kernel(const double* L, int64_t ldl, int64_t q, float* M,
                                                           int64_t ldm) {
  extern __shared__ double sm[];
  double* s = sm;                        // [128][129]
  double* dl = sm + 128 * 129;           // [128] diagonal of L
  const int64_t r0 = (int64_t)blockIdx.x * kTile;
  const int nb = (int)(q - r0 < kTile ? q - r0 : kTile);
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e % nb;
    if (j < i) s[i * 129 + j] = L[(r0 + i) * ldl + r0 + j];
    else if (j == i) dl[i] = L[(r0 + i) * ldl + r0 + j];
  }
  __syncthreads();
  const int c = threadIdx.x;
  if (c < nb) {
    const double xcc = 1.0 / dl[c];
    M[(r0 + c) * ldm + r0 + c] = (float)xcc;
    for (int i = c + 1; i < nb; ++i) {
      double acc = -s[i * 129 + c] * xcc;
      for (int k = c + 1; k < i; ++k) acc -= s[i * 129 + k] * s[c * 129 + k];
      const double v = acc / dl[i];
      s[c * 129 + i] = v;
      M[(r0 + i) * ldm + r0 + c] = (float)v;
    }
  }
}

void launch_leaf_inverse(const double* L, int64_t ldl, int64_t q, float* Minv, int64_t ldm, cudaStream_t s) {
  const int T = (int)cdiv(q, kTile);
  const size_t smem = (size_t)(128 * 129 + 128) * sizeof(double);
  cudaFuncSetAttribute(leaf_inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  count_launch();
  leaf_inverse_kernel<<<T, 128, smem, s>>>(L, ldl, q, Minv, ldm);
}

__global__ void l_to_f32_kernel(const double* L, int64_t ldl, int64_t q, float* Lf, int64_t ldf) {
  const int64_t total = q * q;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / q, j = e - i * q;
    Lf[i * ldf + j] = (j <= i) ? (float)L[i * ldl + j] : 0.0f;
  }
}
void launch_l_to_f32(const double* L, int64_t ldl, int64_t q, float* Lf, int64_t ldf, cudaStream_t s) {
  int64_t g = std::min<int64_t>((q * q + 255) / 256, 148 * 16);
  count_launch();
  l_to_f32_kernel<<<(int)g, 256, 0, s>>>(L, ldl, q, Lf, ldf);
}

// Pack the lower triangle of M (dense, ld ldm) into 128 x 128 tiles, zero outside.
__global__ void __launch_bounds__(256) pack_tiles_kernel(const float* M, int64_t ldm, int64_t q, float* Mt,
                                                         bool sym) {
  const int b = blockIdx.x;
  int I = (int)((sqrtf(8.0f * (float)b + 1.0f) - 1.0f) * 0.5f);
  while ((I + 1) * (I + 2) / 2 <= b) ++I;
  while (I * (I + 1) / 2 > b) --I;
  const int J = b - I * (I + 1) / 2;
  float* out = Mt + (int64_t)b * kTile * kTile;
  for (int e = threadIdx.x; e < kTile * kTile; e += blockDim.x) {
    const int rr = e / kTile, cc = e % kTile;
    const int64_t gi = (int64_t)I * kTile + rr, gj = (int64_t)J * kTile + cc;
    out[e] = (gi < q && gj < q && (gj <= gi || sym)) ? M[gi * ldm + gj] : 0.0f;
  }
}
void launch_pack_tiles(const float* M, int64_t ldm, int64_t q, int T, float* Mt, cudaStream_t s, bool sym) {
  count_launch();
  pack_tiles_kernel<<<T * (T + 1) / 2, 256, 0, s>>>(M, ldm, q, Mt, sym);
}

}  // namespace pogs
