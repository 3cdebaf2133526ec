// Per-iteration kernels of graph-form ADMM (Algorithm 1 + Section 3.2 over-relaxation +
// Section 3.4 stopping + Algorithm 3), all on the pre-conditioned problem (Eq. 12).
//
// One iteration, tall case (m >= n), reading A^ twice and the cached factor twice:
//   prox_step   : x^{1/2}, y^{1/2}, mu^{1/2}, nu^{1/2}, relaxed c = x_r, d = y_r        (m+n elts)
//   gemv_t      : [t, s, u] = A^T [d, nu^{1/2}, y~] -> r = c + t, ||s + mu||, x~ = -u   (A pass 1)
//   trmv (N)    : z = L^{-1} r                                                          (L pass 1)
//   trmv (T)    : x^{k+1} = L^{-T} z, x~ += c - x^{k+1}                                 (L pass 2)
//   gemv_n      : [y^{k+1}, w] = A [x^{k+1}, x^{1/2}] -> y~ += d - y^{k+1}, ||w - y^{1/2}|| (A pass 2)
//   check       : Section 3.4 test, gap, Algorithm 3, graph conditional
// The fat case (m < n) swaps the roles of the two GEMVs (Section 3.5 reduced update).
//
// Algorithm 1 projects (x_r + x~, y_r + y~).  Here the projection takes (x_r, y_r) and x~ is
// re-derived from y~ as -A^T y~ once per iteration (a third right-hand side of the column-sum
// pass, no extra traffic on A).  Both are identities of the method: the Section 3.3 invariant
// x~ + A^T y~ = 0 makes (x~, y~) orthogonal to the graph, so Pi(x_r + x~, y_r + y~) =
// Pi(x_r, y_r).  In FP32 the difference matters once rho is small: x~, y~ grow like 1/rho, and
// projecting their sum with the O(1) relaxed point loses that many digits, while updating
// x~ additively without re-deriving it lets the invariant drift.
#include <cstdio>

#include "kernels.h"
#include "epi.cuh"
#include "prox.cuh"

namespace pogs {

// ------------------------------------------------------------------------------------------
// Prox step (Algorithm 1 step 3, Section 3.2, Section 3.3).
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) prox_step_kernel(
    int n, int m, const float* __restrict__ x, float* __restrict__ xt, float* __restrict__ xh,
    float* __restrict__ cx, float* __restrict__ mu, const float* __restrict__ y,
    float* __restrict__ yt, float* __restrict__ yh, float* __restrict__ dy,
    float* __restrict__ nu, FnDev g, FnDev f, const DevState* __restrict__ st,
    const DevCfg* __restrict__ cfg, Df* __restrict__ part) {
  __shared__ double sh[6 * 8];
  if (st->done) return;
  const float rho = (float)st->rho;
  const float pend = (float)st->pend;
  const float alpha = (float)cfg->alpha;
  Df acc[6] = {};   // ||mu||^2, x.mu, g(x), ||y||^2, y.nu, f(y)
  const int total = n + m;
  const bool rescale = pend != 1.0f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    if (i < n) {
      const int j = i;
      const float xtj = pend * xt[j], xj = x[j], v = xj - xtj;
      if (rescale) xt[j] = xtj;   // Section 3.2: x~ <- (rho^k / rho^{k+1}) x~
      const int h = g.h[j];
      const float a = g.a[j], b = g.b[j], c = g.c[j], d = g.d[j], e = g.e[j];
      const float xhj = prox_param(h, a, b, c, d, e, rho, v);
      const float muj = -rho * (xhj - v);
      const float xr = alpha * xhj + (1.0f - alpha) * xj;
      xh[j] = xhj;
      cx[j] = xr;
      mu[j] = muj;
      df_add_prod(acc[0], muj, muj);
      df_add_prod(acc[1], xhj, muj);
      df_add(acc[2], f_param(h, a, b, c, d, e, xhj));
    } else {
      const int k = i - n;
      const float ytk = pend * yt[k], yk = y[k], v = yk - ytk;
      if (rescale) yt[k] = ytk;
      const int h = f.h[k];
      const float a = f.a[k], b = f.b[k], c = f.c[k], d = f.d[k], e = f.e[k];
      const float yhk = prox_param(h, a, b, c, d, e, rho, v);
      const float nuk = -rho * (yhk - v);
      const float yr = alpha * yhk + (1.0f - alpha) * yk;
      yh[k] = yhk;
      dy[k] = yr;
      nu[k] = nuk;
      df_add_prod(acc[3], yhk, yhk);
      df_add_prod(acc[4], yhk, nuk);
      df_add(acc[5], f_param(h, a, b, c, d, e, yhk));
    }
  }
  double tot[6];
  block_sum_df<6>(acc, tot, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int t = 0; t < 6; ++t) {
      const float hi = (float)tot[t];
      part[blockIdx.x * 6 + t] = Df{hi, (float)(tot[t] - (double)hi)};
    }
  }
}

void launch_prox_step(int n, int m, const float* x, float* xt, float* xh, float* cx, float* mu,
                      const float* y, float* yt, float* yh, float* dy, float* nu, FnDev g, FnDev f,
                      const DevState* st, const DevCfg* cfg, Df* part, int nblocks, cudaStream_t s) {
  count_launch();
  prox_step_kernel<<<nblocks, 256, 0, s>>>(n, m, x, xt, xh, cx, mu, y, yt, yh, dy, nu, g, f, st, cfg, part);
}

// ------------------------------------------------------------------------------------------
// Column sums t = A^T [v1, v2] (A row-major m x lda, zero-padded columns).  Block (bx, by)
// streams rows [by*R, by*R+R) of the 1024-column slab bx (256 threads x float4); partial
// sums go to part[by][rhs][col]; with FIN, the last block of each slab reduces the splits in a
// fixed order and applies the epilogue; without, the launch only streams and
// pogs_colsum_finish_kernel (the next launch) does the same reduction with every slab's
// partials in flight at once.
// ------------------------------------------------------------------------------------------
template <int NRHS, bool SQ, int EPI, bool FIN = true>
__global__ void __launch_bounds__(256, 5) pogs_colsum_kernel(const float* __restrict__ A, int64_t lda, int m, int n,
                                                     const float* __restrict__ v1,
                                                     const float* __restrict__ v2,
                                                     const float* __restrict__ v3, int rows, int keep_rows,
                                                     float* __restrict__ part, unsigned* __restrict__ cnt,
                                                     EpiArgs ep, const DevState* __restrict__ guard) {
  __shared__ double sh[2 * 8];
  if (guard && guard->done) return;
  if (ep.cg_done && *ep.cg_done) return;
  const int tid = threadIdx.x;
  const int64_t c0 = (int64_t)blockIdx.x * 1024 + 4 * tid;
  const bool active = c0 < lda;
  const int r0 = blockIdx.y * rows;
  const int r1 = min(m, r0 + rows);
  float acc[NRHS][4];
#pragma unroll
  for (int r = 0; r < NRHS; ++r) acc[r][0] = acc[r][1] = acc[r][2] = acc[r][3] = 0.0f;
  if (active) {
    const float* Ap = A + c0;
    const uint64_t ps = l2_evict_first(), pk = l2_evict_last();
    int i = r0;
    for (; i + 8 <= r1; i += 8) {
      float4 a[8];
      const uint64_t pol = i < keep_rows ? pk : ps;   // by the batch's first row
#pragma unroll
      for (int u = 0; u < 8; ++u)
        a[u] = ldg_stream(reinterpret_cast<const float4*>(Ap + (int64_t)(i + u) * lda), pol);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        float4 av = a[u];
        if (SQ) { av.x *= av.x; av.y *= av.y; av.z *= av.z; av.w *= av.w; }
        const float w1 = __ldg(v1 + i + u);
        acc[0][0] = fmaf(av.x, w1, acc[0][0]); acc[0][1] = fmaf(av.y, w1, acc[0][1]);
        acc[0][2] = fmaf(av.z, w1, acc[0][2]); acc[0][3] = fmaf(av.w, w1, acc[0][3]);
        if constexpr (NRHS >= 2) {
          const float w2 = __ldg(v2 + i + u);
          acc[1][0] = fmaf(av.x, w2, acc[1][0]); acc[1][1] = fmaf(av.y, w2, acc[1][1]);
          acc[1][2] = fmaf(av.z, w2, acc[1][2]); acc[1][3] = fmaf(av.w, w2, acc[1][3]);
        }
        if constexpr (NRHS == 3) {
          const float w3 = __ldg(v3 + i + u);
          acc[2][0] = fmaf(av.x, w3, acc[2][0]); acc[2][1] = fmaf(av.y, w3, acc[2][1]);
          acc[2][2] = fmaf(av.z, w3, acc[2][2]); acc[2][3] = fmaf(av.w, w3, acc[2][3]);
        }
      }
    }
    for (; i < r1; ++i) {
      float4 av = ldg_stream(reinterpret_cast<const float4*>(Ap + (int64_t)i * lda), i < keep_rows ? pk : ps);
      if (SQ) { av.x *= av.x; av.y *= av.y; av.z *= av.z; av.w *= av.w; }
      const float w1 = __ldg(v1 + i);
      acc[0][0] = fmaf(av.x, w1, acc[0][0]); acc[0][1] = fmaf(av.y, w1, acc[0][1]);
      acc[0][2] = fmaf(av.z, w1, acc[0][2]); acc[0][3] = fmaf(av.w, w1, acc[0][3]);
      if constexpr (NRHS >= 2) {
        const float w2 = __ldg(v2 + i);
        acc[1][0] = fmaf(av.x, w2, acc[1][0]); acc[1][1] = fmaf(av.y, w2, acc[1][1]);
        acc[1][2] = fmaf(av.z, w2, acc[1][2]); acc[1][3] = fmaf(av.w, w2, acc[1][3]);
      }
      if constexpr (NRHS == 3) {
        const float w3 = __ldg(v3 + i);
        acc[2][0] = fmaf(av.x, w3, acc[2][0]); acc[2][1] = fmaf(av.y, w3, acc[2][1]);
        acc[2][2] = fmaf(av.z, w3, acc[2][2]); acc[2][3] = fmaf(av.w, w3, acc[2][3]);
      }
    }
#pragma unroll
    for (int r = 0; r < NRHS; ++r)
      *reinterpret_cast<float4*>(part + ((int64_t)blockIdx.y * NRHS + r) * lda + c0) =
          make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
  }
  if (!FIN) return;
  if (!arrive_last(cnt + blockIdx.x, gridDim.y)) return;
  Df res[2] = {};
  if (active) {
    float s[NRHS][4];
#pragma unroll
    for (int r = 0; r < NRHS; ++r) s[r][0] = s[r][1] = s[r][2] = s[r][3] = 0.0f;
    // SPU splits' partials are loaded before they are added (in split order), so that the slab's
    // final reduction waits for one L2 round trip per SPU splits, not per split
    constexpr int SPU = NRHS == 3 ? 2 : 3;
    const int nsp = (int)gridDim.y;
    const float4* pp = reinterpret_cast<const float4*>(part + c0);
    const int64_t rs = lda >> 2, ss = NRHS * rs;   // float4 strides: right-hand side, split
    int sp = 0;
    for (; sp + SPU <= nsp; sp += SPU) {
      float4 p[SPU][NRHS];
#pragma unroll
      for (int u = 0; u < SPU; ++u)
#pragma unroll
        for (int r = 0; r < NRHS; ++r) p[u][r] = __ldcg(pp + (sp + u) * ss + r * rs);
#pragma unroll
      for (int u = 0; u < SPU; ++u)
#pragma unroll
        for (int r = 0; r < NRHS; ++r) {
          s[r][0] += p[u][r].x; s[r][1] += p[u][r].y; s[r][2] += p[u][r].z; s[r][3] += p[u][r].w;
        }
    }
    for (; sp < nsp; ++sp) {
#pragma unroll
      for (int r = 0; r < NRHS; ++r) {
        const float4 q = __ldcg(pp + sp * ss + r * rs);
        s[r][0] += q.x; s[r][1] += q.y; s[r][2] += q.z; s[r][3] += q.w;
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t j = c0 + u;
      if (j < n) epi_t<EPI>(ep, (int)j, s[0][u], NRHS >= 2 ? s[1][u] : 0.0f, NRHS == 3 ? s[NRHS - 1][u] : 0.0f, res);
    }
  }
  double tot[2];
  block_sum_df<2>(res, tot, sh);
  if (threadIdx.x == 0 && ep.res_part) {
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const float hi = (float)tot[t];
      ep.res_part[2 * blockIdx.x + t] = Df{hi, (float)(tot[t] - (double)hi)};
    }
  }
}

// Final reduction and epilogue of the column sums after a streaming launch
// (pogs_colsum_kernel<..., false>): one block per 1024-column slab, NRHS x 256 threads.  Thread
// (r, c) adds the nsp row splits' partials of right-hand side r for the four columns
// c0 = 1024 bx + 4 c .. + 3 in split order, eight loads in flight, into shared memory; then
// every thread applies the epilogue to the slab's columns bx * 1024 + tid, + blockDim, ...
// (consecutive threads on consecutive columns), and the block's residual partials go to
// res_part[bx] as in the streaming kernel's own final reduction.
template <int NRHS, int EPI>
__global__ void __launch_bounds__(768, 1) pogs_colsum_finish_kernel(const float* __restrict__ part, int64_t lda,
                                                                    int n, int nsp, EpiArgs ep,
                                                                    const DevState* __restrict__ guard) {
  __shared__ float4 sums[NRHS][256];
  __shared__ double sh[2 * 24];
  if (guard && guard->done) return;
  if (ep.cg_done && *ep.cg_done) return;
  const int tid = threadIdx.x, r = tid >> 8, c = tid & 255;
  const int64_t cb = (int64_t)blockIdx.x * 1024;
  const int64_t c0 = cb + 4 * c;
  if (c0 < lda) {
    const int64_t rs = lda >> 2, ss = NRHS * rs;
    const float4* pp = reinterpret_cast<const float4*>(part + c0) + r * rs;
    float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
    int sp = 0;
    for (; sp + 8 <= nsp; sp += 8) {
      float4 q[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) q[u] = __ldcg(pp + (sp + u) * ss);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        t.x += q[u].x; t.y += q[u].y; t.z += q[u].z; t.w += q[u].w;
      }
    }
    for (; sp < nsp; ++sp) {
      const float4 q = __ldcg(pp + sp * ss);
      t.x += q.x; t.y += q.y; t.z += q.z; t.w += q.w;
    }
    sums[r][c] = t;
  }
  __syncthreads();
  Df res[2] = {};
  const float* s0 = reinterpret_cast<const float*>(sums[0]);
  const float* s1 = reinterpret_cast<const float*>(sums[NRHS >= 2 ? 1 : 0]);
  const float* s2 = reinterpret_cast<const float*>(sums[NRHS - 1]);
  for (int l = tid; l < 1024; l += blockDim.x) {
    const int64_t j = cb + l;
    if (j < n) epi_t<EPI>(ep, (int)j, s0[l], NRHS >= 2 ? s1[l] : 0.0f, NRHS == 3 ? s2[l] : 0.0f, res);
  }
  double tot[2];
  block_sum_df<2>(res, tot, sh);
  if (threadIdx.x == 0 && ep.res_part) {
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const float hi = (float)tot[t];
      ep.res_part[2 * blockIdx.x + t] = Df{hi, (float)(tot[t] - (double)hi)};
    }
  }
}

// ------------------------------------------------------------------------------------------
// Row dots u = A [x1, x2].  Block (bx, by) covers rows [bx*RB, bx*RB+RB) and the column
// chunk by (CB floats, staged from x1/x2 in shared memory); one warp per row, float4 lanes,
// shuffle reduction; partials part[by][rhs][row]; the last chunk-block of a row block
// reduces in a fixed order and applies the epilogue.
// ------------------------------------------------------------------------------------------
// U: float4 loads in flight per lane.  8 when a block holds at least 32 rows (long-running
// blocks, where per-warp memory parallelism matters more than resident blocks), else 4.
template <int NRHS, bool SQ, int EPI, int U>
__global__ void __launch_bounds__(256) pogs_rowdot_kernel(const float* __restrict__ A, int64_t lda, int m, int n,
                                                     const float* __restrict__ x1,
                                                     const float* __restrict__ x2, int rows, int cols,
                                                     int keep_rows, float* __restrict__ part,
                                                     unsigned* __restrict__ cnt,
                                                     EpiArgs ep, const DevState* __restrict__ guard) {
  extern __shared__ float4 sx[];
  __shared__ double sh[2 * 8];
  if (guard && guard->done) return;
  if (ep.cg_done && *ep.cg_done) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t cbeg = (int64_t)blockIdx.y * cols;
  const int64_t cend = min((int64_t)lda, cbeg + cols);
  const int nq = (int)((cend - cbeg) >> 2);      // valid float4 in this chunk (lda % 4 == 0)
  const int nqs = cols >> 2;                     // shared-memory stride per rhs
  for (int qq = tid; qq < nq; qq += blockDim.x) {
    sx[qq] = __ldg(reinterpret_cast<const float4*>(x1 + cbeg) + qq);
    if constexpr (NRHS == 2) sx[nqs + qq] = __ldg(reinterpret_cast<const float4*>(x2 + cbeg) + qq);
  }
  __syncthreads();
  const int r0 = blockIdx.x * rows;
  const int r1 = min(m, r0 + rows);
  const uint64_t ps = l2_evict_first(), pk = l2_evict_last();
  for (int row = r0 + warp; row < r1; row += 8) {
    const float4* Ar = reinterpret_cast<const float4*>(A + (int64_t)row * lda + cbeg);
    const uint64_t pol = row < keep_rows ? pk : ps;
    float s1 = 0.0f, s2 = 0.0f;
    int qq = lane;
    for (; qq + 32 * (U - 1) < nq; qq += 32 * U) {
      float4 a[U];
#pragma unroll
      for (int u = 0; u < U; ++u) a[u] = ldg_stream(Ar + qq + 32 * u, pol);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        float4 av = a[u];
        if (SQ) { av.x *= av.x; av.y *= av.y; av.z *= av.z; av.w *= av.w; }
        const float4 xv = sx[qq + 32 * u];
        s1 = fmaf(av.x, xv.x, fmaf(av.y, xv.y, fmaf(av.z, xv.z, fmaf(av.w, xv.w, s1))));
        if constexpr (NRHS == 2) {
          const float4 xw = sx[nqs + qq + 32 * u];
          s2 = fmaf(av.x, xw.x, fmaf(av.y, xw.y, fmaf(av.z, xw.z, fmaf(av.w, xw.w, s2))));
        }
      }
    }
    for (; qq < nq; qq += 32) {
      float4 av = ldg_stream(Ar + qq, pol);
      if (SQ) { av.x *= av.x; av.y *= av.y; av.z *= av.z; av.w *= av.w; }
      const float4 xv = sx[qq];
      s1 = fmaf(av.x, xv.x, fmaf(av.y, xv.y, fmaf(av.z, xv.z, fmaf(av.w, xv.w, s1))));
      if constexpr (NRHS == 2) {
        const float4 xw = sx[nqs + qq];
        s2 = fmaf(av.x, xw.x, fmaf(av.y, xw.y, fmaf(av.z, xw.z, fmaf(av.w, xw.w, s2))));
      }
    }
    s1 = warp_sum(s1);
    if constexpr (NRHS == 2) s2 = warp_sum(s2);
    if (lane == 0) {
      part[((int64_t)blockIdx.y * NRHS) * m + row] = s1;
      if constexpr (NRHS == 2) part[((int64_t)blockIdx.y * NRHS + 1) * m + row] = s2;
    }
  }
  if (!arrive_last(cnt + blockIdx.x, gridDim.y)) return;
  Df res[2] = {};
  for (int row = r0 + tid; row < r1; row += blockDim.x) {
    float u1 = 0.0f, u2 = 0.0f;
    // four chunks' partials per round trip, added in chunk order
    const int nsp = (int)gridDim.y;
    for (int sp0 = 0; sp0 < nsp; sp0 += 4) {
      float p1[4], p2[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const bool ok = sp0 + u < nsp;
        p1[u] = ok ? __ldcg(part + ((int64_t)(sp0 + u) * NRHS) * m + row) : 0.0f;
        if constexpr (NRHS == 2) p2[u] = ok ? __ldcg(part + ((int64_t)(sp0 + u) * NRHS + 1) * m + row) : 0.0f;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (sp0 + u < nsp) {
          u1 += p1[u];
          if constexpr (NRHS == 2) u2 += p2[u];
        }
      }
    }
    epi_n<EPI>(ep, row, u1, u2, res);
  }
  double tot[2];
  block_sum_df<2>(res, tot, sh);
  if (threadIdx.x == 0 && ep.res_part) {
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const float hi = (float)tot[t];
      ep.res_part[2 * blockIdx.x + t] = Df{hi, (float)(tot[t] - (double)hi)};
    }
  }
}

// ------------------------------------------------------------------------------------------
// Triangular products with the cached inverse factor M = L^{-1}, stored as 128 x 128 tiles
// of the lower triangle (tile (I,J), J <= I, at linear index I(I+1)/2 + J, row-major inside;
// padding rows/cols are zero).  One block per tile; partial tile products are reduced by
// the last block of each tile row (z = M v) or tile column (x = M^T v).
// ------------------------------------------------------------------------------------------
// Sum of k partials p[0], p[stride], ... in index order, sixteen loads in flight per round trip.
__device__ __forceinline__ float sum_slots(const float* __restrict__ p, int k, int64_t stride) {
  float s = 0.0f;
  int i = 0;
  for (; i + 16 <= k; i += 16) {
    float v[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) v[u] = __ldcg(p + (int64_t)(i + u) * stride);
#pragma unroll
    for (int u = 0; u < 16; ++u) s += v[u];
  }
  for (; i < k; ++i) s += __ldcg(p + (int64_t)i * stride);
  return s;
}

__device__ __forceinline__ void tile_coords(int b, int& I, int& J) {
  int i = (int)((sqrtf(8.0f * (float)b + 1.0f) - 1.0f) * 0.5f);
  while ((i + 1) * (i + 2) / 2 <= b) ++i;
  while (i * (i + 1) / 2 > b) --i;
  I = i;
  J = b - i * (i + 1) / 2;
}

// Tile (I, J) of the lower triangle in column order: column J holds the T - J tiles (J..T-1, J)
// and starts at index J T - J (J - 1) / 2.
__device__ __forceinline__ void tile_coords_col(int c, int T, int& I, int& J) {
  const float tf = (float)T + 0.5f;
  int j = (int)(tf - sqrtf(fmaxf(tf * tf - 2.0f * (float)c, 0.0f)));
  if (j < 0) j = 0;
  while (j > 0 && (int64_t)j * T - (int64_t)j * (j - 1) / 2 > c) --j;
  while ((int64_t)(j + 1) * T - (int64_t)(j + 1) * j / 2 <= c) ++j;
  J = j;
  I = j + (int)(c - ((int64_t)j * T - (int64_t)j * (j - 1) / 2));
}

template <bool TRANS, int EPI>
__global__ void __launch_bounds__(256) trmv_kernel(const float* __restrict__ Mt, int T, int q,
                                                   const float* __restrict__ vin, float* __restrict__ part,
                                                   unsigned* __restrict__ cnt, EpiArgs ep,
                                                   const DevState* __restrict__ guard) {
  __shared__ float4 shc[8][32];
  if (guard && guard->done) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int b = blockIdx.x;
  int I, J;
  tile_coords(b, I, J);
  const float4* tile = reinterpret_cast<const float4*>(Mt + (int64_t)b * kTile * kTile);
  if (!TRANS) {
    const float4 rv = __ldg(reinterpret_cast<const float4*>(vin + (int64_t)J * kTile) + lane);
    float4 a[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) a[u] = ldg_stream(tile + (warp * 16 + u) * 32 + lane);
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      float s = a[u].x * rv.x + a[u].y * rv.y + a[u].z * rv.z + a[u].w * rv.w;
      s = warp_sum(s);
      if (lane == 0) part[(int64_t)b * kTile + warp * 16 + u] = s;
    }
    if (!arrive_last(cnt + I, I + 1)) return;
    if (tid < kTile) {
      const int64_t base = (int64_t)I * (I + 1) / 2;
      epi_r<EPI>(ep, I * kTile + tid, q, sum_slots(part + base * kTile + tid, I + 1, kTile));
    }
  } else {
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 a[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) a[u] = ldg_stream(tile + (warp * 16 + u) * 32 + lane);
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const float zr = __ldg(vin + (int64_t)I * kTile + warp * 16 + u);
      acc.x = fmaf(a[u].x, zr, acc.x); acc.y = fmaf(a[u].y, zr, acc.y);
      acc.z = fmaf(a[u].z, zr, acc.z); acc.w = fmaf(a[u].w, zr, acc.w);
    }
    shc[warp][lane] = acc;
    __syncthreads();
    const int64_t slot = (int64_t)J * T - (int64_t)J * (J - 1) / 2 + (I - J);
    if (tid < kTile) {
      const float* shf = reinterpret_cast<const float*>(&shc[0][0]);
      float s = 0.0f;
#pragma unroll
      for (int w = 0; w < 8; ++w) s += shf[w * kTile + tid];
      part[slot * kTile + tid] = s;
    }
    if (!arrive_last(cnt + J, T - J)) return;
    if (tid < kTile) {
      const int64_t base = (int64_t)J * T - (int64_t)J * (J - 1) / 2;
      epi_r<EPI>(ep, J * kTile + tid, q, sum_slots(part + base * kTile + tid, T - J, kTile));
    }
  }
}

// Symmetric product y = S v with S = M^T M = (I + G)^{-1} stored as its lower 128 x 128 tiles
// (diagonal tiles full).  One block per tile (I, J): its rows give block I the contribution
// S_IJ v_J (slot J of block I), and for I > J its columns give block J the contribution
// S_IJ^T v_I (slot I of block J), both from one read of the tile.  Every output block receives
// T contributions; the last block to deliver one sums the T slots in slot order and applies the
// epilogue.  One pass over the packed triangle instead of the two of M v and M^T z.  Blocks
// take the tiles in column order, so that output block J is complete once tile column J has
// been read and its final sum overlaps the rest of the pass (in row order every block waits for
// the last tile row).  LD16: all sixteen rows of a warp in flight at once (one round trip; for
// grids of at most two blocks per SM), else two batches of eight (fewer registers, more
// resident blocks).
template <int EPI, bool LD16>
__global__ void __launch_bounds__(256) symv_kernel(const float* __restrict__ St, int T, int q,
                                                   const float* __restrict__ vin, float* __restrict__ part,
                                                   unsigned* __restrict__ cnt, EpiArgs ep,
                                                   const DevState* __restrict__ guard) {
  __shared__ float4 shc[8][32];
  if (guard && guard->done) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int I, J;
  tile_coords_col(blockIdx.x, T, I, J);
  const int64_t b = (int64_t)I * (I + 1) / 2 + J;
  const float4* tile = reinterpret_cast<const float4*>(St + b * kTile * kTile);
  const float4 vj = __ldg(reinterpret_cast<const float4*>(vin + (int64_t)J * kTile) + lane);
  const bool off = I != J;
  // v_I entries of this warp's rows, loaded with the tile (not one dependent load per row)
  float zh[16];
#pragma unroll
  for (int u = 0; u < 16; ++u) zh[u] = __ldg(vin + (int64_t)I * kTile + warp * 16 + u);
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  // rows -> block I, slot J; columns (off-diagonal tiles) -> block J, slot I
  constexpr int NB = LD16 ? 1 : 2, NU = 16 / NB;
#pragma unroll
  for (int h = 0; h < NB; ++h) {
    float4 a[NU];
#pragma unroll
    for (int u = 0; u < NU; ++u) a[u] = ldg_stream(tile + (warp * 16 + h * NU + u) * 32 + lane);
#pragma unroll
    for (int u = 0; u < NU; ++u) {
      const int r = warp * 16 + h * NU + u;
      float s = a[u].x * vj.x + a[u].y * vj.y + a[u].z * vj.z + a[u].w * vj.w;
      s = warp_sum(s);
      if (lane == 0) part[((int64_t)I * T + J) * kTile + r] = s;
      if (off) {
        const float zr = zh[h * NU + u];
        acc.x = fmaf(a[u].x, zr, acc.x); acc.y = fmaf(a[u].y, zr, acc.y);
        acc.z = fmaf(a[u].z, zr, acc.z); acc.w = fmaf(a[u].w, zr, acc.w);
      }
    }
  }
  if (off) {
    shc[warp][lane] = acc;
    __syncthreads();
    if (tid < kTile) {
      const float* shf = reinterpret_cast<const float*>(&shc[0][0]);
      float s = 0.0f;
#pragma unroll
      for (int w = 0; w < 8; ++w) s += shf[w * kTile + tid];
      part[((int64_t)J * T + I) * kTile + tid] = s;
    }
  }
  auto finish = [&](int blk) {
    if (tid < kTile) epi_r<EPI>(ep, blk * kTile + tid, q, sum_slots(part + (int64_t)blk * T * kTile + tid, T, kTile));
  };
  if (arrive_last(cnt + I, T)) finish(I);
  if (I != J && arrive_last(cnt + J, T)) finish(J);
}

// ------------------------------------------------------------------------------------------
// Stopping test (Section 3.4 + half-tuple gap) and Algorithm 3, single block.
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) check_kernel(DevState* st, const DevCfg* __restrict__ cfg,
                                                    const Df* __restrict__ prox_part, int nprox,
                                                    const Df* __restrict__ pri_part, int npri,
                                                    const Df* __restrict__ dual_part, int ndual,
                                                    cudaGraphConditionalHandle h, int use_cond) {
  __shared__ double sh[10 * 8];
  if (st->done) {
    if (use_cond && threadIdx.x == 0) cudaGraphSetConditional(h, 0u);
    return;
  }
  Df a[10] = {};
  for (int i = threadIdx.x; i < nprox; i += blockDim.x) {
#pragma unroll
    for (int t = 0; t < 6; ++t) df_add(a[t], prox_part[6 * i + t]);
  }
  for (int i = threadIdx.x; i < npri; i += blockDim.x) {
    df_add(a[6], pri_part[2 * i]);
    df_add(a[7], pri_part[2 * i + 1]);
  }
  for (int i = threadIdx.x; i < ndual; i += blockDim.x) {
    df_add(a[8], dual_part[2 * i]);
    df_add(a[9], dual_part[2 * i + 1]);
  }
  double v[10];
  block_sum_df<10>(a, v, sh);
  if (threadIdx.x != 0) return;
  const double mu2 = v[0], xmu = v[1], gobj = v[2], yh2 = v[3], ynu = v[4], fobj = v[5];
  // square roots of the FP64 sums in FP32 (the FP64 square root is a long sequence on the
  // FP64 pipe; seven significant digits are far more than the tolerance test needs)
  auto rt = [](double a) { return (double)sqrtf((float)a); };
  const double r_pri = rt(v[6]), r_pri_u = rt(v[7]), r_dual = rt(v[8]), r_dual_u = rt(v[9]);
  const double eps_pri = cfg->abs_tol + cfg->rel_tol * rt(yh2);
  const double eps_dual = cfg->abs_tol + cfg->rel_tol * rt(mu2);
  const double gap = ynu + xmu;
  const double obj = fobj + gobj;
  const double eps_gap = cfg->abs_tol + cfg->rel_tol * fabs(obj);
  st->r_pri = r_pri; st->r_dual = r_dual; st->eps_pri = eps_pri; st->eps_dual = eps_dual;
  st->gap = gap; st->obj = obj; st->r_pri_u = r_pri_u; st->r_dual_u = r_dual_u;
  const int k = st->k;
  st->k = k + 1;
  int done = 0;
  if (st->err != 0) {
    st->status = st->err;
    done = 1;
  } else if (!isfinite(r_pri) || !isfinite(r_dual) || !isfinite(gap) || !isfinite(obj)) {
    st->status = POGS_ERR_NONFINITE;
    done = 1;
  } else if (r_pri < eps_pri && r_dual < eps_dual && (!cfg->gap_stop || fabs(gap) < eps_gap)) {
    st->status = POGS_OK;
    done = 1;
  } else if (k + 1 >= cfg->max_iter) {
    st->status = POGS_MAX_ITER;
    done = 1;
  }
  double pend = 1.0;
  if (!done && cfg->adaptive) {
    const double rho = st->rho;
    double rho_new = rho;
    if (r_dual < eps_dual && cfg->tau * k > st->l) {
      rho_new = cfg->delta * rho;
      pend = cfg->inv_delta;        // rho^k / rho^{k+1}
      st->u = k;
    } else if (r_pri < eps_pri && cfg->tau * k > st->u) {
      rho_new = rho * cfg->inv_delta;
      pend = cfg->delta;
      st->l = k;
    }
    st->rho = rho_new;
  }
  st->pend = pend;
  st->done = done;
  if (use_cond) cudaGraphSetConditional(h, done ? 0u : 1u);
}

// ------------------------------------------------------------------------------------------
// Small elementwise kernels.
// ------------------------------------------------------------------------------------------
__global__ void prox_eval_kernel(FnDev fn, int64_t k, const float* v, const float* rv, float rho, float* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x) {
    const float r = rv ? rv[i] : rho;
    out[i] = prox_param(fn.h[i], fn.a[i], fn.b[i], fn.c[i], fn.d[i], fn.e[i], r, v[i]);
  }
}

// Pre-conditioned parameters (Eq. 12): f^(y^) = f(y^/D): a/D, d/D, e/D^2 (is_f);
// g^(x^) = g(E x^): a E, d E, e E^2.  Validates a != 0, c >= 0, e >= 0, h in range.
__global__ void fold_kernel(FnDev raw, int64_t k, const float* scale, int is_f, uint8_t* h, float* a,
                            float* b, float* c, float* d, float* e, int* err) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x) {
    const int hv = raw.h[i];
    const float av = raw.a ? raw.a[i] : 1.0f, bv = raw.b ? raw.b[i] : 0.0f;
    const float cv = raw.c ? raw.c[i] : 1.0f, dv = raw.d ? raw.d[i] : 0.0f, ev = raw.e ? raw.e[i] : 0.0f;
    if (hv < 0 || hv > POGS_XLOGX || !(av != 0.0f) || !(cv >= 0.0f) || !(ev >= 0.0f) ||
        !isfinite(av) || !isfinite(bv) || !isfinite(cv) || !isfinite(dv) || !isfinite(ev))
      atomicCAS(err, 0, POGS_ERR_ARG);   // first error wins
    const float s = scale[i];
    const float m1 = is_f ? 1.0f / s : s;
    h[i] = (uint8_t)hv;
    a[i] = av * m1;
    b[i] = bv;
    c[i] = cv;
    d[i] = dv * m1;
    e[i] = ev * m1 * m1;
  }
}

__global__ void fill_kernel(float* p, int64_t k, float v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x) p[i] = v;
}

// Returned tuple (Section 5) in the original variables: x = E x^, mu = mu^/E, y = y^/D, nu = D nu^.
__global__ void unscale_kernel(int n, int m, const float* xh, const float* mu, const float* yh,
                               const float* nu, const float* D, const float* E, float* x, float* muo,
                               float* y, float* nuo) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n + m; i += gridDim.x * blockDim.x) {
    if (i < n) {
      if (x) x[i] = E[i] * xh[i];
      if (muo) muo[i] = mu[i] / E[i];
    } else {
      const int k = i - n;
      if (y) y[k] = yh[k] / D[k];
      if (nuo) nuo[k] = D[k] * nu[k];
    }
  }
}

__global__ void axpby_kernel(int64_t k, float a, const float* x, float b, const float* y, float* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = a * x[i] + b * y[i];
}

static int grid_for(int64_t k, int per = 256) {
  int64_t g = (k + per - 1) / per;
  if (g < 1) g = 1;
  if (g > 148 * 8) g = 148 * 8;
  return (int)g;
}

void launch_prox_eval(FnDev fn, int64_t k, const float* v, const float* rv, float rho, float* out, cudaStream_t s) {
  count_launch();
  prox_eval_kernel<<<grid_for(k), 256, 0, s>>>(fn, k, v, rv, rho, out);
}
void launch_fold(FnDev raw, int64_t k, const float* scale, int is_f, uint8_t* h, float* a, float* b, float* c,
                 float* d, float* e, int* err, cudaStream_t s) {
  count_launch();
  fold_kernel<<<grid_for(k), 256, 0, s>>>(raw, k, scale, is_f, h, a, b, c, d, e, err);
}
// Warm start (Section 5) into the pre-conditioned variables: v = src / scale * factor;
// out_pos = v, out_neg = -v (when given).  x^0: x^ = x0 / E.  nu^0: w = nu0 / D / rho and
// y~ = -w (x~ = A^T w follows with a column-sum pass).
__global__ void warm_kernel(const float* __restrict__ src, const float* __restrict__ scale, int64_t k, float factor,
                            float* __restrict__ out_pos, float* __restrict__ out_neg) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x) {
    const float v = src[i] / scale[i] * factor;
    out_pos[i] = v;
    if (out_neg) out_neg[i] = -v;
  }
}
void launch_warm(const float* src, const float* scale, int64_t k, float factor, float* out_pos, float* out_neg,
                 cudaStream_t s) {
  count_launch();
  warm_kernel<<<grid_for(k), 256, 0, s>>>(src, scale, k, factor, out_pos, out_neg);
}

void launch_fill(float* p, int64_t k, float v, cudaStream_t s) {
  count_launch();
  fill_kernel<<<grid_for(k), 256, 0, s>>>(p, k, v);
}
void launch_unscale(int n, int m, const float* xh, const float* mu, const float* yh, const float* nu,
                    const float* D, const float* E, float* x, float* muo, float* y, float* nuo, cudaStream_t s) {
  count_launch();
  unscale_kernel<<<grid_for(n + m), 256, 0, s>>>(n, m, xh, mu, yh, nu, D, E, x, muo, y, nuo);
}
void launch_axpby(int64_t k, float a, const float* x, float b, const float* y, float* out, cudaStream_t s) {
  count_launch();
  axpby_kernel<<<grid_for(k), 256, 0, s>>>(k, a, x, b, y, out);
}

// ------------------------------------------------------------------------------------------
// Dispatch.
// ------------------------------------------------------------------------------------------
// A^ between 128 MB and 512 MB (one to four times L2) keeps its leading 48 MB in L2 across the
// passes; a larger one gains too little from it, a smaller one stays in L2 largely anyway.
constexpr size_t kL2KeepBytes = size_t(48) << 20;
constexpr size_t kL2KeepMin = size_t(128) << 20, kL2KeepMax = size_t(512) << 20;

// Returns the lines of `bytes` at p to normal L2 eviction priority (one 128-byte line per
// thread step): the end of the passes over a matrix whose leading rows were read evict-last.
__global__ void l2_release_kernel(const char* __restrict__ p, int64_t lines) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < lines; i += (int64_t)gridDim.x * blockDim.x)
    asm volatile("applypriority.global.L2::evict_normal [%0], 128;" ::"l"(p + 128 * i) : "memory");
}

void launch_l2_release(const float* A, size_t bytes, cudaStream_t s) {
  const int64_t lines = (int64_t)(bytes / 128);
  if (lines <= 0) return;
  count_launch();
  l2_release_kernel<<<(int)std::min<int64_t>(cdiv(lines, 256), 148 * 8), 256, 0, s>>>(
      reinterpret_cast<const char*>(A), lines);
}
GemvGeom choose_geometry(int64_t m, int64_t n, int64_t lda, int num_sms) {
  GemvGeom g{};
  // the leading rows of A^ up to kL2KeepBytes stay in L2 across passes (the rest streams through
  // under evict-first), so each pass reads that much less from HBM
  const size_t abytes = (size_t)m * lda * sizeof(float);
  g.keep_rows = abytes > kL2KeepMin && abytes <= kL2KeepMax
                    ? (int)std::min<int64_t>(m, (int64_t)(kL2KeepBytes / ((size_t)lda * sizeof(float))))
                    : 0;
  // column sums: 1024-column slabs, rows split so that the grid covers ~4 blocks per SM
  g.t_cols_per_blk = 1024;
  g.t_ncolblk = (int)cdiv(lda, 1024);
  int64_t target = (int64_t)num_sms * 5;   // 5 resident 256-thread blocks per SM at the kernel's register count
  int64_t nsplit = cdiv(target, g.t_ncolblk);
  // whole 8-row steps, and at least 64 rows per split: the slab's last block sums the splits
  // serially, which dominates the launch for small matrices split too finely
  int64_t rows = round_up(cdiv(m, nsplit), 8);
  if (rows < 64) rows = std::min<int64_t>(64, round_up(m, 8));
  g.t_rows = (int)rows;
  g.t_nsplit = (int)cdiv(m, rows);
  // row dots: column chunks of <= 4096 floats; rows per block chosen for ~5 blocks per SM
  // (measured on both large shapes against 2, 3, 4 and 8: fewer, longer-running blocks with
  // eight loads in flight per lane stream closest to the copy bandwidth)
  int64_t nchunk = cdiv(lda, 4096);
  int64_t cols = round_up(cdiv(lda, nchunk), 128);
  g.n_cols = (int)cols;
  g.n_ncolsplit = (int)cdiv(lda, cols);
  int64_t tgt = (int64_t)num_sms * 5;
  int64_t nrb = cdiv(tgt, g.n_ncolsplit);
  // a multiple of 8 rows per block, so that each of the 8 warps gets the same number of rows
  int64_t rb = round_up(cdiv(m, nrb), 8);
  rb = rb > 256 ? 256 : rb;
  g.n_rows = (int)rb;
  g.n_nrowblk = (int)cdiv(m, rb);
  return g;
}

template <int NRHS, bool SQ>
static void gemv_t_dispatch(int epi, const float* A, int64_t lda, int m, int n, const float* v1, const float* v2,
                            const float* v3, const GemvGeom& g, float* part, unsigned* cnt, const EpiArgs& ep,
                            const DevState* guard, cudaStream_t s) {
  dim3 grid(g.t_ncolblk, g.t_nsplit);
  const bool split = colsum_split(g, epi);
  count_launch(split ? 2 : 1);
#define POGS_T(E) pogs_colsum_kernel<NRHS, SQ, E><<<grid, 256, 0, s>>>(A, lda, m, n, v1, v2, v3, g.t_rows, g.keep_rows, part, cnt, ep, guard)
#define POGS_TS(E)                                                                                              \
  do {                                                                                                          \
    if (split) {                                                                                                \
      pogs_colsum_kernel<NRHS, SQ, E, false><<<grid, 256, 0, s>>>(A, lda, m, n, v1, v2, v3, g.t_rows, g.keep_rows, \
                                                                  part, cnt, ep, guard);                        \
      pogs_colsum_finish_kernel<NRHS, E><<<g.t_ncolblk, 256 * NRHS, 0, s>>>(part, lda, n, g.t_nsplit, ep, guard); \
    } else {                                                                                                    \
      POGS_T(E);                                                                                                \
    }                                                                                                           \
  } while (0)
  switch (epi) {
    case EPT_RAW: POGS_TS(EPT_RAW); break;
    case EPT_TALL_R: POGS_TS(EPT_TALL_R); break;
    case EPT_FAT_X: POGS_TS(EPT_FAT_X); break;
    case EPT_SK_COL: POGS_TS(EPT_SK_COL); break;
    case EPT_REFINE: POGS_TS(EPT_REFINE); break;
    case EPT_CG_R: POGS_T(EPT_CG_R); break;
    case EPT_CG_S0: POGS_T(EPT_CG_S0); break;
    case EPT_CG_Q: POGS_T(EPT_CG_Q); break;
    case EPT_CG_S: POGS_T(EPT_CG_S); break;
  }
#undef POGS_T
#undef POGS_TS
}

bool colsum_split(const GemvGeom& g, int epi) {
  return !g.sparse && g.t_nsplit >= 4 &&
         (epi == EPT_RAW || epi == EPT_TALL_R || epi == EPT_FAT_X || epi == EPT_SK_COL || epi == EPT_REFINE);
}

void launch_gemv_t(int nrhs, bool sq, int epi, const float* A, int64_t lda, int m, int n, const float* v1,
                   const float* v2, const float* v3, const GemvGeom& g, float* part, unsigned* cnt,
                   const EpiArgs& ep, const DevState* guard, cudaStream_t s) {
  if (g.sparse) {
    launch_spmv(true, nrhs, sq, epi, g, m, n, v1, v2, v3, ep, guard, s);
    return;
  }
  if (nrhs == 3) gemv_t_dispatch<3, false>(epi, A, lda, m, n, v1, v2, v3, g, part, cnt, ep, guard, s);
  else if (nrhs == 2) gemv_t_dispatch<2, false>(epi, A, lda, m, n, v1, v2, v3, g, part, cnt, ep, guard, s);
  else if (sq) gemv_t_dispatch<1, true>(epi, A, lda, m, n, v1, v2, v3, g, part, cnt, ep, guard, s);
  else gemv_t_dispatch<1, false>(epi, A, lda, m, n, v1, v2, v3, g, part, cnt, ep, guard, s);
}

template <int NRHS, bool SQ>
static void gemv_n_dispatch(int epi, const float* A, int64_t lda, int m, int n, const float* x1, const float* x2,
                            const GemvGeom& g, float* part, unsigned* cnt, const EpiArgs& ep,
                            const DevState* guard, cudaStream_t s) {
  dim3 grid(g.n_nrowblk, g.n_ncolsplit);
  count_launch();
  const size_t smem = (size_t)NRHS * g.n_cols * sizeof(float);
  // smem <= 2 x 4096 floats = 32 KB: no opt-in needed (and nothing to set during capture)
#define POGS_N(E)                                                                                         \
  do {                                                                                                    \
    if (g.n_rows >= 32)                                                                                   \
      pogs_rowdot_kernel<NRHS, SQ, E, 8><<<grid, 256, smem, s>>>(A, lda, m, n, x1, x2, g.n_rows, g.n_cols,        \
                                                            g.keep_rows, part, cnt, ep, guard);            \
    else                                                                                                  \
      pogs_rowdot_kernel<NRHS, SQ, E, 4><<<grid, 256, smem, s>>>(A, lda, m, n, x1, x2, g.n_rows, g.n_cols,        \
                                                            g.keep_rows, part, cnt, ep, guard);            \
  } while (0)
  switch (epi) {
    case EPN_RAW: POGS_N(EPN_RAW); break;
    case EPN_TALL_Y: POGS_N(EPN_TALL_Y); break;
    case EPN_FAT_R: POGS_N(EPN_FAT_R); break;
    case EPN_SK_ROW: POGS_N(EPN_SK_ROW); break;
    case EPN_REFINE: POGS_N(EPN_REFINE); break;
    case EPN_CG_R: POGS_N(EPN_CG_R); break;
    case EPN_CG_S0: POGS_N(EPN_CG_S0); break;
    case EPN_CG_Q: POGS_N(EPN_CG_Q); break;
    case EPN_CG_S: POGS_N(EPN_CG_S); break;
  }
#undef POGS_N
}

void launch_gemv_n(int nrhs, bool sq, int epi, const float* A, int64_t lda, int m, int n, const float* x1,
                   const float* x2, const GemvGeom& g, float* part, unsigned* cnt, const EpiArgs& ep,
                   const DevState* guard, cudaStream_t s) {
  if (g.sparse) {
    launch_spmv(false, nrhs, sq, epi, g, m, n, x1, x2, nullptr, ep, guard, s);
    return;
  }
  if (nrhs == 2) gemv_n_dispatch<2, false>(epi, A, lda, m, n, x1, x2, g, part, cnt, ep, guard, s);
  else if (sq) gemv_n_dispatch<1, true>(epi, A, lda, m, n, x1, x2, g, part, cnt, ep, guard, s);
  else gemv_n_dispatch<1, false>(epi, A, lda, m, n, x1, x2, g, part, cnt, ep, guard, s);
}

void launch_symv(int epi, const float* St, int T, int q, const float* vin, float* part, unsigned* cnt,
                 const EpiArgs& ep, const DevState* guard, cudaStream_t s) {
  const int nt = T * (T + 1) / 2;
  count_launch();
  const bool ld16 = nt <= 2 * 148;
#define POGS_S(E)                                                                         \
  do {                                                                                    \
    if (ld16) symv_kernel<E, true><<<nt, 256, 0, s>>>(St, T, q, vin, part, cnt, ep, guard);  \
    else symv_kernel<E, false><<<nt, 256, 0, s>>>(St, T, q, vin, part, cnt, ep, guard);      \
  } while (0)
  switch (epi) {
    case EPR_RAW: POGS_S(EPR_RAW); break;
    case EPR_TALL_X: POGS_S(EPR_TALL_X); break;
    case EPR_FAT_Y: POGS_S(EPR_FAT_Y); break;
    case EPR_ADD: POGS_S(EPR_ADD); break;
  }
#undef POGS_S
}

void launch_trmv(bool trans, int epi, const float* Mt, int T, int q, const float* vin, float* part, unsigned* cnt,
                 const EpiArgs& ep, const DevState* guard, cudaStream_t s) {
  const int nt = T * (T + 1) / 2;
  count_launch();
#define POGS_R(TR, E) trmv_kernel<TR, E><<<nt, 256, 0, s>>>(Mt, T, q, vin, part, cnt, ep, guard)
  if (!trans) {
    switch (epi) {
      case EPR_RAW: POGS_R(false, EPR_RAW); break;
      case EPR_ADD: POGS_R(false, EPR_ADD); break;
    }
  } else {
    switch (epi) {
      case EPR_RAW: POGS_R(true, EPR_RAW); break;
      case EPR_TALL_X: POGS_R(true, EPR_TALL_X); break;
      case EPR_FAT_Y: POGS_R(true, EPR_FAT_Y); break;
      case EPR_ADD: POGS_R(true, EPR_ADD); break;
    }
  }
#undef POGS_R
}

void launch_check(DevState* st, const DevCfg* cfg, const Df* prox_part, int nprox, const Df* pri_part,
                  int npri, const Df* dual_part, int ndual, unsigned long long cond_handle, int use_cond,
                  cudaStream_t s) {
  count_launch();
  check_kernel<<<1, 256, 0, s>>>(st, cfg, prox_part, nprox, pri_part, npri, dual_part, ndual,
                                 (cudaGraphConditionalHandle)cond_handle, use_cond);
}

}  // namespace pogs
