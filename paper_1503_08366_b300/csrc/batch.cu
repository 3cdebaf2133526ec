// Batched graph-form ADMM: many independent small instances of uneven (m, n).
//
// Setup runs one CTA per instance (Algorithm 2 + Frobenius rescale, folding of D and E into
// the parameters, Gram + I in FP64, blocked Cholesky, FP32 inverse factor).  The iteration is
// a persistent kernel: each CTA takes the next instance from a device work queue and runs the
// whole ADMM loop for it (Algorithm 1 + over-relaxation + Section 3.4 stopping + Algorithm 3)
// with block-level synchronisation between the phases, then takes the next one.  An
// instance's matrix and factor stay resident in L2 (or in shared memory when small enough)
// across its iterations.
//
// Every instance is computed by one CTA of kBatchThreads threads with fixed loop and
// reduction orders, so its result does not depend on which other instances share the batch,
// on the grid size, on the schedule or on whether its matrix is staged in shared memory.
#include <cstdio>

#include "batch.h"
#include "prox.cuh"

namespace pogs {

namespace {

constexpr int NT = kBatchThreads;
constexpr int NW = NT / 32;

// Block-wide FP64 sums of NV values per thread, result in every thread (fixed order).
template <int NV>
__device__ __forceinline__ void bsum(double (&v)[NV], double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int t = 0; t < NV; ++t) v[t] = warp_sum(v[t]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int t = 0; t < NV; ++t) sh[t * NW + wid] = v[t];
  }
  __syncthreads();
#pragma unroll
  for (int t = 0; t < NV; ++t) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < NW; ++w) s += sh[t * NW + w];
    v[t] = s;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------------------------
// Setup 1: Sinkhorn-Knopp (Algorithm 2, p = 2), Frobenius rescale (Section 4.1.2), A^ = D A E,
// folded parameters (Eq. 12).
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) bsetup_equil_kernel(BInst* insts, BCfg cfg) {
  __shared__ double sh[4 * NW];
  __shared__ int s_err;
  BInst I = insts[blockIdx.x];
  const int m = I.m, n = I.n, lda = I.lda, q = I.q;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float* d = I.D;   // d, then D
  float* e = I.E;   // e, then E
  if (tid == 0) s_err = 0;
  for (int j = tid; j < n; j += NT) e[j] = 1.0f;
  for (int i = tid; i < m; i += NT) d[i] = 1.0f;
  // non-finite input check
  int bad = 0;
  for (int i = 0; i < m; ++i)
    for (int j = tid; j < n; j += NT)
      if (!isfinite(I.A[(int64_t)i * lda + j])) bad = 1;
  if (bad) atomicExch(&s_err, POGS_ERR_NONFINITE);
  __syncthreads();
  const double gamma = cfg.gamma_scale > 0 ? cfg.gamma_scale : (double)(m + n) * sqrt(1.1920928955078125e-07);
  const float rreg = (float)(gamma / m), creg = (float)(gamma / n);
  const int sweeps = cfg.equil ? cfg.sk_sweeps : 0;
  double fro[1] = {0.0};
  for (int s = 0; s < sweeps; ++s) {
    for (int i = warp; i < m; i += NW) {
      float acc = 0.0f;
      for (int j = lane; j < n; j += 32) {
        const float a = I.A[(int64_t)i * lda + j];
        acc = fmaf(a * a, e[j], acc);
      }
      acc = warp_sum(acc);
      if (lane == 0) d[i] = (float)n / (acc + rreg);
    }
    __syncthreads();
    fro[0] = 0.0;
    for (int j = tid; j < n; j += NT) {
      float acc = 0.0f;
      for (int i = 0; i < m; ++i) {
        const float a = I.A[(int64_t)i * lda + j];
        acc = fmaf(a * a, d[i], acc);
      }
      const float ej = (float)m / (acc + creg);
      e[j] = ej;
      fro[0] += (double)ej * (double)acc;
    }
    __syncthreads();
  }
  if (sweeps == 0) {
    fro[0] = 0.0;
    for (int j = tid; j < n; j += NT) {
      float acc = 0.0f;
      for (int i = 0; i < m; ++i) {
        const float a = I.A[(int64_t)i * lda + j];
        acc = fmaf(a, a, acc);
      }
      fro[0] += (double)acc;
    }
  }
  bsum<1>(fro, sh);
  const double sinv = 1.0 / sqrt(fro[0] / (double)q);
  for (int i = tid; i < m; i += NT) d[i] = (float)sqrt((double)d[i] * sinv);
  for (int j = tid; j < n; j += NT) e[j] = (float)sqrt((double)e[j] * sinv);
  __syncthreads();
  for (int i = 0; i < m; ++i)
    for (int j = tid; j < n; j += NT) I.A[(int64_t)i * lda + j] *= d[i] * e[j];
  // parameters of f^ (length m) and g^ (length n)
  for (int k = tid; k < m + n; k += NT) {
    const bool isf = k < m;
    const int i = isf ? k : k - m;
    const uint8_t* h0 = isf ? I.fh0 : I.gh0;
    const float *a0 = isf ? I.fa0 : I.ga0, *b0 = isf ? I.fb0 : I.gb0, *c0 = isf ? I.fc0 : I.gc0;
    const float *d0 = isf ? I.fd0 : I.gd0, *e0 = isf ? I.fe0 : I.ge0;
    const int hv = h0[i];
    const float av = a0 ? a0[i] : 1.0f, bv = b0 ? b0[i] : 0.0f, cv = c0 ? c0[i] : 1.0f;
    const float dv = d0 ? d0[i] : 0.0f, ev = e0 ? e0[i] : 0.0f;
    if (hv < 0 || hv > POGS_XLOGX || !(av != 0.0f) || !(cv >= 0.0f) || !(ev >= 0.0f) || !isfinite(av) ||
        !isfinite(bv) || !isfinite(cv) || !isfinite(dv) || !isfinite(ev))
      atomicCAS(&s_err, 0, POGS_ERR_ARG);
    const float sc = isf ? 1.0f / d[i] : e[i];
    if (isf) {
      I.fh[i] = (uint8_t)hv; I.fa[i] = av * sc; I.fb[i] = bv; I.fc[i] = cv; I.fd[i] = dv * sc; I.fe[i] = ev * sc * sc;
    } else {
      I.gh[i] = (uint8_t)hv; I.ga[i] = av * sc; I.gb[i] = bv; I.gc[i] = cv; I.gd[i] = dv * sc; I.ge[i] = ev * sc * sc;
    }
  }
  __syncthreads();
  if (tid == 0) I.out->status = s_err;
}

// ---------------------------------------------------------------------------------------------
// Setup 2: H = I + G in FP64 (lower), G = A^T A (tall) or A A^T (fat), FP32 products, 32 x 32
// tiles with 32-deep K chunks staged in shared memory.
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) bsetup_gram_kernel(BInst* insts) {
  __shared__ float Xs[32][33], Ys[32][33];
  BInst I = insts[blockIdx.x];
  if (I.out->status != 0) return;
  const int q = I.q, K = I.tall ? I.m : I.n, lda = I.lda;
  const int T = (q + 31) / 32;
  const int tid = threadIdx.x;
  const int r = tid >> 3, c4 = (tid & 7) * 4;
  for (int t = 0; t < T * (T + 1) / 2; ++t) {
    int ti = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
    while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
    while (ti * (ti + 1) / 2 > t) --ti;
    const int tj = t - ti * (ti + 1) / 2;
    const int r0 = ti * 32, s0 = tj * 32;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k0 = 0; k0 < K; k0 += 32) {
      for (int e = tid; e < 32 * 32; e += NT) {
        const int kk = e >> 5, rr = e & 31;
        float xv = 0.f, yv = 0.f;
        if (I.tall) {   // X = A^T: X[row][k] = A[k][row], read along rows of A
          if (k0 + kk < K && r0 + rr < q) xv = I.A[(int64_t)(k0 + kk) * lda + r0 + rr];
          if (k0 + kk < K && s0 + rr < q) yv = I.A[(int64_t)(k0 + kk) * lda + s0 + rr];
          Xs[kk][rr] = xv;
          Ys[kk][rr] = yv;
        } else {        // X = A: X[row][k] = A[row][k]
          const int kk2 = e & 31, rr2 = e >> 5;
          if (k0 + kk2 < K && r0 + rr2 < q) xv = I.A[(int64_t)(r0 + rr2) * lda + k0 + kk2];
          if (k0 + kk2 < K && s0 + rr2 < q) yv = I.A[(int64_t)(s0 + rr2) * lda + k0 + kk2];
          Xs[kk2][rr2] = xv;
          Ys[kk2][rr2] = yv;
        }
      }
      __syncthreads();
#pragma unroll 8
      for (int kk = 0; kk < 32; ++kk) {
        const float a = Xs[kk][r];
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] = fmaf(a, Ys[kk][c4 + u], acc[u]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int gi = r0 + r, gj = s0 + c4 + u;
      if (gi < q && gj < q && gj <= gi) I.H[(int64_t)gi * q + gj] = (double)acc[u] + (gi == gj ? 1.0 : 0.0);
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Setup 3: right-looking blocked Cholesky of H (32-column panels): FP64 diagonal blocks and
// panel solves; trailing update from the FP32-rounded panel in FP32 (mixed) or in FP64.
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) bsetup_chol_kernel(BInst* insts, int mixed) {
  extern __shared__ float Pf[];            // [q][33] FP32 panel
  __shared__ double Ld[32][33], Xi[32][33];
  __shared__ int s_err;
  BInst I = insts[blockIdx.x];
  if (I.out->status != 0) return;
  const int q = I.q;
  double* H = I.H;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_err = 0;
  for (int k0 = 0; k0 < q; k0 += 32) {
    const int nb = min(32, q - k0);
    for (int e = tid; e < 32 * 32; e += NT) {
      const int i = e >> 5, j = e & 31;
      Ld[i][j] = (i < nb && j <= i) ? H[(int64_t)(k0 + i) * q + k0 + j] : 0.0;
    }
    __syncthreads();
    if (warp == 0) {
      for (int j = 0; j < nb; ++j) {
        if (lane == 0) {
          double djj = Ld[j][j];
          if (!(djj > 0.0) || !isfinite(djj)) {
            atomicCAS(&s_err, 0, POGS_ERR_NUMERIC);
            djj = 1.0;
          }
          Ld[j][j] = sqrt(djj);
        }
        __syncwarp();
        const double ljj = Ld[j][j];
        for (int i = j + 1 + lane; i < nb; i += 32) Ld[i][j] /= ljj;
        __syncwarp();
        for (int i = j + 1 + lane; i < nb; i += 32)
          for (int k = j + 1; k <= i; ++k) Ld[i][k] -= Ld[i][j] * Ld[k][j];
        __syncwarp();
      }
      // inverse of the diagonal factor, one column per lane
      if (lane < nb) {
        const int c = lane;
        for (int i = 0; i < nb; ++i) {
          double v = 0.0;
          if (i >= c) {
            double acc = (i == c) ? 1.0 : 0.0;
            for (int k = c; k < i; ++k) acc -= Ld[i][k] * Xi[k][c];
            v = acc / Ld[i][i];
          }
          Xi[i][c] = v;
        }
      }
    }
    __syncthreads();
    for (int e = tid; e < nb * nb; e += NT) {
      const int i = e / nb, j = e % nb;
      if (j <= i) H[(int64_t)(k0 + i) * q + k0 + j] = Ld[i][j];
    }
    // panel: rows below the block, P = H_panel L_kk^{-T} (FP64); FP32 copy for the update
    const int R = q - k0 - nb;
    for (int ii = tid; ii < R; ii += NT) {
      double h[32];
      double* row = H + (int64_t)(k0 + nb + ii) * q + k0;
#pragma unroll
      for (int k = 0; k < 32; ++k) h[k] = k < nb ? row[k] : 0.0;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        if (j < nb) {
          double p = 0.0;
          for (int k = 0; k <= j; ++k) p += h[k] * Xi[j][k];
          row[j] = p;
          Pf[ii * 33 + j] = (float)p;
        }
      }
    }
    __syncthreads();
    // trailing update of the lower triangle
    for (int ii = 0; ii < R; ++ii) {
      double* hrow = H + (int64_t)(k0 + nb + ii) * q + k0 + nb;
      for (int jj = tid; jj <= ii; jj += NT) {
        if (mixed) {
          float acc = 0.0f;
          for (int k = 0; k < nb; ++k) acc = fmaf(Pf[ii * 33 + k], Pf[jj * 33 + k], acc);
          hrow[jj] -= (double)acc;
        } else {
          const double* pi = H + (int64_t)(k0 + nb + ii) * q + k0;
          const double* pj = H + (int64_t)(k0 + nb + jj) * q + k0;
          double acc = 0.0;
          for (int k = 0; k < nb; ++k) acc += pi[k] * pj[k];
          hrow[jj] -= acc;
        }
      }
    }
    __syncthreads();
  }
  if (tid == 0 && s_err != 0) I.out->status = s_err;
}

// ---------------------------------------------------------------------------------------------
// Setup 4: M = L^{-1} (FP32, dense lower with zeros above the diagonal, ld q) by block forward
// substitution on 32 x 32 blocks, one block row at a time: W_ii = L_ii^{-1} by FP64 substitution
// (warp 0, lane = column, rounded to FP32), then for every j < i at once
// M_ij = -W_ii sum_{k=j}^{i-1} L_ik M_kj, the sum in FP32 over the FP32-rounded L (the warps take
// the blocks j in turn, lane = column of the block, 32 row accumulators per lane).  FP64 work
// is q/32 diagonal blocks instead of the whole triangle (B300's FP64 rate is a small fraction of
// its FP32 rate); the products carry FP32 accuracy, as those of the single-problem inverse.
// ---------------------------------------------------------------------------------------------
constexpr int kInvRowMax = 480;   // columns of L left of the last block row (q <= 512)
constexpr int kInvSmem = kInvRowMax * 32 * (int)sizeof(float);

__global__ void __launch_bounds__(NT) bsetup_inverse_kernel(BInst* insts) {
  extern __shared__ __align__(16) float Lt[];   // block row i of L left of the diagonal, FP32, Lt[k * 32 + r]
  __shared__ double Ld[32][33];
  __shared__ float Wd[32][33];
  BInst I = insts[blockIdx.x];
  if (I.out->status != 0) return;
  const int q = I.q, T = (q + 31) / 32;
  const double* L = I.H;
  float* M = I.M;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int ib = 0; ib < T; ++ib) {
    const int r0 = ib * 32, nb = min(32, q - r0);
    for (int e = tid; e < 32 * 32; e += NT) {
      const int r = e >> 5, c = e & 31;
      Ld[r][c] = (r < nb && c < nb) ? L[(int64_t)(r0 + r) * q + r0 + c] : (r == c ? 1.0 : 0.0);
    }
    for (int e = tid; e < r0 * 32; e += NT) {
      const int r = e / r0, k = e - r * r0;   // consecutive threads along a row of L
      Lt[k * 32 + r] = r < nb ? (float)L[(int64_t)(r0 + r) * q + k] : 0.0f;
    }
    // zeros right of the diagonal block
    for (int r = 0; r < nb; ++r)
      for (int c = r0 + 32 + tid; c < q; c += NT) M[(int64_t)(r0 + r) * q + c] = 0.0f;
    __syncthreads();
    if (warp == 0) {
      // W = L_ii^{-1}, column c = lane: v_r = (delta_rc - sum_{c<=k<r} L_rk v_k) / L_rr
      double v[32];
#pragma unroll
      for (int r = 0; r < 32; ++r) {
        double acc = r == lane ? 1.0 : 0.0;
#pragma unroll
        for (int k = 0; k < r; ++k) acc -= Ld[r][k] * v[k];
        v[r] = r < lane ? 0.0 : acc / Ld[r][r];
      }
#pragma unroll
      for (int r = 0; r < 32; ++r) {
        Wd[r][lane] = (float)v[r];
        if (r < nb && lane < nb) M[(int64_t)(r0 + r) * q + r0 + lane] = (float)v[r];
      }
    }
    __syncthreads();
    for (int jb = warp; jb < ib; jb += NW) {
      const int c = jb * 32 + lane;
      float t[32];
#pragma unroll
      for (int r = 0; r < 32; ++r) t[r] = 0.0f;
      for (int k = jb * 32; k < r0; k += 4) {
        float mk[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) mk[u] = M[(int64_t)(k + u) * q + c];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float4* lr = reinterpret_cast<const float4*>(Lt + (k + u) * 32);
#pragma unroll
          for (int r4 = 0; r4 < 8; ++r4) {
            const float4 l = lr[r4];
            t[4 * r4 + 0] = fmaf(l.x, mk[u], t[4 * r4 + 0]);
            t[4 * r4 + 1] = fmaf(l.y, mk[u], t[4 * r4 + 1]);
            t[4 * r4 + 2] = fmaf(l.z, mk[u], t[4 * r4 + 2]);
            t[4 * r4 + 3] = fmaf(l.w, mk[u], t[4 * r4 + 3]);
          }
        }
      }
      // M_ij = -W_ii T (W lower triangular)
#pragma unroll
      for (int r = 0; r < 32; ++r) {
        float a = 0.0f;
#pragma unroll
        for (int s2 = 0; s2 <= r; ++s2) a = fmaf(Wd[r][s2], t[s2], a);
        if (r < nb) M[(int64_t)(r0 + r) * q + c] = -a;
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------------
// Iteration phases (one CTA).
// ---------------------------------------------------------------------------------------------
using Loop = BLoop;

__device__ __forceinline__ void zero_state(const BInst& I) {
  for (int j = threadIdx.x; j < I.n; j += NT) { I.x[j] = 0.0f; I.xt[j] = 0.0f; }
  for (int i = threadIdx.x; i < I.m; i += NT) { I.y[i] = 0.0f; I.yt[i] = 0.0f; }
}

__device__ __forceinline__ float dot4(const float4 a, const float4 v, float s) {
  return fmaf(a.w, v.w, fmaf(a.z, v.z, fmaf(a.y, v.y, fmaf(a.x, v.x, s))));
}

// Row dots u = A [x1, x2] for two rows ia and ib of the instance together (one warp; ib ignored
// when !hasb).  Rows and x1, x2 start on 16-byte boundaries (row pitch a multiple of 4
// floats): lane l takes the float4 column groups l, l + 32, ..., four groups per step while a
// whole step fits, then one at a time, and the last n mod 4 columns one per lane; every load of
// a step (eight float4 of A, eight of x) is issued before its arithmetic, and the x loads are
// shared by the two rows.
__device__ __forceinline__ void rowdots2(const float* A, int lda, int n, const float* x1, const float* x2, int ia,
                                         int ib, bool hasb, float (&u)[4]) {
  const int lane = threadIdx.x & 31;
  const float* ar = A + (int64_t)ia * lda;
  const float* br = A + (int64_t)(hasb ? ib : ia) * lda;
  const float4* a = reinterpret_cast<const float4*>(ar);
  const float4* b = reinterpret_cast<const float4*>(br);
  const float4* p1 = reinterpret_cast<const float4*>(x1);
  const float4* p2 = reinterpret_cast<const float4*>(x2);
  // float4 groups only where every row and vector is 16-byte aligned (the arenas lay them out so);
  // otherwise every column one at a time below
  const bool vec4 = ((reinterpret_cast<uintptr_t>(ar) | reinterpret_cast<uintptr_t>(br) |
                      reinterpret_cast<uintptr_t>(x1) | reinterpret_cast<uintptr_t>(x2)) & 15) == 0;
  const int nf = vec4 ? n >> 2 : 0;
  float s1a = 0.f, s2a = 0.f, s1b = 0.f, s2b = 0.f;
  int g = lane;
  for (; g + 96 < nf; g += 128) {
    float4 av[4], bv[4], v1[4], v2[4];
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      av[w] = a[g + 32 * w];
      bv[w] = b[g + 32 * w];
      v1[w] = p1[g + 32 * w];
      v2[w] = p2[g + 32 * w];
    }
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      s1a = dot4(av[w], v1[w], s1a);
      s2a = dot4(av[w], v2[w], s2a);
      s1b = dot4(bv[w], v1[w], s1b);
      s2b = dot4(bv[w], v2[w], s2b);
    }
  }
  for (; g < nf; g += 32) {
    const float4 av = a[g], bv = b[g], v1 = p1[g], v2 = p2[g];
    s1a = dot4(av, v1, s1a);
    s2a = dot4(av, v2, s2a);
    s1b = dot4(bv, v1, s1b);
    s2b = dot4(bv, v2, s2b);
  }
  for (int c = 4 * nf + lane; c < n; c += 32) {
    const float v1 = x1[c], v2 = x2[c], av = ar[c], bv = br[c];
    s1a = fmaf(av, v1, s1a);
    s2a = fmaf(av, v2, s2a);
    s1b = fmaf(bv, v1, s1b);
    s2b = fmaf(bv, v2, s2b);
  }
  u[0] = warp_sum(s1a);
  u[1] = warp_sum(s2a);
  u[2] = warp_sum(s1b);
  u[3] = warp_sum(s2b);
}

// z_i = sum_{k <= i} M_ik r_k for R rows i0 + t * stride (t < R; rows past q give nothing),
// one warp.  Each row sums its terms in the order of a single-row walk (lane k, steps of 128
// with four terms each while k + 96 <= i, then the tail k <= i in steps of 32); the R rows'
// loads are issued together, so one round trip to L2 serves R rows.
template <int R>
__device__ __forceinline__ void lower_rowdots(const float* M, int q, const float* r, int i0, int stride,
                                              float (&s)[R]) {
  const int lane = threadIdx.x & 31;
  int it[R];
  const float* mi[R];
  int imax = -1;
#pragma unroll
  for (int t = 0; t < R; ++t) {
    const int i = i0 + t * stride;
    it[t] = i < q ? i : -1;
    mi[t] = M + (int64_t)(i < q ? i : 0) * q;
    imax = it[t] > imax ? it[t] : imax;
    s[t] = 0.f;
  }
  for (int k0 = 0; k0 <= imax; k0 += 128) {
    const int k = k0 + lane;
    float rv[4], mv[R][4];
#pragma unroll
    for (int u = 0; u < 4; ++u) rv[u] = k + 32 * u <= imax ? r[k + 32 * u] : 0.f;
#pragma unroll
    for (int t = 0; t < R; ++t)
#pragma unroll
      for (int u = 0; u < 4; ++u) mv[t][u] = k + 32 * u <= it[t] ? mi[t][k + 32 * u] : 0.f;
#pragma unroll
    for (int t = 0; t < R; ++t) {
      if (k + 96 <= it[t]) {
#pragma unroll
        for (int u = 0; u < 4; ++u) s[t] = fmaf(mv[t][u], rv[u], s[t]);
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (k + 32 * u <= it[t]) s[t] = fmaf(mv[t][u], rv[u], s[t]);
      }
    }
  }
#pragma unroll
  for (int t = 0; t < R; ++t) s[t] = warp_sum(s[t]);
}

// z = M r over the q rows of the lower-triangular M: warp w takes rows w, w + NW, ... eight
// at a time.
__device__ __forceinline__ void lower_matvec(const float* M, int q, const float* r, float* z) {
  constexpr int R = 8;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = warp; i < q; i += R * NW) {
    float sv[R];
    lower_rowdots<R>(M, q, r, i, NW, sv);
    if (lane == 0) {
#pragma unroll
      for (int t = 0; t < R; ++t)
        if (i + t * NW < q) z[i + t * NW] = sv[t];
    }
  }
}

// Per-row scalars of a warp's rows, 32 rows at a time: lane l loads the values of row
// i0 + l * NW (the warp's l-th row of the group) before the group's row dots, and finishes that
// row afterwards, so the rows' epilogues run side by side instead of one after another.
template <int NS>
struct RowScalars {
  float v[NS];
  __device__ __forceinline__ void load(const float* const (&src)[NS], int i, bool ok) {
#pragma unroll
    for (int c = 0; c < NS; ++c) v[c] = ok ? src[c][i] : 1.0f;
  }
};

// Copies len floats from src to the shared-memory area dst with every thread (loads in flight
// together) when `use`; returns the pointer the phase reads.  The caller synchronises.
__device__ __forceinline__ const float* stage_vec(float* dst, const float* src, int len, bool use) {
  if (!use) return src;
  for (int i = threadIdx.x; i < len; i += NT) dst[i] = src[i];
  return dst;
}

// Column sums t_r[j] = sum_i X[i][j] v_r[i] (r < NR) over `rows` rows of a row-major matrix, by
// the whole CTA: warp w takes rows w, w + NW, ...; lane l the columns c0 + l + 32 t (t < 4) of
// each 128-column chunk, so every warp reads whole rows; the warps' partial sums meet in `red`
// (NW x NR x 128 floats) and are added in warp order.  pre(j) loads what the epilogue of column
// j needs (before the cross-warp sum, so its latency overlaps it); fn(j, t, p) finishes column j
// (one thread).  RB rows' loads are in flight per warp step; each column still sums its rows
// in increasing order.  VEC: lane l takes the four consecutive columns c0 + 4 l .. + 3 with one
// float4 load per row (X 16-byte aligned, ldx a multiple of 4), else the columns c0 + l + 32 t.
template <int NR, int RB, bool VEC, class Pre, class Fn>
__device__ __forceinline__ void cta_colsum(const float* X, int ldx, int rows, int cols, const float* v1,
                                           const float* v2, const float* v3, float* red, Pre pre, Fn fn) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float* v[3] = {v1, v2, v3};
  // float4 rows only where X and its pitch keep every row 16-byte aligned
  const bool v4 = VEC && ((reinterpret_cast<uintptr_t>(X) | ((uintptr_t)ldx * sizeof(float))) & 15) == 0;
  for (int c0 = 0; c0 < cols; c0 += 128) {
    float acc[NR][4];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r][0] = acc[r][1] = acc[r][2] = acc[r][3] = 0.0f;
    for (int i0 = warp; i0 < rows; i0 += RB * NW) {
      float a[RB][4], w[RB][NR];
#pragma unroll
      for (int h = 0; h < RB; ++h) {
        const int i = i0 + h * NW;
        const bool ok = i < rows;
        const float* row = X + (int64_t)(ok ? i : 0) * ldx + c0;
#pragma unroll
        for (int r = 0; r < NR; ++r) w[h][r] = ok ? v[r][i] : 0.0f;
        if (v4) {   // columns c0 + 4 lane .. + 3: one float4 (16-byte rows; columns >= cols read as 0)
          const int j = 4 * lane;
          float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
          if (ok && c0 + j < cols) q = *reinterpret_cast<const float4*>(row + j);
          a[h][0] = q.x;
          a[h][1] = c0 + j + 1 < cols ? q.y : 0.0f;
          a[h][2] = c0 + j + 2 < cols ? q.z : 0.0f;
          a[h][3] = c0 + j + 3 < cols ? q.w : 0.0f;
        } else {
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const int j = lane + 32 * t;
            a[h][t] = (ok && c0 + j < cols) ? row[j] : 0.0f;
          }
        }
      }
#pragma unroll
      for (int h = 0; h < RB; ++h)
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
          for (int r = 0; r < NR; ++r) acc[r][t] = fmaf(a[h][t], w[h][r], acc[r][t]);
    }
    const bool mine = tid < 128 && c0 + tid < cols;
    const auto p = pre(mine ? c0 + tid : 0);
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
      for (int t = 0; t < 4; ++t) red[(warp * NR + r) * 128 + (v4 ? 4 * lane + t : lane + 32 * t)] = acc[r][t];
    __syncthreads();
    if (mine) {
      float t[NR];
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        float sum = 0.0f;
#pragma unroll
        for (int w = 0; w < NW; ++w) sum += red[(w * NR + r) * 128 + tid];
        t[r] = sum;
      }
      fn(c0 + tid, t, p);
    }
    __syncthreads();
  }
}

struct F2 {
  float a, b;
};
struct F3 {
  float a, b, c;
};

__device__ void run_instance(const BInst& I, const BCfg& cfg, float* smemA, float* sv, double* red, float* red3,
                             Loop* L, int max_steps) {
  BOut* out = I.out;
  const int m = I.m, n = I.n, q = I.q, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // the vectors each phase reads are staged in shared memory when three of the longest fit
  const int n4 = I.lda;   // n rounded up to a multiple of 4: row pitch and staged-vector offsets
  const bool vs = 3 * (m > n4 ? m : n4) <= kBatchVecFloats;
  const float* A = I.A;
  const int lda = I.lda;
  if (I.stage_smem) {   // same values, same loop order: only where they are read from changes
    for (int i = 0; i < m; ++i)
      for (int j = tid; j < n4; j += NT) smemA[i * n4 + j] = j < n ? I.A[(int64_t)i * I.lda + j] : 0.0f;
    A = smemA;
  }
  const bool resume = I.loop && I.loop->started;
  if (!resume) zero_state(I);
  if (tid == 0) {
    if (resume) {
      *L = *I.loop;
    } else {
      L->rho = cfg.rho0;
      L->pend = 1.0;
      L->k = L->l = L->u = L->done = 0;
      L->status = POGS_MAX_ITER;
      L->started = 1;
    }
  }
  __syncthreads();
  int steps = 0;
  const float alpha = (float)cfg.alpha;
  while (true) {
    const float rho = (float)L->rho, pend = (float)L->pend;
    const bool rescale = pend != 1.0f;
    // ---- prox step (Algorithm 1, Section 3.2, 3.3) ----
    Df pv[6] = {};   // double-float partial sums on the FP32 pipes (B300's FP64 rate is a small fraction)
    for (int k = tid; k < n + m; k += NT) {
      if (k < n) {
        const int j = k;
        const float xtj = pend * I.xt[j], xj = I.x[j], v = xj - xtj;
        if (rescale) I.xt[j] = xtj;
        const int h = I.gh[j];
        const float a = I.ga[j], b = I.gb[j], c = I.gc[j], d = I.gd[j], e = I.ge[j];
        const float xhj = prox_param(h, a, b, c, d, e, rho, v);
        const float muj = -rho * (xhj - v);
        I.xh[j] = xhj;
        I.cx[j] = alpha * xhj + (1.0f - alpha) * xj;
        I.mu[j] = muj;
        df_add_prod(pv[0], muj, muj);
        df_add_prod(pv[1], xhj, muj);
        df_add(pv[2], f_param(h, a, b, c, d, e, xhj));
      } else {
        const int i = k - n;
        const float yti = pend * I.yt[i], yi = I.y[i], v = yi - yti;
        if (rescale) I.yt[i] = yti;
        const int h = I.fh[i];
        const float a = I.fa[i], b = I.fb[i], c = I.fc[i], d = I.fd[i], e = I.fe[i];
        const float yhi = prox_param(h, a, b, c, d, e, rho, v);
        const float nui = -rho * (yhi - v);
        I.yh[i] = yhi;
        I.dy[i] = alpha * yhi + (1.0f - alpha) * yi;
        I.nu[i] = nui;
        df_add_prod(pv[3], yhi, yhi);
        df_add_prod(pv[4], yhi, nui);
        df_add(pv[5], f_param(h, a, b, c, d, e, yhi));
      }
    }
    double pvs[6];
    block_sum_df<6>(pv, pvs, red);   // totals in thread 0; its barriers publish the prox outputs
    Df rs[4] = {};   // primal^2, primal_u^2, dual^2, dual_u^2
    if (I.tall) {
      // r = c + A^T d ; x~ = -A^T y~ ; dual residual (A^T nu + mu)
      const float* v1 = stage_vec(sv, I.dy, m, vs);
      const float* v2 = stage_vec(sv + m, I.nu, m, vs);
      const float* v3 = stage_vec(sv + 2 * m, I.yt, m, vs);
      __syncthreads();
      cta_colsum<3, 8, true>(
          A, lda, m, n, v1, v2, v3, red3, [&](int j) { return F3{I.cx[j], I.mu[j], I.E[j]}; },
          [&](int j, const float* t, const F3& p) {
            I.r[j] = p.a + t[0];
            I.xt[j] = -t[2];
            const float dr = t[1] + p.b;
            df_add_prod(rs[2], dr, dr);
            const float du = dr / p.c;
            df_add_prod(rs[3], du, du);
          });
      const float* rr = stage_vec(sv, I.r, q, vs);
      __syncthreads();
      float* zz = vs ? sv + q : I.z;
      lower_matvec(I.M, q, rr, zz);   // z = M r
      __syncthreads();
      cta_colsum<1, 8, false>(
          I.M, q, q, q, zz, nullptr, nullptr, red3, [&](int j) { return F2{I.xt[j], I.cx[j]}; },
          [&](int j, const float* t, const F2& p) {   // x = M^T z ; x~ += c - x
            I.x[j] = t[0];
            I.xt[j] = p.a + (p.b - t[0]);
          });
      const float* xx = stage_vec(sv, I.x, n, vs);
      const float* xs = stage_vec(sv + n4, I.xh, n, vs);
      __syncthreads();
      for (int g = warp; g < m; g += 32 * NW) {   // y = A x, w = A x^ ; y~ += d - y ; primal residual
        RowScalars<4> sc;
        const float* const src[4] = {I.yt, I.dy, I.yh, I.D};
        const int im = g + lane * NW;
        sc.load(src, im, im < m);
        float mu1 = 0.f, mu2 = 0.f;   // this lane's row of the group
        for (int t = 0; t < 32; t += 2) {   // two rows per step
          const int i = g + t * NW;
          if (i >= m) break;
          float u[4];
          rowdots2(A, lda, n, xx, xs, i, i + NW, i + NW < m, u);
          if (lane == t) { mu1 = u[0]; mu2 = u[1]; }
          if (lane == t + 1) { mu1 = u[2]; mu2 = u[3]; }
        }
        if (im < m) {
          I.y[im] = mu1;
          I.yt[im] = sc.v[0] + (sc.v[1] - mu1);
          const float pr = mu2 - sc.v[2];
          df_add_prod(rs[0], pr, pr);
          const float pu = pr / sc.v[3];
          df_add_prod(rs[1], pu, pu);
        }
      }
    } else {
      const float* cc = stage_vec(sv, I.cx, n, vs);
      const float* xs = stage_vec(sv + n4, I.xh, n, vs);
      __syncthreads();
      float* rw = vs ? sv + 2 * n4 : I.r;     // r, read by the next phase only
      for (int g = warp; g < m; g += 32 * NW) {   // r = A c - d ; primal residual
        RowScalars<3> sc;
        const float* const src[3] = {I.dy, I.yh, I.D};
        const int im = g + lane * NW;
        sc.load(src, im, im < m);
        float mu1 = 0.f, mu2 = 0.f;   // this lane's row of the group
        for (int t = 0; t < 32; t += 2) {   // two rows per step
          const int i = g + t * NW;
          if (i >= m) break;
          float u[4];
          rowdots2(A, lda, n, cc, xs, i, i + NW, i + NW < m, u);
          if (lane == t) { mu1 = u[0]; mu2 = u[1]; }
          if (lane == t + 1) { mu1 = u[2]; mu2 = u[3]; }
        }
        if (im < m) {
          rw[im] = mu1 - sc.v[0];
          const float pr = mu2 - sc.v[1];
          df_add_prod(rs[0], pr, pr);
          const float pu = pr / sc.v[2];
          df_add_prod(rs[1], pu, pu);
        }
      }
      __syncthreads();
      float* zz = vs ? sv : I.z;               // (r sits after the 2 n4 staged floats: no overlap)
      lower_matvec(I.M, q, rw, zz);   // z = M r
      __syncthreads();
      cta_colsum<1, 8, false>(
          I.M, q, q, q, zz, nullptr, nullptr, red3, [&](int i) { return F2{I.dy[i], I.yt[i]}; },
          [&](int i, const float* t, const F2& p) {
            const float d = p.a, yp = d + t[0];   // v = M^T z ; y = d + v ; y~ += d - y ; w = d - y
            I.y[i] = yp;
            I.yt[i] = p.b + (d - yp);
            I.w[i] = d - yp;
          });
      const float* v1 = stage_vec(sv, I.w, m, vs);
      const float* v2 = stage_vec(sv + m, I.nu, m, vs);
      const float* v3 = stage_vec(sv + 2 * m, I.yt, m, vs);
      __syncthreads();
      cta_colsum<3, 8, true>(
          A, lda, m, n, v1, v2, v3, red3, [&](int j) { return F3{I.cx[j], I.mu[j], I.E[j]}; },
          [&](int j, const float* t, const F3& p) {
            const float xp = p.a + t[0];   // x = c + A^T w ; x~ = -A^T y~ ; dual residual
            I.x[j] = xp;
            I.xt[j] = -t[2];
            const float dr = t[1] + p.b;
            df_add_prod(rs[2], dr, dr);
            const float du = dr / p.c;
            df_add_prod(rs[3], du, du);
          });
    }
    double rss[4];
    block_sum_df<4>(rs, rss, red);
    // ---- stopping test (Section 3.4 + gap) and Algorithm 3 ----
    if (tid == 0) {
      // square roots in FP32 of the FP64 totals (seven significant digits are far more than the
      // tolerance test needs; the FP64 square root is a long sequence on the FP64 pipe)
      auto rt = [](double a) { return (double)sqrtf((float)a); };
      const double r_pri = rt(rss[0]), r_dual = rt(rss[2]);
      const double eps_pri = cfg.abs_tol + cfg.rel_tol * rt(pvs[3]);
      const double eps_dual = cfg.abs_tol + cfg.rel_tol * rt(pvs[0]);
      const double gap = pvs[4] + pvs[1], obj = pvs[5] + pvs[2];
      const double eps_gap = cfg.abs_tol + cfg.rel_tol * fabs(obj);
      const int k = L->k;
      L->k = k + 1;
      int done = 0;
      if (!isfinite(r_pri) || !isfinite(r_dual) || !isfinite(gap) || !isfinite(obj)) {
        L->status = POGS_ERR_NONFINITE;
        done = 1;
      } else if (r_pri < eps_pri && r_dual < eps_dual && (!cfg.gap_stop || fabs(gap) < eps_gap)) {
        L->status = POGS_OK;
        done = 1;
      } else if (k + 1 >= cfg.max_iter) {
        L->status = POGS_MAX_ITER;
        done = 1;
      }
      double pend_new = 1.0;
      if (!done && cfg.adaptive) {
        const double rho0 = L->rho;
        double rho1 = rho0;
        if (r_dual < eps_dual && cfg.tau * k > L->l) {
          rho1 = cfg.delta * rho0;
          L->u = k;
        } else if (r_pri < eps_pri && cfg.tau * k > L->u) {
          rho1 = rho0 / cfg.delta;
          L->l = k;
        }
        pend_new = rho0 / rho1;
        L->rho = rho1;
      }
      L->pend = pend_new;
      L->done = done;
      if (done) {
        BOut o;
        o.status = L->status;
        o.iters = L->k;
        o.rho = L->rho;
        o.r_pri = r_pri;
        o.r_dual = r_dual;
        o.eps_pri = eps_pri;
        o.eps_dual = eps_dual;
        o.gap = gap;
        o.obj = obj;
        o.r_pri_u = rt(rss[1]);
        o.r_dual_u = rt(rss[3]);
        *out = o;
      }
    }
    __syncthreads();
    ++steps;
    if (L->done || (max_steps > 0 && steps >= max_steps)) break;
  }
  if (tid == 0 && I.loop) *I.loop = *L;
  const bool finished = L->done != 0;
  __syncthreads();
  if (!finished) return;
  // returned tuple in the original variables (Section 5)
  for (int j = tid; j < n; j += NT) {
    I.ox[j] = I.E[j] * I.xh[j];
    I.omu[j] = I.mu[j] / I.E[j];
  }
  for (int i = tid; i < m; i += NT) {
    I.oy[i] = I.yh[i] / I.D[i];
    I.onu[i] = I.D[i] * I.nu[i];
  }
  __syncthreads();
}

__global__ void __launch_bounds__(NT) batch_admm_kernel(BInst* insts, int count, BCfg cfg, int* queue,
                                                       const int* order, int max_steps, int a_floats) {
  extern __shared__ float smemA[];
  float* sv = smemA + a_floats;   // kBatchVecFloats of vector staging after the matrix budget
  __shared__ double red[6 * NW];
  __shared__ float red3[NW * 3 * 128];
  __shared__ Loop L;
  __shared__ int s_idx;
  while (true) {
    if (threadIdx.x == 0) s_idx = atomicAdd(queue, 1);
    __syncthreads();
    const int pos = s_idx;
    __syncthreads();
    if (pos >= count) break;
    const int idx = order ? order[pos] : pos;
    const BInst& I = insts[idx];
    if (I.out->status != 0 && I.out->iters == 0) continue;   // setup failed: reported as is
    if (I.loop && I.loop->done) continue;                      // already finished
    run_instance(I, cfg, smemA, sv, red, red3, &L, max_steps);
  }
}

}  // namespace

int batch_max_smem() { return 184 * 1024; }

int batch_setup(BInst* d_inst, int count, const BCfg& cfg, cudaStream_t s) {
  if (count <= 0) return 0;
  count_launch(4);
  bsetup_equil_kernel<<<count, NT, 0, s>>>(d_inst, cfg);
  bsetup_gram_kernel<<<count, NT, 0, s>>>(d_inst);
  const int chol_smem = 512 * 33 * sizeof(float);
  static PerDeviceOnce attr;
  if (attr.run([&] {
        if (cudaFuncSetAttribute(bsetup_chol_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, chol_smem) ==
                cudaSuccess &&
            cudaFuncSetAttribute(batch_admm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 batch_max_smem() + kBatchVecFloats * (int)sizeof(float)) == cudaSuccess &&
            cudaFuncSetAttribute(bsetup_inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kInvSmem) ==
                cudaSuccess)
          return 0;
        cudaGetLastError();
        return -1;
      }) != 0)
    return POGS_ERR_CUDA;
  bsetup_chol_kernel<<<count, NT, chol_smem, s>>>(d_inst, cfg.mixed_chol);
  bsetup_inverse_kernel<<<count, NT, kInvSmem, s>>>(d_inst);
  return cudaGetLastError() == cudaSuccess ? 0 : POGS_ERR_CUDA;
}

int batch_iterate(BInst* d_inst, int count, const BCfg& cfg, int* d_queue, const int* d_order, int grid,
                  int smem_bytes, int max_steps, cudaStream_t s) {
  if (count <= 0) return 0;
  count_launch();
  batch_admm_kernel<<<grid, NT, smem_bytes + kBatchVecFloats * sizeof(float), s>>>(d_inst, count, cfg, d_queue,
                                                                                  d_order, max_steps, smem_bytes / 4);
  return cudaGetLastError() == cudaSuccess ? 0 : POGS_ERR_CUDA;
}

}  // namespace pogs
