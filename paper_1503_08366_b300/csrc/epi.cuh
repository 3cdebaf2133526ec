// Epilogues of the two passes over A^ (dense column sums / row dots, and the CSR kernels
// that replace them for sparse A): each receives one output index and its accumulated
// products and writes the fused per-element update and the residual partials.
#pragma once
#include "kernels.h"

namespace pogs {

// CGLS epilogues (indirect projection), shared by both GEMV orientations with one right-hand
// side: i indexes the output vector, u = (M v)_i.  Codes 5..8 of EpiT / EpiN.
template <int E>
__device__ __forceinline__ void epi_cg(const EpiArgs& ep, int i, float u, Df* res) {
  if constexpr (E == 5) {            // r_top = top - M u0
    const float r = ep.cg_top[i] - u;
    ep.cg_rt[i] = r;
    df_add_prod(res[0], r, r);
  } else if constexpr (E == 6) {     // r_bot = sign * bot - u0; s = M^T r_top + r_bot; p = s
    const float rb = ep.cg_sign * ep.cg_bot[i] - ep.cg_u[i];
    const float sv = u + rb;
    ep.cg_rb[i] = rb;
    ep.cg_s[i] = sv;
    ep.cg_p[i] = sv;
    df_add_prod(res[0], sv, sv);
    df_add_prod(res[1], rb, rb);
  } else if constexpr (E == 7) {     // q = M p
    ep.out1[i] = u;
    df_add_prod(res[0], u, u);
  } else {                           // s = M^T r_top + r_bot
    const float sv = u + ep.cg_rb[i];
    ep.cg_s[i] = sv;
    df_add_prod(res[0], sv, sv);
  }
}

template <int EPI>
__device__ __forceinline__ void epi_t(const EpiArgs& ep, int j, float t1, float t2, float t3, Df* res) {
  if constexpr (EPI == EPT_RAW) {
    ep.out1[j] = t1;
    if (ep.out2) ep.out2[j] = t2;
  } else if constexpr (EPI == EPT_TALL_R) {
    ep.r[j] = ep.cx[j] + t1;
    ep.xt[j] = -t3;                     // x~ re-derived as -A^T y~ (Section 3.3 invariant)
    const float dr = t2 + ep.mu[j];
    df_add_prod(res[0], dr, dr);
    const float du = dr / ep.E[j];
    df_add_prod(res[1], du, du);
  } else if constexpr (EPI == EPT_FAT_X) {
    const float c = ep.cx[j];
    const float xp = c + t1;
    ep.x[j] = xp;
    ep.xt[j] = -t3;                     // x~^{k+1} = -A^T y~^{k+1} (Section 3.3 invariant)
    const float dr = t2 + ep.mu[j];
    df_add_prod(res[0], dr, dr);
    const float du = dr / ep.E[j];
    df_add_prod(res[1], du, du);
  } else if constexpr (EPI == EPT_SK_COL) {
    // sk_num < 0: keep e (Frobenius norm only, no Sinkhorn-Knopp update)
    float ej;
    if (ep.sk_num > 0.0f) {
      ej = ep.sk_num / (t1 + ep.sk_reg);
      ep.sk_vec[j] = ej;
    } else {
      ej = ep.sk_vec[j];
    }
    df_add_prod(res[0], ej, t1);   // sum_ij d_i A_ij^2 e_j = ||D A E||_F^2 (p = 2)
  } else if constexpr (EPI == EPT_REFINE) {
    ep.out1[j] = ep.in1[j] - ep.in2[j] - t1;
  } else if constexpr (EPI >= EPT_CG_R) {
    epi_cg<EPI>(ep, j, t1, res);
  }
}

template <int EPI>
__device__ __forceinline__ void epi_n(const EpiArgs& ep, int i, float u1, float u2, Df* res) {
  if constexpr (EPI == EPN_RAW) {
    ep.out1[i] = u1;
    if (ep.out2) ep.out2[i] = u2;
  } else if constexpr (EPI == EPN_TALL_Y) {
    ep.y[i] = u1;
    ep.yt[i] += ep.dy[i] - u1;          // y~ <- y~ + y_r - y^{k+1}
    const float pr = u2 - ep.yh[i];
    df_add_prod(res[0], pr, pr);
    const float pu = pr / ep.D[i];
    df_add_prod(res[1], pu, pu);
  } else if constexpr (EPI == EPN_FAT_R) {
    ep.r[i] = u1 - ep.dy[i];
    const float pr = u2 - ep.yh[i];
    df_add_prod(res[0], pr, pr);
    const float pu = pr / ep.D[i];
    df_add_prod(res[1], pu, pu);
  } else if constexpr (EPI == EPN_SK_ROW) {
    ep.sk_vec[i] = ep.sk_num / (u1 + ep.sk_reg);
  } else if constexpr (EPI == EPN_REFINE) {
    ep.out1[i] = ep.in1[i] - ep.in2[i] - u1;
  } else if constexpr (EPI >= EPN_CG_R) {
    epi_cg<EPI>(ep, i, u1, res);
  }
}

// Epilogue of the products with the cached inverse (packed-triangle or sparse LDL^T solves): one
// element idx of the result v.
template <int EPI>
__device__ __forceinline__ void epi_r(const EpiArgs& ep, int idx, int q, float v) {
  if constexpr (EPI == EPR_RAW) {
    ep.out1[idx] = v;
  } else if constexpr (EPI == EPR_ADD) {
    if (idx < q) ep.out1[idx] = ep.in1[idx] + v;
  } else if constexpr (EPI == EPR_TALL_X) {
    if (idx < q) {
      const float c = ep.cx[idx];
      const float xv = ep.in1 ? ep.in1[idx] + v : v;   // in1: refinement base x0
      ep.x[idx] = xv;
      ep.xt[idx] += c - xv;             // x~ <- x~ + x_r - x^{k+1}
    }
  } else if constexpr (EPI == EPR_FAT_Y) {
    if (idx < q) {
      const float d = ep.dy[idx];
      const float yp = d + (ep.in1 ? ep.in1[idx] + v : v);
      ep.y[idx] = yp;
      ep.yt[idx] += d - yp;             // y~ <- y~ + y_r - y^{k+1}
      ep.w[idx] = d - yp;
    }
  }
}

}  // namespace pogs
