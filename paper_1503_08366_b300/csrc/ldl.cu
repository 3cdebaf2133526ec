// Sparse LDL^T of the quasi-definite K = [I A^T; A -I] on the device (Section 3.5: the direct
// projection for sparse A, factored once and cached).  See ldl.h for the symbolic side.
//
// Factorization (multifrontal, level by level of the supernodal tree, leaves first): one CTA per
// supernode s assembles its frontal matrix F_s (nf = w + h rows: its w own columns, then the h
// rows R_s below them) from the entries of K in its columns and the update matrices of its
// children (in child order, so the sums are the same on every run), eliminates the w own columns
// in FP64 (right-looking LDL^T without pivoting: K is quasi-definite, every pivot is nonzero), and
// writes its panel [X11; L21] with D on the diagonal, X11 = L11^{-1} (unit lower, strictly lower
// part stored) formed once here, and its update matrix F22 - L21 D L21^T.  Fronts of up to 96 rows
// live in shared memory, larger ones in global scratch.
//
// Solve (per projection): permute the right-hand side into the new order, forward substitution
// level by level from the leaves (each supernode adds its children's update vectors, forms
// y_s = X11 t_s and passes -L21 y_s on to its parent as its own update vector), division by D,
// backward substitution from the root (each supernode gathers the finished unknowns of R_s, then
// applies X11^T), then the epilogue of the projection on the unknowns it returns.  With the
// inverse diagonal blocks cached, a supernode's part of each solve is a few dense matrix-vector
// products with all their loads independent, not a chain of w dependent column steps.
#include <algorithm>
#include <cstring>

#include "epi.cuh"
#include "ldl.h"

namespace pogs {
namespace {

constexpr int kLdlThreads = 256;

struct FrontArgs {
  const int *nodes, *first, *width, *row_off, *child_off, *child, *rel_off, *rel, *asm_off, *asm_pos, *asm_src;
  const int64_t *panel_off, *upd_off, *front_off;
  const float* va;
  double *panel, *upd, *front;
  int* err;
};

// F (nf x nf, row-major, lower part used): assemble, eliminate the first w columns, write out.
__device__ void ldl_front(const FrontArgs& a, int s, double* F) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int w = a.width[s], h = a.row_off[s + 1] - a.row_off[s], nf = w + h;
  for (int i = tid; i < nf * nf; i += blockDim.x) F[i] = 0.0;
  __syncthreads();
  for (int t = a.asm_off[s] + tid; t < a.asm_off[s + 1]; t += blockDim.x) {
    const int src = a.asm_src[t];
    F[a.asm_pos[t]] = src >= 0 ? (double)a.va[src] : (src == -1 ? 1.0 : -1.0);
  }
  __syncthreads();
  for (int k = a.child_off[s]; k < a.child_off[s + 1]; ++k) {   // extend-add, children in order
    const int c = a.child[k];
    const int hc = a.row_off[c + 1] - a.row_off[c];
    const int* rl = a.rel + a.rel_off[c];
    const double* U = a.upd + a.upd_off[c];
    for (int idx = tid; idx < hc * hc; idx += blockDim.x) {
      const int i = idx / hc, j = idx - i * hc;
      if (j <= i) F[rl[i] * nf + rl[j]] += U[idx];
    }
    __syncthreads();
  }
  __shared__ int s_bad;
  if (tid == 0) s_bad = 0;
  __syncthreads();
  for (int k = 0; k < w; ++k) {
    double dk = F[k * nf + k];
    if (!(fabs(dk) > 1e-300) || !isfinite(dk)) {   // cannot happen for quasi-definite K
      if (tid == 0) s_bad = 1;
      dk = 1.0;
    }
    for (int i = k + 1 + tid; i < nf; i += blockDim.x) F[i * nf + k] /= dk;
    __syncthreads();
    for (int i = k + 1 + warp; i < nf; i += nwarps) {
      const double lik = F[i * nf + k] * dk;
      for (int j = k + 1 + lane; j <= i; j += 32) F[i * nf + j] -= lik * F[j * nf + k];
    }
    __syncthreads();
  }
  if (tid == 0 && s_bad) atomicExch(a.err, POGS_ERR_NUMERIC);
  // X11 = L11^{-1}: from L11 X11 = I, X_ij = -sum_{k=j}^{i-1} L_ik X_kj (i > j, X_jj = 1); thread j
  // forms column j top down and keeps it in row j of F's upper triangle (F[j][i] = X_ij), which
  // the elimination leaves unused and no other thread reads
  for (int j = tid; j < w; j += blockDim.x)
    for (int i = j + 1; i < w; ++i) {
      double acc = F[i * nf + j];
      for (int k = j + 1; k < i; ++k) acc = fma(F[i * nf + k], F[j * nf + k], acc);
      F[j * nf + i] = -acc;
    }
  __syncthreads();
  // panel: rows i < w hold X11 below the diagonal and D on it, rows i >= w hold L21
  double* P = a.panel + a.panel_off[s];
  for (int idx = tid; idx < nf * w; idx += blockDim.x) {
    const int i = idx / w, j = idx - i * w;
    P[idx] = i >= w ? F[i * nf + j] : i > j ? F[j * nf + i] : i == j ? F[i * nf + i] : 0.0;
  }
  if (h > 0 && a.upd_off) {
    double* U = a.upd + a.upd_off[s];
    for (int idx = tid; idx < h * h; idx += blockDim.x) {
      const int i = idx / h, j = idx - i * h;
      U[idx] = (j <= i) ? F[(w + i) * nf + w + j] : 0.0;
    }
  }
}

__global__ void __launch_bounds__(kLdlThreads) ldl_front_smem_kernel(FrontArgs a, int base) {
  extern __shared__ double Fs[];
  ldl_front(a, a.nodes[base + blockIdx.x], Fs);
}

__global__ void __launch_bounds__(kLdlThreads) ldl_front_global_kernel(FrontArgs a, int base) {
  const int s = a.nodes[base + blockIdx.x];
  ldl_front(a, s, a.front + a.front_off[s]);
}

struct SolveArgs {
  const int *nodes, *first, *width, *row_off, *rows, *child_off, *child, *rel_off, *rel, *vec_off;
  const int64_t* panel_off;
  const double* panel;
  double *y, *uvec;
};

// Forward substitution for the supernodes of one level: t = [y_s; 0] + children's update
// vectors, t[:w] <- X11 t[:w], t[w:] -= L21 t[:w]; y_s = t[:w], the supernode's update vector =
// t[w:].
__global__ void __launch_bounds__(128) ldl_forward_kernel(SolveArgs a, int base) {
  extern __shared__ double t[];
  const int s = a.nodes[base + blockIdx.x];
  const int tid = threadIdx.x;
  const int f = a.first[s], w = a.width[s], h = a.row_off[s + 1] - a.row_off[s], nf = w + h;
  for (int i = tid; i < nf; i += blockDim.x) t[i] = i < w ? a.y[f + i] : 0.0;
  __syncthreads();
  for (int k = a.child_off[s]; k < a.child_off[s + 1]; ++k) {
    const int c = a.child[k];
    const int hc = a.row_off[c + 1] - a.row_off[c];
    const int* rl = a.rel + a.rel_off[c];
    const double* u = a.uvec + a.vec_off[c];
    for (int i = tid; i < hc; i += blockDim.x) t[rl[i]] += u[i];
    __syncthreads();
  }
  const double* P = a.panel + a.panel_off[s];
  // t[0:w] <- X11 t[0:w], z_i = t_i + sum_{k<i} X_ik t_k: rows in chunks of blockDim, the last chunk
  // first (a chunk reads t only at its own and earlier rows, which are still unchanged)
  const int bd = blockDim.x;
  for (int c0 = ((w - 1) / bd) * bd; c0 >= 0; c0 -= bd) {
    const int i = c0 + tid;
    double z = 0.0;
    if (i < w) {
      const double* Xi = P + (int64_t)i * w;
      z = t[i];
      for (int k = 0; k < i; ++k) z = fma(Xi[k], t[k], z);
    }
    __syncthreads();
    if (i < w) t[i] = z;
    __syncthreads();
  }
  // t[w:] -= L21 t[0:w]
  for (int r = w + tid; r < nf; r += blockDim.x) {
    const double* Lr = P + (int64_t)r * w;
    double acc = 0.0;
    for (int k = 0; k < w; ++k) acc = fma(Lr[k], t[k], acc);
    t[r] -= acc;
  }
  __syncthreads();
  for (int i = tid; i < nf; i += blockDim.x) {
    if (i < w) a.y[f + i] = t[i];
    else a.uvec[a.vec_off[s] + i - w] = t[i];
  }
}

// Backward substitution for the supernodes of one level (from the root): t = D^{-1} y_s -
// L21^T y[R_s] (rows of R_s are finished), then t <- L11^{-T} t = X11^T t.
__global__ void __launch_bounds__(128) ldl_backward_kernel(SolveArgs a, int base) {
  extern __shared__ double t[];
  const int s = a.nodes[base + blockIdx.x];
  const int tid = threadIdx.x;
  const int f = a.first[s], w = a.width[s], h = a.row_off[s + 1] - a.row_off[s], nf = w + h;
  const double* P = a.panel + a.panel_off[s];
  const int* R = a.rows + a.row_off[s];
  for (int i = tid; i < nf; i += blockDim.x) t[i] = i < w ? a.y[f + i] / P[i * w + i] : a.y[R[i - w]];
  __syncthreads();
  for (int k = tid; k < w; k += blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < h; ++i) acc += P[(w + i) * w + k] * t[w + i];
    t[k] -= acc;
  }
  __syncthreads();
  // t[0:w] <- X11^T t[0:w], x_k = t_k + sum_{i>k} X_ik t_i: rows in chunks of blockDim, the first
  // chunk first (a chunk reads t only at its own and later rows, which are still unchanged)
  const int bd = blockDim.x;
  for (int c0 = 0; c0 < w; c0 += bd) {
    const int k = c0 + tid;
    double x = 0.0;
    if (k < w) {
      x = t[k];
      for (int i = k + 1; i < w; ++i) x = fma(P[(int64_t)i * w + k], t[i], x);
    }
    __syncthreads();
    if (k < w) t[k] = x;
    __syncthreads();
  }
  for (int i = tid; i < w; i += blockDim.x) a.y[f + i] = t[i];
}

// y[k] = sign * v[perm[k] - base] on the unknowns of one block, 0 elsewhere.
__global__ void ldl_permute_in_kernel(const int* __restrict__ perm, int N, int base, int len, float sign,
                                      const float* __restrict__ v, double* __restrict__ y) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
    const int o = perm[k] - base;
    y[k] = (o >= 0 && o < len) ? (double)sign * (double)v[o] : 0.0;
  }
}

template <int EPI>
__global__ void ldl_permute_out_kernel(const int* __restrict__ perm, int N, int base, int len,
                                       const double* __restrict__ y, EpiArgs ep) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
    const int o = perm[k] - base;
    if (o >= 0 && o < len) epi_r<EPI>(ep, o, len, (float)y[k]);
  }
}

template <class T>
int upload(LdlFactor& F, T** dst, const std::vector<T>& src, cudaStream_t s) {
  void* p = nullptr;
  const size_t bytes = std::max<size_t>(1, src.size()) * sizeof(T);
  if (pool_alloc(&p, bytes, s) != 0) return POGS_ERR_OOM;
  F.allocs.push_back(p);
  F.device_bytes += (int64_t)bytes;
  if (!src.empty() && cudaMemcpyAsync(p, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return POGS_ERR_CUDA;
  *dst = static_cast<T*>(p);
  return 0;
}

template <class T>
int alloc(LdlFactor& F, T** dst, size_t count, cudaStream_t s) {
  void* p = nullptr;
  const size_t bytes = std::max<size_t>(1, count) * sizeof(T);
  if (pool_alloc(&p, bytes, s) != 0) return POGS_ERR_OOM;
  F.allocs.push_back(p);
  F.device_bytes += (int64_t)bytes;
  *dst = static_cast<T*>(p);
  return 0;
}

}  // namespace

void LdlFactor::release(cudaStream_t s) {
  for (void* p : allocs) cudaFreeAsync(p, s);
  allocs.clear();
  device_bytes = 0;
}

int ldl_factor(const LdlSymbolic& S, const float* va, LdlFactor& F, int* err, cudaStream_t s) {
  F = LdlFactor();
  F.N = S.N;
  F.n = S.n;
  F.m = S.m;
  F.ns = S.ns;
  F.levels = S.levels;
  F.max_front = S.max_front;
  F.panel_entries = S.panel_total;
  F.level_off = S.level_off;
  // the solve kernels loop over any block size: each level gets the smallest of 32, 64 or 128
  // threads that covers its largest front (the many small fronts near the leaves then fit more
  // CTAs per SM)
  F.level_threads.assign(S.levels, 32);
  for (int l = 0; l < S.levels; ++l) {
    int nfmax = 0;
    for (int k = S.level_off[l]; k < S.level_off[l + 1]; ++k) {
      const int s2 = S.level_nodes[k];
      nfmax = std::max(nfmax, S.width[s2] + (S.row_off[s2 + 1] - S.row_off[s2]));
    }
    F.level_threads[l] = nfmax <= 32 ? 32 : nfmax <= 64 ? 64 : 128;
  }
  // the solve keeps one front column vector per CTA in shared memory
  if ((size_t)S.max_front * sizeof(double) > 160 * 1024) return POGS_ERR_CAPACITY;
  int rc = 0;
  auto up = [&](auto** d, const auto& v) { if (rc == 0) rc = upload(F, d, v, s); };
  up(&F.perm, S.perm);
  up(&F.first, S.first);
  up(&F.width, S.width);
  up(&F.row_off, S.row_off);
  up(&F.rows, S.rows);
  up(&F.child_off, S.child_off);
  up(&F.child, S.child);
  up(&F.level_nodes, S.level_nodes);
  up(&F.rel_off, S.rel_off);
  up(&F.rel, S.rel);
  up(&F.vec_off, S.vec_off);
  up(&F.panel_off, S.panel_off);
  if (rc == 0) rc = alloc(F, &F.panel, (size_t)S.panel_total, s);
  if (rc == 0) rc = alloc(F, &F.y, (size_t)S.N, s);
  if (rc == 0) rc = alloc(F, &F.uvec, (size_t)S.vec_total, s);
  if (rc != 0) return rc;
  // factorization-only data: assembly maps, update arena, global fronts (freed at the end)
  LdlFactor tmp;
  int *asm_off = nullptr, *asm_pos = nullptr, *asm_src = nullptr;
  int64_t *upd_off = nullptr, *front_off = nullptr;
  double *upd = nullptr, *front = nullptr;
  auto upt = [&](auto** d, const auto& v) { if (rc == 0) rc = upload(tmp, d, v, s); };
  upt(&asm_off, S.asm_off);
  upt(&asm_pos, S.asm_pos);
  upt(&asm_src, S.asm_src);
  std::vector<int64_t> uo(S.upd_off);
  if (uo.empty()) uo.push_back(0);
  upt(&upd_off, uo);
  upt(&front_off, S.front_off);
  if (rc == 0) rc = alloc(tmp, &upd, (size_t)S.upd_total, s);
  if (rc == 0) rc = alloc(tmp, &front, (size_t)S.front_max, s);
  if (rc != 0) {
    tmp.release(s);
    return rc;
  }
  FrontArgs a{F.level_nodes, F.first, F.width, F.row_off, F.child_off, F.child, F.rel_off, F.rel, asm_off,
              asm_pos, asm_src, F.panel_off, upd_off, front_off, va, F.panel, upd, front, err};
  const size_t smem = (size_t)S.smem_front_max * S.smem_front_max * sizeof(double);
  static PerDeviceOnce attr;
  if (attr.run([] {
        const int bytes = LdlSymbolic::kSmemFront * LdlSymbolic::kSmemFront * (int)sizeof(double);
        if (cudaFuncSetAttribute(ldl_front_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) ==
                cudaSuccess &&
            cudaFuncSetAttribute(ldl_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024) ==
                cudaSuccess &&
            cudaFuncSetAttribute(ldl_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024) ==
                cudaSuccess)
          return 0;
        cudaGetLastError();
        return -1;
      }) != 0) {
    tmp.release(s);
    return POGS_ERR_CUDA;
  }
  for (int l = 0; l < S.levels; ++l) {
    const int b = S.level_off[l], split = S.level_split[l], e = S.level_off[l + 1];
    if (split > b) {
      count_launch();
      ldl_front_smem_kernel<<<split - b, kLdlThreads, smem, s>>>(a, b);
    }
    if (e > split) {
      count_launch();
      ldl_front_global_kernel<<<e - split, kLdlThreads, 0, s>>>(a, split);
    }
  }
  rc = cudaGetLastError() == cudaSuccess ? 0 : POGS_ERR_CUDA;
  tmp.release(s);
  return rc;
}

int ldl_launches(const LdlFactor& F) { return 2 + 2 * F.levels; }

void ldl_apply(const LdlFactor& F, bool tall, const float* v, int epi, const EpiArgs& ep, cudaStream_t s) {
  const int base = tall ? 0 : F.n, len = tall ? F.n : F.m;
  const int grid = std::min(1184, (F.N + 255) / 256);
  count_launch(ldl_launches(F));
  ldl_permute_in_kernel<<<grid, 256, 0, s>>>(F.perm, F.N, base, len, tall ? 1.0f : -1.0f, v, F.y);
  SolveArgs a{F.level_nodes, F.first, F.width, F.row_off, F.rows, F.child_off, F.child, F.rel_off, F.rel,
              F.vec_off, F.panel_off, F.panel, F.y, F.uvec};
  const size_t smem = (size_t)F.max_front * sizeof(double);
  for (int l = 0; l < F.levels; ++l) {
    const int b = F.level_off[l], cnt = F.level_off[l + 1] - b;
    ldl_forward_kernel<<<cnt, F.level_threads[l], smem, s>>>(a, b);
  }
  for (int l = F.levels - 1; l >= 0; --l) {
    const int b = F.level_off[l], cnt = F.level_off[l + 1] - b;
    ldl_backward_kernel<<<cnt, F.level_threads[l], smem, s>>>(a, b);
  }
  switch (epi) {
    case EPR_RAW: ldl_permute_out_kernel<EPR_RAW><<<grid, 256, 0, s>>>(F.perm, F.N, base, len, F.y, ep); break;
    case EPR_TALL_X: ldl_permute_out_kernel<EPR_TALL_X><<<grid, 256, 0, s>>>(F.perm, F.N, base, len, F.y, ep); break;
    case EPR_FAT_Y: ldl_permute_out_kernel<EPR_FAT_Y><<<grid, 256, 0, s>>>(F.perm, F.N, base, len, F.y, ep); break;
    case EPR_ADD: ldl_permute_out_kernel<EPR_ADD><<<grid, 256, 0, s>>>(F.perm, F.N, base, len, F.y, ep); break;
  }
}

}  // namespace pogs
