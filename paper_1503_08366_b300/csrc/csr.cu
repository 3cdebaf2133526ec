// Sparse A (Section 3.5's sparse case, Section 4.1 equilibration on the nonzeros).  A is
// ingested in CSR form (row pointers, sorted unique column indices, values) and kept twice
// in HBM: as CSR of A^ (m rows) for the row-dot pass and as CSR of A^T (n rows) for the
// column-sum pass, so that both passes are gathers over contiguous rows with no atomics and
// a fixed summation order.  The transposed copy is built on the device by a stable multi-split
// (warp-level ranks of equal column indices), so its entries of every column come in
// increasing row order; `perm` maps each of its entries back to the CSR entry it copies.
//
// The two pass kernels replace the dense GEMVs one for one and call the same epilogues
// (epi.cuh), so Algorithm 2, the projection passes, refinement and CGLS run unchanged on
// sparse A.
#include "epi.cuh"
#include "kernels.h"

namespace pogs {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// Rows of a CSR matrix times up to three vectors: G lanes per row (a power of two <= 32),
// lane-strided products, a fixed xor-shuffle tree inside the group, then the pass's epilogue
// on the group's first lane (TR: the column-sum epilogue, row = column of A).  Every thread
// makes the same number of row trips so that the shuffles always see whole warps.  Each block
// writes its two residual partials to ep.res_part[2 * blockIdx.x + t].
// PK: the right-hand sides come interleaved in vp (float2 for two, float4 for three), one
// gather per nonzero instead of one per right-hand side.
template <int NRHS, int PK>
struct Gather {
  const float *v1, *v2, *v3;
  const float* vp;
  __device__ __forceinline__ void operator()(int c, float a, float& s1, float& s2, float& s3) const {
    if constexpr (PK && NRHS == 3) {
      const float4 x = __ldg(reinterpret_cast<const float4*>(vp) + c);
      s1 = fmaf(a, x.x, s1);
      s2 = fmaf(a, x.y, s2);
      s3 = fmaf(a, x.z, s3);
    } else if constexpr (PK && NRHS == 2) {
      const float2 x = __ldg(reinterpret_cast<const float2*>(vp) + c);
      s1 = fmaf(a, x.x, s1);
      s2 = fmaf(a, x.y, s2);
    } else {
      s1 = fmaf(a, __ldg(v1 + c), s1);
      if constexpr (NRHS >= 2) s2 = fmaf(a, __ldg(v2 + c), s2);
      if constexpr (NRHS == 3) s3 = fmaf(a, __ldg(v3 + c), s3);
    }
  }
};

// Eight resident 256-thread blocks per SM (at most 32 registers); the grid is one such wave.
constexpr int kSpmvBlocksPerSm = 8;

template <int NRHS, bool SQ, bool TR, int EPI, int G, int PK>
__global__ void __launch_bounds__(256, kSpmvBlocksPerSm) spmv_kernel(const int* __restrict__ rp, const int* __restrict__ ci,
                                                   const float* __restrict__ va, int nrows,
                                                   const float* __restrict__ v1, const float* __restrict__ v2,
                                                   const float* __restrict__ v3, const float* __restrict__ vp,
                                                   EpiArgs ep, const DevState* __restrict__ guard) {
  const Gather<NRHS, PK> gather{v1, v2, v3, vp};
  __shared__ double sh[2 * 8];
  if (guard && guard->done) return;
  if (ep.cg_done && *ep.cg_done) return;
  const int lg = threadIdx.x & (G - 1);
  const int group = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G);
  const int ngroups = (int)((int64_t)gridDim.x * blockDim.x / G);
  const int trips = (nrows + ngroups - 1) / ngroups;
  Df res[2] = {};
  for (int t = 0; t < trips; ++t) {
    const int row = group + t * ngroups;
    float s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
    if (row < nrows) {
      const int k1 = __ldg(rp + row + 1);
      int k = __ldg(rp + row) + lg;
      // four entries per lane per step: their values and indices load together, then the gathers
      for (; k + 3 * G < k1; k += 4 * G) {
        float a[4];
        int c[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          a[u] = __ldg(va + k + u * G);
          c[u] = __ldg(ci + k + u * G);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) gather(c[u], SQ ? a[u] * a[u] : a[u], s1, s2, s3);
      }
      for (; k < k1; k += G) {
        const float av = __ldg(va + k);
        gather(__ldg(ci + k), SQ ? av * av : av, s1, s2, s3);
      }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      s1 += __shfl_xor_sync(kFull, s1, o, G);
      if constexpr (NRHS >= 2) s2 += __shfl_xor_sync(kFull, s2, o, G);
      if constexpr (NRHS == 3) s3 += __shfl_xor_sync(kFull, s3, o, G);
    }
    if (lg == 0 && row < nrows) {
      if constexpr (TR) epi_t<EPI>(ep, row, s1, s2, s3, res);
      else epi_n<EPI>(ep, row, s1, s2, res);
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

// Structure and value checks, one warp per row: rp[0] = 0, rp[m] = nnz, rp nondecreasing,
// column indices in [0, n) and strictly increasing in each row, finite values.  Reads stay in
// bounds whatever the input (a bad row is flagged and skipped).
__global__ void csr_check_kernel(const int* __restrict__ rp, const int* __restrict__ ci,
                                 const float* __restrict__ va, int m, int n, int64_t nnz, int* err) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int bad = 0, nonfinite = 0;
  for (int64_t r = w0; r < m; r += nw) {
    const int64_t a = rp[r], b = rp[r + 1];
    if ((r == 0 && a != 0) || (r == m - 1 && b != nnz) || a < 0 || b < a || b > nnz) {
      bad = 1;
      continue;
    }
    for (int64_t k = a + lane; k < b; k += 32) {
      const int c = ci[k];
      if (c < 0 || c >= n || (k > a && c <= ci[k - 1])) bad = 1;
      if (!isfinite(va[k])) nonfinite = 1;
    }
  }
  if (bad) atomicCAS(err, 0, POGS_ERR_ARG);
  else if (nonfinite) atomicCAS(err, 0, POGS_ERR_NONFINITE);
}

// rowidx[k] = row of CSR entry k (one warp per row).
__global__ void csr_rows_kernel(const int* __restrict__ rp, int m, int* __restrict__ rowidx) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = w0; r < m; r += nw)
    for (int k = rp[r] + lane; k < rp[r + 1]; k += 32) rowidx[k] = (int)r;
}

// Stable multi-split of the CSR entries by column.  Warp w owns entries [w*C, min(nnz,(w+1)*C))
// and row w of the table cnt (nch x n).  count: cnt[w][j] = entries of column j in the chunk.
// place: cnt[w][j] holds the chunk's first position in column j (relative to colptr[j]);
// entries of equal column inside a step of 32 are ranked by lane, so the order of every column
// is the CSR order (increasing row).
template <bool PLACE>
__global__ void csr_split_kernel(const int* __restrict__ ci, const float* __restrict__ va,
                                 const int* __restrict__ rowidx, int64_t nnz, int64_t chunk, int nch, int n,
                                 int* __restrict__ cnt, const int* __restrict__ colptr, int* __restrict__ t_ci,
                                 float* __restrict__ t_va, int* __restrict__ perm) {
  const int lane = threadIdx.x & 31;
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (w >= nch) return;
  const int64_t k0 = w * chunk, k1 = min(nnz, k0 + chunk);
  int* row = cnt + w * (int64_t)n;
  const unsigned lt = (1u << lane) - 1u;
  for (int64_t base = k0; base < k1; base += 32) {
    const int64_t k = base + lane;
    const bool on = k < k1;
    const int j = on ? ci[k] : -1;
    const unsigned peers = __match_any_sync(kFull, j);
    const int leader = __ffs(peers) - 1;
    if (on) {
      if constexpr (PLACE) {
        const int64_t pos = (int64_t)colptr[j] + row[j] + __popc(peers & lt);
        t_ci[pos] = rowidx[k];
        t_va[pos] = va[k];
        perm[pos] = (int)k;
      }
    }
    __syncwarp();
    if (on && lane == leader) row[j] += __popc(peers);
    __syncwarp();
  }
}

// Per column: turn the chunk counts into exclusive chunk offsets; tot[j] = entries of column j.
__global__ void csr_chunk_offsets_kernel(int* __restrict__ cnt, int nch, int n, int* __restrict__ tot) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    int run = 0;
    for (int w = 0; w < nch; ++w) {
      const int c = cnt[(int64_t)w * n + j];
      cnt[(int64_t)w * n + j] = run;
      run += c;
    }
    tot[j] = run;
  }
}

// colptr = exclusive scan of tot (n + 1 entries), one block of 1024 threads, in order.
__global__ void __launch_bounds__(1024) scan_kernel(const int* __restrict__ tot, int n, int* __restrict__ colptr) {
  __shared__ int wsum[32];
  __shared__ int carry_s;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  for (int base = 0; base < n; base += 1024) {
    const int i = base + threadIdx.x;
    const int v = i < n ? tot[i] : 0;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
      int ws = wsum[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, ws, o);
        if (lane >= o) ws += y;
      }
      wsum[lane] = ws;
    }
    __syncthreads();
    const int carry = carry_s;
    const int incl = x + (wid > 0 ? wsum[wid - 1] : 0) + carry;
    if (i < n) colptr[i] = incl - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry_s = incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) colptr[n] = carry_s;
}

// A^ = D A E on the CSR values (the dense path's expression), then the transposed copy's
// values by the permutation (exact copies).
__global__ void csr_scale_kernel(const int* __restrict__ rp, const int* __restrict__ ci, float* __restrict__ va,
                                 int m, const float* __restrict__ D, const float* __restrict__ E) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = w0; r < m; r += nw) {
    const float d = D[r];
    for (int k = rp[r] + lane; k < rp[r + 1]; k += 32) va[k] *= d * E[ci[k]];
  }
}

__global__ void gather_kernel(const float* __restrict__ src, const int* __restrict__ perm, int64_t k,
                              float* __restrict__ dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[perm[i]];
}

// Interleave two or three right-hand sides for the packed gathers: vp[i] = (v1, v2[, v3, 0]).
template <int NRHS>
__global__ void pack_rhs_kernel(const float* __restrict__ v1, const float* __restrict__ v2,
                                const float* __restrict__ v3, int k, float* __restrict__ vp,
                                const DevState* __restrict__ guard, const int* __restrict__ cg_done) {
  if (guard && guard->done) return;
  if (cg_done && *cg_done) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) {
    if constexpr (NRHS == 3) reinterpret_cast<float4*>(vp)[i] = make_float4(v1[i], v2[i], v3[i], 0.0f);
    else reinterpret_cast<float2*>(vp)[i] = make_float2(v1[i], v2[i]);
  }
}

// Dense copy of the CSR matrix into a zeroed m x lda row-major buffer.
__global__ void csr_densify_kernel(const int* __restrict__ rp, const int* __restrict__ ci,
                                   const float* __restrict__ va, int m, float* __restrict__ A, int64_t lda) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = w0; r < m; r += nw)
    for (int k = rp[r] + lane; k < rp[r + 1]; k += 32) A[r * lda + ci[k]] = va[k];
}

int grid_rows(int64_t rows, int per_block, int num_sms, int per_sm = 8) {
  const int64_t g = (rows + per_block - 1) / per_block;
  const int64_t cap = (int64_t)num_sms * per_sm;
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

template <int NRHS, bool SQ, bool TR, int G, int PK>
void spmv_dispatch(int epi, const int* rp, const int* ci, const float* va, int nrows, const float* v1,
                   const float* v2, const float* v3, const float* vp, int grid, const EpiArgs& ep,
                   const DevState* guard, cudaStream_t s) {
#define POGS_S(E) \
  spmv_kernel<NRHS, SQ, TR, E, G, PK><<<grid, 256, 0, s>>>(rp, ci, va, nrows, v1, v2, v3, vp, ep, guard)
  if constexpr (TR) {
    switch (epi) {
      case EPT_RAW: POGS_S(EPT_RAW); break;
      case EPT_TALL_R: POGS_S(EPT_TALL_R); break;
      case EPT_FAT_X: POGS_S(EPT_FAT_X); break;
      case EPT_SK_COL: POGS_S(EPT_SK_COL); break;
      case EPT_REFINE: POGS_S(EPT_REFINE); break;
      case EPT_CG_R: POGS_S(EPT_CG_R); break;
      case EPT_CG_S0: POGS_S(EPT_CG_S0); break;
      case EPT_CG_Q: POGS_S(EPT_CG_Q); break;
      case EPT_CG_S: POGS_S(EPT_CG_S); break;
    }
  } else {
    switch (epi) {
      case EPN_RAW: POGS_S(EPN_RAW); break;
      case EPN_TALL_Y: POGS_S(EPN_TALL_Y); break;
      case EPN_FAT_R: POGS_S(EPN_FAT_R); break;
      case EPN_SK_ROW: POGS_S(EPN_SK_ROW); break;
      case EPN_REFINE: POGS_S(EPN_REFINE); break;
      case EPN_CG_R: POGS_S(EPN_CG_R); break;
      case EPN_CG_S0: POGS_S(EPN_CG_S0); break;
      case EPN_CG_Q: POGS_S(EPN_CG_Q); break;
      case EPN_CG_S: POGS_S(EPN_CG_S); break;
    }
  }
#undef POGS_S
}

template <int NRHS, bool SQ, bool TR, int PK>
void spmv_lanes(int lanes, int epi, const int* rp, const int* ci, const float* va, int nrows, const float* v1,
                const float* v2, const float* v3, const float* vp, int grid, const EpiArgs& ep,
                const DevState* guard, cudaStream_t s) {
  switch (lanes) {
    case 4: spmv_dispatch<NRHS, SQ, TR, 4, PK>(epi, rp, ci, va, nrows, v1, v2, v3, vp, grid, ep, guard, s); break;
    case 8: spmv_dispatch<NRHS, SQ, TR, 8, PK>(epi, rp, ci, va, nrows, v1, v2, v3, vp, grid, ep, guard, s); break;
    case 16: spmv_dispatch<NRHS, SQ, TR, 16, PK>(epi, rp, ci, va, nrows, v1, v2, v3, vp, grid, ep, guard, s); break;
    default: spmv_dispatch<NRHS, SQ, TR, 32, PK>(epi, rp, ci, va, nrows, v1, v2, v3, vp, grid, ep, guard, s); break;
  }
}

template <bool TR>
void spmv_rhs(int nrhs, bool sq, bool pk, int lanes, int epi, const int* rp, const int* ci, const float* va,
              int nrows, const float* v1, const float* v2, const float* v3, const float* vp, int grid,
              const EpiArgs& ep, const DevState* guard, cudaStream_t s) {
  if (nrhs == 3 && pk) spmv_lanes<3, false, TR, 1>(lanes, epi, rp, ci, va, nrows, v1, v2, v3, vp, grid, ep, guard, s);
  else if (nrhs == 3) spmv_lanes<3, false, TR, 0>(lanes, epi, rp, ci, va, nrows, v1, v2, v3, vp, grid, ep, guard, s);
  else if (nrhs == 2 && pk) spmv_lanes<2, false, TR, 1>(lanes, epi, rp, ci, va, nrows, v1, v2, v3, vp, grid, ep, guard, s);
  else if (nrhs == 2) spmv_lanes<2, false, TR, 0>(lanes, epi, rp, ci, va, nrows, v1, v2, v3, vp, grid, ep, guard, s);
  else if (sq) spmv_lanes<1, true, TR, 0>(lanes, epi, rp, ci, va, nrows, v1, v2, v3, vp, grid, ep, guard, s);
  else spmv_lanes<1, false, TR, 0>(lanes, epi, rp, ci, va, nrows, v1, v2, v3, vp, grid, ep, guard, s);
}

}  // namespace

// Lanes per row: 8 lanes already read whole 32-byte sectors of the values and indices, and
// fewer lanes per row give each lane more entries to keep in flight; long rows get more lanes.
int csr_lanes(int64_t rows, int64_t nnz) {
  const double avg = rows > 0 ? (double)nnz / (double)rows : 0.0;
  return avg >= 512 ? 32 : (avg >= 160 ? 16 : (avg >= 6 ? 8 : 4));
}

void csr_geometry(GemvGeom& g, int64_t m, int64_t n, int64_t nnz, int num_sms) {
  g.sparse = 1;
  g.sp_lanes_n = csr_lanes(m, nnz);
  g.sp_lanes_t = csr_lanes(n, nnz);
  g.n_nrowblk = grid_rows(m, 256 / g.sp_lanes_n, num_sms, kSpmvBlocksPerSm);
  g.t_ncolblk = grid_rows(n, 256 / g.sp_lanes_t, num_sms, kSpmvBlocksPerSm);
  g.keep_rows = 0;
  // the dense kernels' partial buffers are not used
  g.t_cols_per_blk = 1024;
  g.t_nsplit = 1;
  g.t_rows = 1;
  g.n_rows = 1;
  g.n_cols = 128;
  g.n_ncolsplit = 1;
}

// The gathered vectors have m entries (column sums) or n (row dots); from kPackMin entries on
// they no longer stay in L1 and two or three right-hand sides are interleaved first.
constexpr int kPackMin = 8192;

bool csr_packs(const GemvGeom& g, bool trans, int nrhs, int m, int n) {
  return g.sparse && g.pack && nrhs >= 2 && (trans ? m : n) >= kPackMin;
}

int csr_pack_launches(const GemvGeom& g, int m, int n) {
  return (csr_packs(g, true, 3, m, n) ? 1 : 0) + (csr_packs(g, false, 2, m, n) ? 1 : 0);
}

void launch_spmv(bool trans, int nrhs, bool sq, int epi, const GemvGeom& g, int m, int n, const float* v1,
                 const float* v2, const float* v3, const EpiArgs& ep, const DevState* guard, cudaStream_t s) {
  const bool pk = csr_packs(g, trans, nrhs, m, n);
  if (pk) {
    const int k = trans ? m : n;
    count_launch();
    if (nrhs == 3) pack_rhs_kernel<3><<<grid_rows(k, 256, 148), 256, 0, s>>>(v1, v2, v3, k, g.pack, guard, ep.cg_done);
    else pack_rhs_kernel<2><<<grid_rows(k, 256, 148), 256, 0, s>>>(v1, v2, v3, k, g.pack, guard, ep.cg_done);
  }
  count_launch();
  if (trans)
    spmv_rhs<true>(nrhs, sq, pk, g.sp_lanes_t, epi, g.rp_t, g.ci_t, g.va_t, n, v1, v2, v3, g.pack, g.t_ncolblk, ep,
                   guard, s);
  else
    spmv_rhs<false>(nrhs, sq, pk, g.sp_lanes_n, epi, g.rp_n, g.ci_n, g.va_n, m, v1, v2, v3, g.pack, g.n_nrowblk, ep,
                    guard, s);
}

void launch_csr_check(const int* rp, const int* ci, const float* va, int64_t m, int64_t n, int64_t nnz, int* err,
                      cudaStream_t s) {
  count_launch();
  csr_check_kernel<<<grid_rows(m, 8, 148), 256, 0, s>>>(rp, ci, va, (int)m, (int)n, nnz, err);
}

int csr_transpose_chunks(int64_t nnz, int64_t n) {
  const int64_t by_table = std::max<int64_t>(1, (int64_t)(64ll << 20) / std::max<int64_t>(n, 1));
  const int64_t by_size = std::max<int64_t>(1, (nnz + 1023) / 1024);
  return (int)std::min<int64_t>(std::min(by_table, by_size), 148 * 32);
}

void launch_csr_transpose(const int* rp, const int* ci, const float* va, int64_t m, int64_t n, int64_t nnz,
                          int nch, int* rowidx, int* cnt, int* tot, int* t_rp, int* t_ci, float* t_va, int* perm,
                          cudaStream_t s) {
  const int64_t chunk = (nnz + nch - 1) / nch;
  const int wgrid = (nch * 32 + 255) / 256;
  count_launch(5);
  csr_rows_kernel<<<grid_rows(m, 8, 148), 256, 0, s>>>(rp, (int)m, rowidx);
  csr_split_kernel<false><<<wgrid, 256, 0, s>>>(ci, va, rowidx, nnz, chunk, nch, (int)n, cnt, nullptr, nullptr,
                                                nullptr, nullptr);
  csr_chunk_offsets_kernel<<<grid_rows(n, 256, 148), 256, 0, s>>>(cnt, nch, (int)n, tot);
  scan_kernel<<<1, 1024, 0, s>>>(tot, (int)n, t_rp);
  csr_split_kernel<true><<<wgrid, 256, 0, s>>>(ci, va, rowidx, nnz, chunk, nch, (int)n, cnt, t_rp, t_ci, t_va,
                                               perm);
}

void launch_csr_scale(const int* rp, const int* ci, float* va, int64_t m, const float* D, const float* E,
                      const int* perm, int64_t nnz, float* t_va, cudaStream_t s) {
  count_launch(2);
  csr_scale_kernel<<<grid_rows(m, 8, 148), 256, 0, s>>>(rp, ci, va, (int)m, D, E);
  gather_kernel<<<grid_rows(nnz, 256, 148), 256, 0, s>>>(va, perm, nnz, t_va);
}

void launch_csr_densify(const int* rp, const int* ci, const float* va, int64_t m, float* A, int64_t lda,
                        cudaStream_t s) {
  count_launch();
  csr_densify_kernel<<<grid_rows(m, 8, 148), 256, 0, s>>>(rp, ci, va, (int)m, A, lda);
}

}  // namespace pogs
