// Indirect projection (Section 3.5): CGLS on the reduced least-squares problem, for matrices
// too large to factor.  With B = [M; I] and b = [top; bot]:
//   tall (M = A^, u = x):   x = argmin ||A^ u - d||^2 + ||u - c||^2,  y = A^ x
//   fat  (M = A^T, u = z):  z = argmin ||A^T u - c||^2 + ||u + d||^2, y = d + z, x = c - A^T z
// (the normal equations of these are the two reduced updates).  CGLS keeps the residual
// r = b - B u = [r_top; r_bot] and s = B^T r; every step applies M and M^T once (the two GEMV
// orientations, with the CGLS epilogues of iter.cu) and the scalar and vector updates below.
// It starts from the previous projection's u (the paper's warm start) and stops when
// ||s|| <= tol ||r|| (LSQR's first stopping test with ||B|| taken as 1, the scale of an
// equilibrated matrix), when ||s|| has grown to 4 times the smallest ||s|| of this projection
// (in FP32, once ||s|| / ||r|| reaches the rounding floor of the matrix-vector products the
// recurrences turn unstable and ||s|| and the error in u grow geometrically), or after
// max_steps.  Once stopped, every later kernel of the projection returns at once (the graph
// keeps a fixed, unrolled sequence of steps).
#include "kernels.h"

namespace pogs {
namespace {

// Sum of k double-float partials (part[stride * i + off]) by one block; result in every thread.
__device__ double sum_parts(const Df* __restrict__ part, int k, int stride, int off, double* sh) {
  Df a = {};
  for (int i = threadIdx.x; i < k; i += blockDim.x) df_add(a, part[(int64_t)stride * i + off]);
  Df v[1] = {a};
  double out[1];
  block_sum_df<1>(v, out, sh);
  __shared__ double b;
  if (threadIdx.x == 0) b = out[0];
  __syncthreads();
  return b;
}

__device__ bool cg_stop_dev(double gamma, double rnorm2, float tol) {
  // square roots in FP32: the test compares two norms to a relative tolerance
  return gamma <= 0.0 || sqrtf((float)gamma) <= tol * sqrtf((float)rnorm2);
}

__global__ void __launch_bounds__(256) cg_start_kernel(CgState* cg, const DevState* st, const Df* r0_part, int nr0,
                                                       const Df* s0_part, int ns0) {
  __shared__ double sh[8];
  if (st && st->done) return;
  const double rt2 = sum_parts(r0_part, nr0, 2, 0, sh);
  const double g0 = sum_parts(s0_part, ns0, 2, 0, sh);
  const double rb2 = sum_parts(s0_part, ns0, 2, 1, sh);
  if (threadIdx.x == 0) {
    cg->gamma = g0;
    cg->pnorm2 = g0;   // p = s
    cg->rnorm2 = rt2 + rb2;
    cg->gmin = g0;
    cg->steps = 0;
    cg->done = (cg->max_steps <= 0 || cg_stop_dev(g0, rt2 + rb2, cg->tol)) ? 1 : 0;
  }
}

__global__ void __launch_bounds__(256) cg_alpha_kernel(const CgState* cg, const DevState* st, const Df* q_part,
                                                       int nq, float* __restrict__ u, float* __restrict__ rt,
                                                       float* __restrict__ rb, const float* __restrict__ p,
                                                       const float* __restrict__ q, int ntop, int nu,
                                                       Df* __restrict__ r_part) {
  __shared__ double sh[8];
  if ((st && st->done) || cg->done) return;
  const double qq = sum_parts(q_part, nq, 2, 0, sh);
  const float alpha = (float)(cg->gamma / (qq + cg->pnorm2));
  Df acc = {};
  const int total = ntop > nu ? ntop : nu;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    if (i < ntop) {
      const float r = rt[i] - alpha * q[i];
      rt[i] = r;
      df_add_prod(acc, r, r);
    }
    if (i < nu) {
      const float pi = p[i];
      u[i] += alpha * pi;
      const float r = rb[i] - alpha * pi;
      rb[i] = r;
      df_add_prod(acc, r, r);
    }
  }
  Df v[1] = {acc};
  double out[1];
  block_sum_df<1>(v, out, sh);
  if (threadIdx.x == 0) {
    const float hi = (float)out[0];
    r_part[2 * blockIdx.x] = Df{hi, (float)(out[0] - (double)hi)};
  }
}

__global__ void __launch_bounds__(256) cg_beta_kernel(CgState* cg, const DevState* st, const Df* s_part, int ns,
                                                      const Df* r_part, int nr, float* __restrict__ p,
                                                      const float* __restrict__ sv, int nu, Df* __restrict__ p_part,
                                                      unsigned* cnt) {
  __shared__ double sh[8];
  if ((st && st->done) || cg->done) return;
  const double gnew = sum_parts(s_part, ns, 2, 0, sh);
  const float beta = (float)(gnew / cg->gamma);
  Df acc = {};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nu; i += gridDim.x * blockDim.x) {
    const float pi = sv[i] + beta * p[i];
    p[i] = pi;
    df_add_prod(acc, pi, pi);
  }
  Df v[1] = {acc};
  double out[1];
  block_sum_df<1>(v, out, sh);
  if (threadIdx.x == 0) {
    const float hi = (float)out[0];
    p_part[2 * blockIdx.x] = Df{hi, (float)(out[0] - (double)hi)};
  }
  // the last block (every block has read gamma) advances the state
  if (!arrive_last(cnt, gridDim.x)) return;
  const double pp = sum_parts(p_part, gridDim.x, 2, 0, sh);
  const double rr = sum_parts(r_part, nr, 2, 0, sh);
  if (threadIdx.x == 0) {
    cg->gamma = gnew;
    cg->pnorm2 = pp;
    cg->rnorm2 = rr;
    cg->steps += 1;
    const bool diverging = gnew > 16.0 * cg->gmin;
    cg->gmin = gnew < cg->gmin ? gnew : cg->gmin;
    cg->done = (cg->steps >= cg->max_steps || diverging || cg_stop_dev(gnew, rr, cg->tol)) ? 1 : 0;
  }
}

__global__ void cg_tall_finish_kernel(int n, float* __restrict__ xt, const float* __restrict__ cx,
                                      const float* __restrict__ x, const DevState* st) {
  if (st && st->done) return;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) xt[j] += cx[j] - x[j];
}

__global__ void cg_fat_finish_kernel(int m, const float* __restrict__ dy, const float* __restrict__ z,
                                     float* __restrict__ y, float* __restrict__ w, float* __restrict__ yt,
                                     const DevState* st) {
  if (st && st->done) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    const float yi = dy[i] + z[i];
    y[i] = yi;
    w[i] = dy[i] - yi;
    yt[i] += dy[i] - yi;
  }
}

int grid_elem(int64_t k) {
  const int64_t g = (k + 255) / 256;
  return (int)(g < 1 ? 1 : (g > 148 * 4 ? 148 * 4 : g));
}

}  // namespace

void launch_cg_start(CgState* cg, const DevState* st, const Df* r0_part, int nr0, const Df* s0_part, int ns0,
                     cudaStream_t s) {
  count_launch();
  cg_start_kernel<<<1, 256, 0, s>>>(cg, st, r0_part, nr0, s0_part, ns0);
}

void launch_cg_alpha(CgState* cg, const DevState* st, const Df* q_part, int nq, float* u, float* rt, float* rb,
                     const float* p, const float* q, int ntop, int nu, Df* r_part, int nblk, cudaStream_t s) {
  count_launch();
  cg_alpha_kernel<<<nblk, 256, 0, s>>>(cg, st, q_part, nq, u, rt, rb, p, q, ntop, nu, r_part);
}

void launch_cg_beta(CgState* cg, const DevState* st, const Df* s_part, int ns, const Df* r_part, int nr,
                    float* p, const float* sv, int nu, Df* p_part, unsigned* cnt, int nblk, cudaStream_t s) {
  count_launch();
  cg_beta_kernel<<<nblk, 256, 0, s>>>(cg, st, s_part, ns, r_part, nr, p, sv, nu, p_part, cnt);
}

void launch_cg_tall_finish(int n, float* xt, const float* cx, const float* x, const DevState* st, cudaStream_t s) {
  count_launch();
  cg_tall_finish_kernel<<<grid_elem(n), 256, 0, s>>>(n, xt, cx, x, st);
}

void launch_cg_fat_finish(int m, const float* dy, const float* z, float* y, float* w, float* yt,
                          const DevState* st, cudaStream_t s) {
  count_launch();
  cg_fat_finish_kernel<<<grid_elem(m), 256, 0, s>>>(m, dy, z, y, w, yt, st);
}

int cg_blocks(int64_t k) { return grid_elem(k); }

}  // namespace pogs
