// Adjoint of the eigenpairs with respect to the values of A and B on their pattern.
//
// For a simple eigenpair (lambda, x) of A x = lambda B x with x^T B x = 1, first-order
// perturbation gives d lambda = x^T (dA - lambda dB) x.  Treating every stored entry
// e = (r_e, c_e) as an independent parameter, a loss with gradient g_lambda[i] has
//   dL/dA_e = sum_i g_i x_i[r_e] x_i[c_e],   dL/dB_e = -sum_i g_i lambda_i x_i[r_e] x_i[c_e],
// a sampled dense-dense product (SDDMM) on the pattern: one warp per row, lanes over
// the eigenpair index, one warp reduction per stored entry.
#include <cuda_runtime.h>

#include "../../include/slrf.h"
#include "common.cuh"
#include "dense.cuh"

namespace slrf {

__global__ void __launch_bounds__(256) eig_grad_kernel(int64_t n, const int64_t *__restrict__ rowptr,
                                                       const int32_t *__restrict__ col, int k,
                                                       const double *__restrict__ evals,
                                                       const double *__restrict__ X, int ldx,
                                                       const double *__restrict__ g, double *__restrict__ gA,
                                                       double *__restrict__ gB) {
  extern __shared__ double sh[];  // per warp: 2 * k weights of row r
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t r = (int64_t)blockIdx.x * 8 + warp;
  if (r >= n) return;
  double *wa = sh + (size_t)warp * 2 * k, *wb = wa + k;
  for (int i = lane; i < k; i += 32) {
    const double xr = X[r * ldx + i];
    wa[i] = g[i] * xr;
    wb[i] = g[i] * evals[i] * xr;
  }
  __syncwarp();
  const int64_t rs = rowptr[r], re = rowptr[r + 1];
  for (int64_t e = rs; e < re; ++e) {
    const int64_t c = col[e];
    const double *xc = X + c * ldx;
    double sa = 0.0, sb = 0.0;
    for (int i = lane; i < k; i += 32) {
      const double x = xc[i];
      sa = fma(wa[i], x, sa);
      sb = fma(wb[i], x, sb);
    }
    sa = warp_sum(sa);
    sb = warp_sum(sb);
    if (lane == 0) {
      gA[e] = sa;
      gB[e] = -sb;
    }
  }
}

int eig_grad_values(int64_t n, const int64_t *rowptr, const int32_t *col, int k, const double *evals,
                    const double *X, int ldx, const double *g, double *gA, double *gB, cudaStream_t st) {
  const size_t smem = 8 * 2 * (size_t)k * sizeof(double);
  if (smem > 200 * 1024) return SLRF_EINVAL;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(eig_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  eig_grad_kernel<<<(unsigned)((n + 7) / 8), 256, smem, st>>>(n, rowptr, col, k, evals, X, ldx, g, gA, gB);
  return cudaGetLastError() == cudaSuccess ? SLRF_OK : SLRF_ECUDA;
}

}  // namespace slrf

// ============================================================================== a13
// Eigenvector terms of the adjoint.  For each eigenpair i (columns of n x k row-major
// blocks, leading dimension k) solve the singular, consistent symmetric system
//   (A - lambda_i B) xi_i = b_i,   b_i = -(g_x_i - B x_i (x_i^T g_x_i))   (b_i orthogonal to x_i)
// by MINRES (Paige & Saunders, 1975) on all columns at once, then make xi_i B-orthogonal
// to x_i.  Per column the Lanczos/Givens scalars live on the device; every column keeps
// iterating until its residual estimate phibar <= tol * ||b_i|| or the cap.
namespace slrf {

struct MinresScal {
  double beta, oldb, dbar, epsln, phibar, cs, sn, alfa, beta1;
  double oldeps, delta, gamma, phi;
  int active, iters;
};

constexpr int kAdjRows = 512;

// partial column sums of x .* y over row chunks: work[chunk][k]
__global__ void colprod_partial_kernel(int64_t n, int k, const double *x, const double *y, double *work) {
  const int c = blockIdx.y * blockDim.x + threadIdx.x;
  if (c >= k) return;
  const int64_t r0 = (int64_t)blockIdx.x * kAdjRows;
  const int64_t r1 = r0 + kAdjRows < n ? r0 + kAdjRows : n;
  double s = 0.0;
  for (int64_t i = r0; i < r1; ++i) s = fma(x[i * k + c], y[i * k + c], s);
  work[(size_t)blockIdx.x * k + c] = s;
}
static void colprod(int64_t n, int k, const double *x, const double *y, double *work, cudaStream_t st) {
  dim3 g((unsigned)((n + kAdjRows - 1) / kAdjRows), (k + 127) / 128);
  colprod_partial_kernel<<<g, 128, 0, st>>>(n, k, x, y, work);
}
__device__ __forceinline__ double colprod_final(const double *work, int nch, int k, int c) {
  double s = 0.0;
  for (int z = 0; z < nch; ++z) s += work[(size_t)z * k + c];
  return s;
}

// b = -(g - Bx (x^T g)); x^T g from partials
__global__ void adj_rhs_kernel(int64_t n, int k, const double *g, const double *BX, const double *work, int nch,
                               double *b) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * k) return;
  const int c = (int)(t % k);
  const double xg = colprod_final(work, nch, k, c);
  b[t] = -(g[t] - BX[t] * xg);
}

// init per column: beta1 = ||b||, r1 = r2 = y = b, x = w = w2 = 0
__global__ void minres_init_scal_kernel(int k, const double *work, int nch, MinresScal *s) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= k) return;
  const double b2 = colprod_final(work, nch, k, c);
  MinresScal m{};
  m.beta1 = sqrt(b2);
  m.beta = m.beta1;
  m.oldb = 0.0;
  m.dbar = 0.0;
  m.epsln = 0.0;
  m.phibar = m.beta1;
  m.cs = -1.0;
  m.sn = 0.0;
  m.active = m.beta1 > 0.0 ? 1 : 0;
  m.iters = 0;
  s[c] = m;
}

// v = y / beta (beta of this step), y = A v - lambda B v - (beta / oldb) r1  [with AV, BV of v]
__global__ void minres_v_kernel(int64_t n, int k, const double *y, const MinresScal *s, double *v) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * k) return;
  const int c = (int)(t % k);
  const MinresScal &m = s[c];
  v[t] = (m.active && m.beta > 0.0) ? y[t] / m.beta : 0.0;
}
__global__ void minres_apply_kernel(int64_t n, int k, const double *AV, const double *BV, const double *lam,
                                    const double *r1, const MinresScal *s, double *y) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * k) return;
  const int c = (int)(t % k);
  const MinresScal &m = s[c];
  double val = fma(-lam[c], BV[t], AV[t]);
  if (m.oldb > 0.0) val -= (m.beta / m.oldb) * r1[t];
  y[t] = val;
}
// alfa = v^T y (final of partials) stored per column
__global__ void minres_alfa_kernel(int k, const double *work, int nch, MinresScal *s) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= k) return;
  s[c].alfa = colprod_final(work, nch, k, c);
}
// y -= (alfa/beta) r2; r1 = r2; r2 = y
__global__ void minres_y2_kernel(int64_t n, int k, const MinresScal *s, double *y, double *r1, double *r2) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * k) return;
  const int c = (int)(t % k);
  const MinresScal &m = s[c];
  const double yy = m.beta > 0.0 ? y[t] - (m.alfa / m.beta) * r2[t] : y[t];
  r1[t] = r2[t];
  r2[t] = yy;
  y[t] = yy;
}
// Givens step with beta_new = ||y|| (final of partials); convergence test
__global__ void minres_scal_kernel(int k, const double *work, int nch, double tol, int itn, MinresScal *s) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= k) return;
  MinresScal m = s[c];
  if (!m.active) return;
  const double bnew = sqrt(colprod_final(work, nch, k, c));
  m.oldb = m.beta;
  m.beta = bnew;
  m.oldeps = m.epsln;
  m.delta = m.cs * m.dbar + m.sn * m.alfa;
  const double gbar = m.sn * m.dbar - m.cs * m.alfa;
  m.epsln = m.sn * m.beta;
  m.dbar = -m.cs * m.beta;
  double gam = sqrt(gbar * gbar + m.beta * m.beta);
  if (!(gam > 1e-300)) gam = 1e-300;
  m.gamma = gam;
  m.cs = gbar / gam;
  m.sn = m.beta / gam;
  m.phi = m.cs * m.phibar;
  m.phibar = m.sn * m.phibar;
  m.iters = itn;
  s[c] = m;
}
// w1 = w2; w2 = w; w = (v - oldeps w1 - delta w2)/gamma; x += phi w; then the column stops
// once phibar <= tol beta1 (the state of a stopped column is frozen)
__global__ void minres_w_kernel(int64_t n, int k, const double *v, const MinresScal *s, double *w, double *w2,
                                double *x) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * k) return;
  const int c = (int)(t % k);
  const MinresScal &m = s[c];
  if (!m.active) return;
  const double w1 = w2[t];
  const double wo = w[t];
  const double wn = (v[t] - m.oldeps * w1 - m.delta * wo) / m.gamma;
  w2[t] = wo;
  w[t] = wn;
  x[t] = fma(m.phi, wn, x[t]);
}
__global__ void minres_stop_kernel(int k, double tol, MinresScal *s, int *notconv, int last) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= k) return;
  MinresScal &m = s[c];
  if (m.active && (m.phibar <= tol * m.beta1 || m.beta == 0.0)) m.active = 0;
  if (last && m.active) atomicExch(notconv, 1);
}
__global__ void minres_count_kernel(int k, const MinresScal *s, int *count) {
  int c = 0;
  for (int i = threadIdx.x; i < k; i += blockDim.x) c += s[i].active;
  c = warp_sum(c);
  __shared__ int sh[4];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) *count = sh[0] + sh[1] + sh[2] + sh[3];
}
// xi -= x (x^T B xi); then YA = X diag(a) + Xi, YB = X diag(b) + Xi diag(lambda)
__global__ void adj_finish_kernel(int64_t n, int k, const double *X, const double *xi, const double *work, int nch,
                                  const double *lam, const double *g_eval, const double *work2, double *YA,
                                  double *YB) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * k) return;
  const int c = (int)(t % k);
  const double xbxi = colprod_final(work, nch, k, c);   // x^T B xi
  const double gx = colprod_final(work2, nch, k, c);    // g_x^T x
  const double xv = X[t];
  const double xiv = xi[t] - xv * xbxi;
  YA[t] = g_eval[c] * xv + xiv;
  YB[t] = (g_eval[c] * lam[c] + 0.5 * gx) * xv + lam[c] * xiv;
}

// gA[e] = sum_i YA[r][i] X[c][i], gB[e] = -sum_i YB[r][i] X[c][i]
__global__ void __launch_bounds__(256) eig_grad2_kernel(int64_t n, const int64_t *__restrict__ rowptr,
                                                        const int32_t *__restrict__ col, int k,
                                                        const double *__restrict__ X, const double *__restrict__ YA,
                                                        const double *__restrict__ YB, double *__restrict__ gA,
                                                        double *__restrict__ gB) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t r = (int64_t)blockIdx.x * 8 + warp;
  if (r >= n) return;
  const int64_t rs = rowptr[r], re = rowptr[r + 1];
  for (int64_t e = rs; e < re; ++e) {
    const int64_t c = col[e];
    double sa = 0.0, sb = 0.0;
    for (int i = lane; i < k; i += 32) {
      const double x = X[c * k + i];
      sa = fma(YA[r * k + i], x, sa);
      sb = fma(YB[r * k + i], x, sb);
    }
    sa = warp_sum(sa);
    sb = warp_sum(sb);
    if (lane == 0) {
      gA[e] = sa;
      gB[e] = -sb;
    }
  }
}

struct AdjBuffers {
  double *b, *y, *v, *r1, *r2, *w, *w2, *x, *AV, *BV, *YA, *YB, *work, *work2;
  MinresScal *scal;
  int *flag;
};

// The caller (slrf.cu) provides n x k scratch blocks (X here has leading dimension k).
int eig_grad_vectors(int64_t n, const int64_t *rowptr, const int32_t *col, const double *valA, const double *valB,
                     int k, const double *evals, const double *X, const double *g_eval, const double *g_X,
                     double *gA, double *gB, AdjBuffers bf, int maxit, double tol, int *h_active, int *notconv,
                     cudaStream_t st) {
  const int nch = (int)((n + kAdjRows - 1) / kAdjRows);
  const int64_t tot = n * k;
  const unsigned gb = (unsigned)((tot + 255) / 256);
  // right-hand sides
  spmm_real(n, rowptr, col, valA, valB, X, k, k, nullptr, bf.BV, k, st);
  colprod(n, k, X, g_X, bf.work2, st);  // x^T g
  adj_rhs_kernel<<<gb, 256, 0, st>>>(n, k, g_X, bf.BV, bf.work2, nch, bf.b);
  colprod(n, k, bf.b, bf.b, bf.work, st);
  minres_init_scal_kernel<<<(k + 127) / 128, 128, 0, st>>>(k, bf.work, nch, bf.scal);
  cudaMemcpyAsync(bf.y, bf.b, tot * sizeof(double), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(bf.r1, bf.b, tot * sizeof(double), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(bf.r2, bf.b, tot * sizeof(double), cudaMemcpyDeviceToDevice, st);
  cudaMemsetAsync(bf.x, 0, tot * sizeof(double), st);
  cudaMemsetAsync(bf.w, 0, tot * sizeof(double), st);
  cudaMemsetAsync(bf.w2, 0, tot * sizeof(double), st);
  cudaMemsetAsync(bf.flag, 0, 2 * sizeof(int), st);
  *notconv = 0;
  int itn = 0;
  while (itn < maxit) {
    const int chunk = maxit - itn < 64 ? maxit - itn : 64;
    for (int j = 0; j < chunk; ++j) {
      ++itn;
      minres_v_kernel<<<gb, 256, 0, st>>>(n, k, bf.y, bf.scal, bf.v);
      spmm_real(n, rowptr, col, valA, valB, bf.v, k, k, bf.AV, bf.BV, k, st);
      minres_apply_kernel<<<gb, 256, 0, st>>>(n, k, bf.AV, bf.BV, evals, bf.r1, bf.scal, bf.y);
      colprod(n, k, bf.v, bf.y, bf.work, st);
      minres_alfa_kernel<<<(k + 127) / 128, 128, 0, st>>>(k, bf.work, nch, bf.scal);
      minres_y2_kernel<<<gb, 256, 0, st>>>(n, k, bf.scal, bf.y, bf.r1, bf.r2);
      colprod(n, k, bf.y, bf.y, bf.work, st);
      minres_scal_kernel<<<(k + 127) / 128, 128, 0, st>>>(k, bf.work, nch, tol, itn, bf.scal);
      minres_w_kernel<<<gb, 256, 0, st>>>(n, k, bf.v, bf.scal, bf.w, bf.w2, bf.x);
      minres_stop_kernel<<<(k + 127) / 128, 128, 0, st>>>(k, tol, bf.scal, bf.flag, itn == maxit);
    }
    // how many columns still iterate: stop early when none
    minres_count_kernel<<<1, 128, 0, st>>>(k, bf.scal, bf.flag + 1);
    if (cudaMemcpyAsync(h_active, bf.flag + 1, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return SLRF_ECUDA;
    if (*h_active == 0) break;
  }
  if (maxit > 0 && itn >= maxit && *h_active > 0) *notconv = 1;
  // B-orthogonal projection, then the pattern gradients
  spmm_real(n, rowptr, col, valA, valB, bf.x, k, k, nullptr, bf.BV, k, st);
  colprod(n, k, X, bf.BV, bf.work, st);  // x^T B xi
  adj_finish_kernel<<<gb, 256, 0, st>>>(n, k, X, bf.x, bf.work, nch, evals, g_eval, bf.work2, bf.YA, bf.YB);
  eig_grad2_kernel<<<(unsigned)((n + 7) / 8), 256, 0, st>>>(n, rowptr, col, k, X, bf.YA, bf.YB, gA, gB);
  return cudaGetLastError() == cudaSuccess ? SLRF_OK : SLRF_ECUDA;
}

size_t adj_work_doubles(int64_t n, int k) { return (size_t)((n + kAdjRows - 1) / kAdjRows) * k; }

}  // namespace slrf
