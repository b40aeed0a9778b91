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
