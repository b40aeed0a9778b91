// FP64 kernels of the outer iteration (arXiv 2510.17334, Alg. 2: B-orthonormalisation, Rayleigh-Ritz, locking): real SpMM,
// tall-skinny Gram and GEMM products, Cholesky-QR building blocks, the projected
// symmetric eigenproblem (parallel cyclic Jacobi), Ritz residuals and locking.
// GB300 executes FP64 at about 2 FMA/clock/SM, so these kernels spread the FP64 work over
// all SMs and keep data traffic small; none of them is on the inner COCG loop.
#include "dense.cuh"
#include "../../include/slrf.h"

namespace slrf {

// ------------------------------------------------------------------------------ real SpMM
// One warp per row; each lane owns U columns (lane + 32 u) of a 32U-column group, U chosen
// per call as ceil(k / 32) up to 8, so a block of k <= 256 columns is one group (no group
// that is mostly padding).  A row's CSR chunk is read once per warp; its entries reach the
// lanes from shared memory (FP64: one broadcast load of (a, b) and one of the column instead
// of five register shuffles), and the gathered row's address is one 32 x 32 -> 64-bit
// multiply-add.
constexpr int kSpmmRows = 8;  // warps (rows) per block

template <int U>
__global__ void __launch_bounds__(256) spmm_real_kernel(int64_t n, const int64_t *__restrict__ rowptr,
                                                        const int32_t *__restrict__ col,
                                                        const double *__restrict__ valA,
                                                        const double *__restrict__ valB,
                                                        const double *__restrict__ X, int ldx, int k,
                                                        double *__restrict__ YA, double *__restrict__ YB,
                                                        int ldy, const int *run_if) {
  if (run_if != nullptr && *run_if == 0) return;
  __shared__ double2 s_ab[kSpmmRows][32];
  __shared__ int s_c[kSpmmRows][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t i = (int64_t)blockIdx.x * kSpmmRows + warp;
  if (i >= n) return;  // warp-uniform; only warp-level synchronisation below
  const int c0 = blockIdx.y * (32 * U) + lane;
  const char *const xl = reinterpret_cast<const char *>(X + c0);
  const unsigned row_bytes = (unsigned)ldx * (unsigned)sizeof(double);
  double sa[U], sb[U];
#pragma unroll
  for (int u = 0; u < U; ++u) { sa[u] = 0.0; sb[u] = 0.0; }
  const int64_t rs = rowptr[i], re = rowptr[i + 1];
  for (int64_t e0 = rs; e0 < re; e0 += 32) {
    const int cnt = (int)(re - e0 < 32 ? re - e0 : 32);
    int cl = 0;
    double al = 0, bl = 0;
    if (lane < cnt) {
      cl = col[e0 + lane];
      al = YA ? valA[e0 + lane] : 0.0;
      bl = YB ? valB[e0 + lane] : 0.0;
    }
    __syncwarp();
    s_ab[warp][lane] = make_double2(al, bl);
    s_c[warp][lane] = cl;
    __syncwarp();
#pragma unroll 4
    for (int t = 0; t < cnt; ++t) {
      const int c = s_c[warp][t];
      const double2 ab = s_ab[warp][t];
      const double *xr = reinterpret_cast<const double *>(xl + (unsigned long long)(unsigned)c * row_bytes);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (c0 + 32 * u < k && CHK(40, (long long)c * ldx + c0 + 32 * u, (long long)n * ldx)) {
          const double x = xr[32 * u];
          if (YA) sa[u] = fma(ab.x, x, sa[u]);
          if (YB) sb[u] = fma(ab.y, x, sb[u]);
        }
      }
    }
  }
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int cc = c0 + 32 * u;
    if (cc < k && CHK(41, (long long)i * ldy + cc, (long long)n * ldy)) {
      if (YA) YA[(size_t)i * ldy + cc] = sa[u];
      if (YB) YB[(size_t)i * ldy + cc] = sb[u];
    }
  }
}

// YB = B X with FP32 products and sums (FP64 in and out): for the first Cholesky-QR pass,
// whose Gram matrix is formed in FP32 anyway.  Same work split as spmm_real_kernel; the
// CSR chunk reaches the lanes by two 32-bit shuffles per entry.
template <int U>
__global__ void __launch_bounds__(256) spmm_b32_kernel(int64_t n, const int64_t *__restrict__ rowptr,
                                                       const int32_t *__restrict__ col,
                                                       const double *__restrict__ valB,
                                                       const double *__restrict__ X, int ldx, int k,
                                                       double *__restrict__ YB, int ldy) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * kSpmmRows + (threadIdx.x >> 5);
  if (i >= n) return;
  const int c0 = blockIdx.y * (32 * U) + lane;
  const char *const xl = reinterpret_cast<const char *>(X + c0);
  const unsigned row_bytes = (unsigned)ldx * (unsigned)sizeof(double);
  float sb[U];
#pragma unroll
  for (int u = 0; u < U; ++u) sb[u] = 0.f;
  const int64_t rs = rowptr[i], re = rowptr[i + 1];
  for (int64_t e0 = rs; e0 < re; e0 += 32) {
    const int cnt = (int)(re - e0 < 32 ? re - e0 : 32);
    int cl = 0;
    float bl = 0.f;
    if (lane < cnt) {
      cl = col[e0 + lane];
      bl = (float)valB[e0 + lane];
    }
#pragma unroll 4
    for (int t = 0; t < cnt; ++t) {
      const int c = __shfl_sync(0xffffffffu, cl, t);
      const float b = __shfl_sync(0xffffffffu, bl, t);
      const double *xr = reinterpret_cast<const double *>(xl + (unsigned long long)(unsigned)c * row_bytes);
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (c0 + 32 * u < k) sb[u] = fmaf(b, (float)xr[32 * u], sb[u]);
    }
  }
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int cc = c0 + 32 * u;
    if (cc < k) YB[(size_t)i * ldy + cc] = (double)sb[u];
  }
}

// YA = A X and YB = B X with FP32 products and sums (FP64 in and out; either output may be
// null): the real sweep that starts the complex-FP32 solves (q0 = c (A g - sigma B g) only
// enters FP32 arithmetic).
template <int U>
__global__ void __launch_bounds__(256) spmm_ab32_kernel(int64_t n, const int64_t *__restrict__ rowptr,
                                                        const int32_t *__restrict__ col,
                                                        const double *__restrict__ valA,
                                                        const double *__restrict__ valB,
                                                        const double *__restrict__ X, int ldx, int k,
                                                        double *__restrict__ YA, double *__restrict__ YB, int ldy) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * kSpmmRows + (threadIdx.x >> 5);
  if (i >= n) return;
  const int c0 = blockIdx.y * (32 * U) + lane;
  const char *const xl = reinterpret_cast<const char *>(X + c0);
  const unsigned row_bytes = (unsigned)ldx * (unsigned)sizeof(double);
  float sa[U], sb[U];
#pragma unroll
  for (int u = 0; u < U; ++u) sa[u] = sb[u] = 0.f;
  const int64_t rs = rowptr[i], re = rowptr[i + 1];
  for (int64_t e0 = rs; e0 < re; e0 += 32) {
    const int cnt = (int)(re - e0 < 32 ? re - e0 : 32);
    int cl = 0;
    float al = 0.f, bl = 0.f;
    if (lane < cnt) {
      cl = col[e0 + lane];
      al = (float)valA[e0 + lane];
      bl = (float)valB[e0 + lane];
    }
#pragma unroll 4
    for (int t = 0; t < cnt; ++t) {
      const int c = __shfl_sync(0xffffffffu, cl, t);
      const float a = __shfl_sync(0xffffffffu, al, t);
      const float b = __shfl_sync(0xffffffffu, bl, t);
      const double *xr = reinterpret_cast<const double *>(xl + (unsigned long long)(unsigned)c * row_bytes);
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (c0 + 32 * u < k) {
          const float x = (float)xr[32 * u];
          sa[u] = fmaf(a, x, sa[u]);
          sb[u] = fmaf(b, x, sb[u]);
        }
    }
  }
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int cc = c0 + 32 * u;
    if (cc < k) {
      if (YA) YA[(size_t)i * ldy + cc] = (double)sa[u];
      if (YB) YB[(size_t)i * ldy + cc] = (double)sb[u];
    }
  }
}

static int spmm_lanes(int k) { return std::min(8, (k + 31) / 32); }

void spmm_ab32(int64_t n, const int64_t *rowptr, const int32_t *col, const double *valA, const double *valB,
               const double *X, int ldx, int k, double *YA, double *YB, int ldy, cudaStream_t st) {
  if (n <= 0 || k <= 0) return;
  const int U = spmm_lanes(k);
  dim3 grid((unsigned)((n + kSpmmRows - 1) / kSpmmRows), (unsigned)((k + 32 * U - 1) / (32 * U)));
#define SPMM_AB32(UU) spmm_ab32_kernel<UU><<<grid, 256, 0, st>>>(n, rowptr, col, valA, valB, X, ldx, k, YA, YB, ldy)
  switch (U) {
    case 1: SPMM_AB32(1); break;
    case 2: SPMM_AB32(2); break;
    case 3: SPMM_AB32(3); break;
    case 4: SPMM_AB32(4); break;
    case 5: SPMM_AB32(5); break;
    case 6: SPMM_AB32(6); break;
    case 7: SPMM_AB32(7); break;
    default: SPMM_AB32(8); break;
  }
#undef SPMM_AB32
}

// Jacobi preconditioner: dsc[i] = A_ii^-1/2 (flag = 1 when a diagonal entry is missing or
// not positive), then the scaled values A_ij dsc_i dsc_j and B_ij dsc_i dsc_j.
__global__ void jacobi_diag_kernel(int64_t n, const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                                   const double *__restrict__ valA, double *__restrict__ dsc, int *flag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double d = 0.0;
  for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e)
    if (col[e] == i) d = valA[e];
  if (d > 0.0 && isfinite(d)) {
    dsc[i] = 1.0 / sqrt(d);
  } else {
    dsc[i] = 1.0;
    atomicExch(flag, 1);
  }
}
__global__ void jacobi_values_kernel(int64_t n, const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                                     const double *__restrict__ valA, const double *__restrict__ valB,
                                     const double *__restrict__ dsc, double *__restrict__ valAs,
                                     double *__restrict__ valBs) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (i >= n) return;
  const double di = dsc[i];
  for (int64_t e = rowptr[i] + lane; e < rowptr[i + 1]; e += 32) {
    const double s = di * dsc[col[e]];
    valAs[e] = valA[e] * s;
    valBs[e] = valB[e] * s;
  }
}
void jacobi_scaling(int64_t n, const int64_t *rowptr, const int32_t *col, const double *valA, const double *valB,
                    double *dsc, double *valAs, double *valBs, int *flag, cudaStream_t st) {
  jacobi_diag_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, rowptr, col, valA, dsc, flag);
  jacobi_values_kernel<<<(unsigned)((n + 7) / 8), 256, 0, st>>>(n, rowptr, col, valA, valB, dsc, valAs, valBs);
}
// CSR sanity: rowptr[0] = 0, non-decreasing, rowptr[n] = nnz, 0 <= col < n.  *flag = 1 on failure.
__global__ void validate_csr_kernel(int64_t n, int64_t nnz, const int64_t *rowptr, const int32_t *col, int *flag) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += stride) {
    const int64_t r = rowptr[i];
    if (r < 0 || r > nnz || (i == 0 && r != 0) || (i == n && r != nnz) || (i > 0 && rowptr[i - 1] > r))
      atomicExch(flag, 1);
  }
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride) {
    const int32_t c = col[e];
    if (c < 0 || (int64_t)c >= n) atomicExch(flag, 1);
  }
}
void validate_csr(int64_t n, int64_t nnz, const int64_t *rowptr, const int32_t *col, int *flag, int blocks,
                  cudaStream_t st) {
  validate_csr_kernel<<<blocks, 256, 0, st>>>(n, nnz, rowptr, col, flag);
}

// Diagnostic of the bounded waits (no counterpart in the paper): one wait that cannot
// complete -- kind 0: the grid barrier expecting one more block than the launch has;
// kind 1: an mbarrier phase that nothing arrives at.  Each gives up at its limit, sets
// *err and returns.
__global__ void wait_selftest_kernel(int kind, unsigned *count, int *err) {
  if (kind == 0) {
    GridBarrier gb{count, err};
    unsigned epoch = 0;
    grid_sync(gb, gridDim.x + 1u, epoch);
  } else {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
      mbar_init(&bar, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_wait(&bar, 0, err, 1);
    __syncthreads();
  }
}
void wait_selftest(int kind, unsigned *count, int *err, cudaStream_t st) {
  wait_selftest_kernel<<<1, 32, 0, st>>>(kind, count, err);
}

__global__ void row_scale_kernel(int64_t n, int k, const double *__restrict__ s, double *X, int ldx) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * k) return;
  const int64_t i = t / k;
  if (CHK(42, i * ldx + t % k, n * ldx)) X[i * ldx + t % k] *= s[i];
}
void row_scale(int64_t n, int k, const double *s, double *X, int ldx, cudaStream_t st) {
  const int64_t tot = n * k;
  if (tot <= 0) return;
  row_scale_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, k, s, X, ldx);
}

void spmm_real(int64_t n, const int64_t *rowptr, const int32_t *col, const double *valA, const double *valB,
               const double *X, int ldx, int k, double *YA, double *YB, int ldy, cudaStream_t st,
               const int *run_if) {
  if (n <= 0 || k <= 0) return;
  const int U = spmm_lanes(k);
  dim3 grid((unsigned)((n + kSpmmRows - 1) / kSpmmRows), (unsigned)((k + 32 * U - 1) / (32 * U)));
#define SPMM_REAL(UU) \
  spmm_real_kernel<UU><<<grid, 256, 0, st>>>(n, rowptr, col, valA, valB, X, ldx, k, YA, YB, ldy, run_if)
  switch (U) {
    case 1: SPMM_REAL(1); break;
    case 2: SPMM_REAL(2); break;
    case 3: SPMM_REAL(3); break;
    case 4: SPMM_REAL(4); break;
    case 5: SPMM_REAL(5); break;
    case 6: SPMM_REAL(6); break;
    case 7: SPMM_REAL(7); break;
    default: SPMM_REAL(8); break;
  }
#undef SPMM_REAL
}

void spmm_b32(int64_t n, const int64_t *rowptr, const int32_t *col, const double *valB, const double *X, int ldx,
              int k, double *YB, int ldy, cudaStream_t st) {
  if (n <= 0 || k <= 0) return;
  const int U = spmm_lanes(k);
  dim3 grid((unsigned)((n + kSpmmRows - 1) / kSpmmRows), (unsigned)((k + 32 * U - 1) / (32 * U)));
#define SPMM_B32(UU) spmm_b32_kernel<UU><<<grid, 256, 0, st>>>(n, rowptr, col, valB, X, ldx, k, YB, ldy)
  switch (U) {
    case 1: SPMM_B32(1); break;
    case 2: SPMM_B32(2); break;
    case 3: SPMM_B32(3); break;
    case 4: SPMM_B32(4); break;
    case 5: SPMM_B32(5); break;
    case 6: SPMM_B32(6); break;
    case 7: SPMM_B32(7); break;
    default: SPMM_B32(8); break;
  }
#undef SPMM_B32
}

__global__ void shifted_residual_kernel(int64_t n, int k, const double *AV, const double *BV, int ld,
                                        const double *theta, double *R, int ldr) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * k) return;
  const int64_t i = t / k;
  const int c = (int)(t % k);
  R[i * ldr + c] = fma(-theta[c], BV[i * ld + c], AV[i * ld + c]);
}

void shifted_residual(int64_t n, int k, const double *AV, const double *BV, int ld, const double *theta,
                      double *R, int ldr, cudaStream_t st) {
  const int64_t tot = n * k;
  if (tot <= 0) return;
  shifted_residual_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, k, AV, BV, ld, theta, R, ldr);
}

__global__ void copy_block_kernel(int64_t n, int k, const double *src, int lds, double *dst, int ldd) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * k) return;
  const int64_t i = t / k;
  const int c = (int)(t % k);
  dst[i * ldd + c] = src[i * lds + c];
}

void copy_block(int64_t n, int k, const double *src, int lds, double *dst, int ldd, cudaStream_t st) {
  const int64_t tot = n * k;
  if (tot <= 0) return;
  copy_block_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, k, src, lds, dst, ldd);
}

__global__ void check_finite_kernel(int64_t count, const double *x, int *flag) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(x[t])) { atomicExch(flag, 1); return; }
}

void check_finite(int64_t count, const double *x, int *flag, cudaStream_t st) {
  if (count <= 0) return;
  int blocks = (int)((count + 255) / 256);
  if (blocks > device_sm_count() * 8) blocks = device_sm_count() * 8;
  check_finite_kernel<<<blocks, 256, 0, st>>>(count, x, flag);
}

// ------------------------------------------------------------------------------ Gram
// 64 x 64 output tile per block, 256 threads with a 4 x 4 register tile each; the rows
// are split into gridDim.z chunks whose partial tiles are summed in order by gram_reduce.
constexpr int kGT = 64;
constexpr int kGR = 16;

__global__ void __launch_bounds__(256) gram_partial_kernel(int64_t n, const double *__restrict__ X, int ldx, int k1,
                                                           const double *__restrict__ Y, int ldy, int k2,
                                                           int64_t rows_per_chunk, bool sym,
                                                           double *__restrict__ work, const int *run_if) {
  if (run_if != nullptr && *run_if == 0) return;
  const int ti = blockIdx.x, tj = blockIdx.y, z = blockIdx.z;
  if (sym && ti > tj) return;
  __shared__ double xs[kGR][kGT];
  __shared__ double ys[kGR][kGT];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4] = {};
  const int64_t r0 = (int64_t)z * rows_per_chunk;
  const int64_t r1 = (r0 + rows_per_chunk < n) ? r0 + rows_per_chunk : n;
  for (int64_t rr = r0; rr < r1; rr += kGR) {
    for (int t = threadIdx.x; t < kGR * kGT; t += 256) {
      const int lr = t / kGT, lc = t % kGT;
      const int64_t row = rr + lr;
      const int cx = ti * kGT + lc, cy = tj * kGT + lc;
      xs[lr][lc] = (row < r1 && cx < k1) ? X[row * ldx + cx] : 0.0;
      ys[lr][lc] = (row < r1 && cy < k2) ? Y[row * ldy + cy] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int lr = 0; lr < kGR; ++lr) {
      double a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) { a[u] = xs[lr][ty * 4 + u]; b[u] = ys[lr][tx * 4 + u]; }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
  double *out = work + (size_t)z * k1 * k2;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int i = ti * kGT + ty * 4 + u, j = tj * kGT + tx * 4 + v;
      if (i < k1 && j < k2) out[(size_t)i * k2 + j] = acc[u][v];
    }
}

// The same product with FP32 inputs and FP32 accumulation inside each row chunk (chunk
// partials are summed in FP64): a Gram accurate to ~1e-6 relative, used where a later
// FP64 pass removes its error (first Cholesky-QR pass, first CGS pass).
__global__ void __launch_bounds__(256) gram32_partial_kernel(int64_t n, const double *__restrict__ X, int ldx, int k1,
                                                             const double *__restrict__ Y, int ldy, int k2,
                                                             int64_t rows_per_chunk, bool sym,
                                                             double *__restrict__ work, const int *run_if) {
  if (run_if != nullptr && *run_if == 0) return;
  const int ti = blockIdx.x, tj = blockIdx.y, z = blockIdx.z;
  if (sym && ti > tj) return;
  __shared__ float xs[kGR][kGT];
  __shared__ float ys[kGR][kGT];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[4][4] = {};
  const int64_t r0 = (int64_t)z * rows_per_chunk;
  const int64_t r1 = (r0 + rows_per_chunk < n) ? r0 + rows_per_chunk : n;
  for (int64_t rr = r0; rr < r1; rr += kGR) {
    for (int t = threadIdx.x; t < kGR * kGT; t += 256) {
      const int lr = t / kGT, lc = t % kGT;
      const int64_t row = rr + lr;
      const int cx = ti * kGT + lc, cy = tj * kGT + lc;
      xs[lr][lc] = (row < r1 && cx < k1) ? (float)X[row * ldx + cx] : 0.0f;
      ys[lr][lc] = (row < r1 && cy < k2) ? (float)Y[row * ldy + cy] : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int lr = 0; lr < kGR; ++lr) {
      float a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) { a[u] = xs[lr][ty * 4 + u]; b[u] = ys[lr][tx * 4 + u]; }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
  double *out = work + (size_t)z * k1 * k2;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int i = ti * kGT + ty * 4 + u, j = tj * kGT + tx * 4 + v;
      if (i < k1 && j < k2) out[(size_t)i * k2 + j] = (double)acc[u][v];
    }
}

__global__ void gram_reduce_kernel(int k1, int k2, int nz, bool sym, const double *work, double *C, int ldc,
                                   const int *run_if) {
  if (run_if != nullptr && *run_if == 0) return;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)k1 * k2) return;
  int i = (int)(t / k2), j = (int)(t % k2);
  int si = i, sj = j;
  if (sym && i > j) { si = j; sj = i; }  // the lower triangle mirrors the upper one
  double s = 0.0;
  for (int z = 0; z < nz; ++z) s += work[(size_t)z * k1 * k2 + (size_t)si * k2 + sj];
  C[(size_t)i * ldc + j] = s;
}

static int gram_chunks(int64_t n, int k1, int k2) {
  const int tiles = ((k1 + kGT - 1) / kGT) * ((k2 + kGT - 1) / kGT);
  int nz = (2 * device_sm_count() + tiles - 1) / tiles;
  const int64_t maxz = (n + 255) / 256;
  if (nz > maxz) nz = (int)maxz;
  if (nz < 1) nz = 1;
  if (nz > 64) nz = 64;
  return nz;
}

size_t gram_work_doubles(int64_t n, int k1, int k2) { return (size_t)gram_chunks(n, k1, k2) * k1 * k2; }

void gram(int64_t n, const double *X, int ldx, int k1, const double *Y, int ldy, int k2, double *C, int ldc,
          bool sym, double *work, cudaStream_t st, bool fp32, const int *run_if) {
  if (k1 <= 0 || k2 <= 0) return;
  const int nz = gram_chunks(n, k1, k2);
  const int64_t rpc = (n + nz - 1) / nz;
  dim3 grid((k1 + kGT - 1) / kGT, (k2 + kGT - 1) / kGT, nz);
  if (fp32) gram32_partial_kernel<<<grid, 256, 0, st>>>(n, X, ldx, k1, Y, ldy, k2, rpc, sym, work, run_if);
  else gram_partial_kernel<<<grid, 256, 0, st>>>(n, X, ldx, k1, Y, ldy, k2, rpc, sym, work, run_if);
  const int64_t tot = (int64_t)k1 * k2;
  gram_reduce_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(k1, k2, nz, sym, work, C, ldc, run_if);
}

// ------------------------------------------------------------------------------ GEMM
__global__ void __launch_bounds__(256) gemm_nn_kernel(int64_t n, const double *__restrict__ X, int ldx, int k1,
                                                      const double *__restrict__ S, int lds, int k2,
                                                      double *__restrict__ Z, int ldz, double alpha, double beta,
                                                      bool upper) {
  __shared__ double xs[kGT][kGR + 1];
  __shared__ double ss[kGR][kGT];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t r0 = (int64_t)blockIdx.x * kGT;
  const int c0 = blockIdx.y * kGT;
  double acc[4][4] = {};
  int kend = k1;
  if (upper && c0 + kGT < kend) kend = c0 + kGT;  // S[i][j] = 0 for i > j
  for (int kk = 0; kk < kend; kk += kGR) {
    for (int t = threadIdx.x; t < kGT * kGR; t += 256) {
      const int lr = t / kGR, lc = t % kGR;
      const int64_t row = r0 + lr;
      xs[lr][lc] = (row < n && kk + lc < k1) ? X[row * ldx + kk + lc] : 0.0;
    }
    for (int t = threadIdx.x; t < kGR * kGT; t += 256) {
      const int lr = t / kGT, lc = t % kGT;
      ss[lr][lc] = (kk + lr < k1 && c0 + lc < k2) ? S[(size_t)(kk + lr) * lds + c0 + lc] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int l = 0; l < kGR; ++l) {
      double a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) { a[u] = xs[ty * 4 + u][l]; b[u] = ss[l][tx * 4 + u]; }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int64_t row = r0 + ty * 4 + u;
    if (row >= n) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int c = c0 + tx * 4 + v;
      if (c < k2) {
        double* zp = Z + row * ldz + c;
        *zp = (beta == 0.0) ? alpha * acc[u][v] : fma(alpha, acc[u][v], beta * *zp);
      }
    }
  }
}

void gemm_nn(int64_t n, const double *X, int ldx, int k1, const double *S, int lds, int k2, double *Z, int ldz,
             double alpha, double beta, bool upper, cudaStream_t st) {
  if (n <= 0 || k2 <= 0) return;
  dim3 grid((unsigned)((n + kGT - 1) / kGT), (k2 + kGT - 1) / kGT);
  gemm_nn_kernel<<<grid, 256, 0, st>>>(n, X, ldx, k1, S, lds, k2, Z, ldz, alpha, beta, upper);
}

// ------------------------------------------------------------------------------ Cholesky
// One block of 1024 threads.  Right-looking Cholesky on the lower triangle of G (in
// place), then the columns of L^{-1} by forward substitution (one warp per column),
// stored transposed as R^{-1} = (L^{-1})^T.
__global__ void __launch_bounds__(1024) chol_inv_kernel(int k, double *G, int ldg, double *Rinv, int ldr,
                                                        int *status, const int *run_if) {
  if (run_if != nullptr && *run_if == 0) return;
  __shared__ int fail;
  __shared__ double colj[512];  // column j of L below the diagonal (k <= 512)
  if (threadIdx.x == 0) fail = 0;
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    if (threadIdx.x == 0) {
      const double d = G[(size_t)j * ldg + j];
      if (!(d > 0.0) || !isfinite(d)) fail = 1;
      else G[(size_t)j * ldg + j] = sqrt(d);
    }
    __syncthreads();
    if (fail) break;
    const double piv = G[(size_t)j * ldg + j];
    for (int i = j + 1 + threadIdx.x; i < k; i += blockDim.x) {
      const double lij = G[(size_t)i * ldg + j] / piv;
      G[(size_t)i * ldg + j] = lij;
      colj[i] = lij;
    }
    __syncthreads();
    // trailing update of the lower triangle: G[i][l] -= L[i][j] L[l][j], j < l <= i
    {
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
      for (int i = j + 1 + warp; i < k; i += nw) {
        const double lij = colj[i];
        for (int l = j + 1 + lane; l <= i; l += 32) G[(size_t)i * ldg + l] -= lij * colj[l];
      }
    }
    __syncthreads();
  }
  if (fail) {
    if (threadIdx.x == 0) *status = SLRF_ECHOL;
    return;
  }
  // columns of L^{-1}: L x = e_c  (x_i = 0 for i < c)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = warp; c < k; c += nw) {
    // x stored in Rinv row c (R^{-1}[c][i] = x_i)
    double *x = Rinv + (size_t)c * ldr;
    for (int i = lane; i < c; i += 32) x[i] = 0.0;
    if (lane == 0) x[c] = 1.0 / G[(size_t)c * ldg + c];
    __syncwarp();
    for (int i = c + 1; i < k; ++i) {
      double s = 0.0;
      for (int l = c + lane; l < i; l += 32) s = fma(G[(size_t)i * ldg + l], x[l], s);
      s = warp_sum(s);
      if (lane == 0) x[i] = -s / G[(size_t)i * ldg + i];
      __syncwarp();
    }
  }
  __syncthreads();
  // Rinv row c holds column c of L^{-1}: Rinv[c][i] = Linv[i][c] = (R^{-1})[c][i] with R = L^T.
  // *status is only ever raised (a failure of an earlier pass must survive).
}

// The same factorisation with the k x k matrix held in shared memory (k^2 + 3k values of T):
// L in the lower triangle, then X = L^{-1} computed row by row in place, X[i][c] (i > c)
// stored at [c][i] and its diagonal 1/L[i][i] in pvi.  Row i of X:  X[i][c] = -(sum_{c <= l < i}
// L[i][l] X[l][c]) / L[i][i].  With T = float it serves the first Cholesky-QR pass, whose
// Gram matrix is only FP32-accurate anyway.
template <typename T>
__global__ void __launch_bounds__(1024) chol_inv_smem_kernel(int k, const double *__restrict__ G, int ldg,
                                                             double *__restrict__ Rinv, int ldr, int *status,
                                                             const int *run_if) {
  if (run_if != nullptr && *run_if == 0) return;
  extern __shared__ __align__(16) unsigned char chol_smem[];
  T *A = reinterpret_cast<T *>(chol_smem);
  T *colj = A + (size_t)k * k;  // column j of L, contiguous (rows of A are k apart: a column
                                // read by consecutive lanes would hit one shared-memory bank)
  T *pv = colj + k;             // pivots L[j][j]
  T *pvi = pv + k;              // 1 / L[j][j] (= X[j][j])
  __shared__ int fail;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  for (int e = tid; e < k * k; e += nt) {
    const int i = e / k, j = e % k;
    A[e] = j <= i ? (T)G[(size_t)i * ldg + j] : T(0);
  }
  // each pivot's square root and reciprocal are taken once, by the thread whose update
  // produced it (FP64 sqrt and division are many FP64-pipe operations on this GPU)
  auto take_pivot = [&](int j, T d) {
    if (!(d > T(0)) || !isfinite((double)d)) fail = 1;
    else { const T r = sqrt(d); pv[j] = r; pvi[j] = T(1) / r; }
  };
  if (tid == 0) fail = 0;
  __syncthreads();
  if (tid == 0) take_pivot(0, A[0]);
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    if (fail) break;
    const T ip = pvi[j];
    for (int i = j + 1 + tid; i < k; i += nt) {
      const T lij = A[i * k + j] * ip;
      A[i * k + j] = lij;
      colj[i] = lij;
    }
    __syncthreads();
    if (tid == 0) A[j * k + j] = pv[j];
    for (int i = j + 1 + warp; i < k; i += nw) {
      const T lij = colj[i];
      for (int l = j + 1 + lane; l <= i; l += 32) {
        const T v = A[i * k + l] - lij * colj[l];
        A[i * k + l] = v;
        if (i == j + 1 && l == j + 1) take_pivot(j + 1, v);
      }
    }
    __syncthreads();
  }
  if (fail) {
    if (tid == 0) *status = SLRF_ECHOL;  // only ever raised
    return;
  }
  // X = L^{-1} row by row: X[i][c] = -(sum_{c <= l < i} L[i][l] X[l][c]) / L[i][i], stored at [c][i]
  for (int i = 1; i < k; ++i) {
    for (int c = warp; c < i; c += nw) {
      T sum = T(0);
      for (int l = c + lane; l < i; l += 32) sum += A[i * k + l] * (l == c ? pvi[c] : A[c * k + l]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
      if (lane == 0) A[c * k + i] = -sum * pvi[i];
    }
    __syncthreads();
  }
  // Rinv[c][i] = X[i][c] (upper triangular)
  for (int e = tid; e < k * k; e += nt) {
    const int c = e / k, i = e % k;
    Rinv[(size_t)c * ldr + i] = i < c ? 0.0 : (double)(i == c ? pvi[c] : A[c * k + i]);
  }
}

constexpr size_t kCholSmemMax = 220 * 1024;

// Blocked Cholesky and inverse over many CTAs.  GB300 runs FP64 at 2 FMA/clock/SM, so the
// k^3/3 + k^3/6 FMAs of one factorisation and inverse need many SMs once k reaches a few
// hundred (k = 480: 18 ms on one SM).  Panels of kCb columns:
//   chol_panel_kernel: every CTA factors the diagonal block D = G[j0.., j0..] itself (a
//     32 x 32 problem in shared memory), then the rows [j1 + 32 blockIdx.x, +32) of the
//     panel below: L[i][j0 + c] = (G[i][j0 + c] - sum_{l < c} L[i][j0 + l] D[c][l]) / D[c][c];
//   chol_syrk_kernel: the trailing lower triangle G[i][l] -= sum_c L[i][j0 + c] L[l][j0 + c],
//     one CTA per 32 x 32 tile (i >= l);
//   tri_inv_kernel: X = L^{-1} by blocks of kCi columns (one CTA each), rows in blocks of kCi:
//     X[I][C] = L[I][I]^{-1} (E[I][C] - L[I][<I] X[<I][C]), stored as R^{-1}[c][i] = X[i][c].
// A pivot that is not positive (or not finite) raises *status (SLRF_ECHOL); every kernel
// returns at once when *status is already raised or *run_if is zero.
constexpr int kCb = 32;
constexpr int kCi = 8;
#ifndef SLRF_CHOL_BLOCKED_MIN
#define SLRF_CHOL_BLOCKED_MIN 96
#endif
constexpr int kCholBlockedMin = SLRF_CHOL_BLOCKED_MIN;  // smallest k for the blocked kernels
__device__ __forceinline__ bool chol_skip(const int *status, const int *run_if) {
  return (run_if != nullptr && *run_if == 0) || *reinterpret_cast<const volatile int *>(status) != 0;
}
__global__ void __launch_bounds__(256) chol_panel_kernel(int k, double *G, int ldg, int j0, int *status,
                                                         const int *run_if) {
  if (chol_skip(status, run_if)) return;
  __shared__ double D[kCb][kCb + 1];
  __shared__ int fail;
  const int b = min(kCb, k - j0);
  const int tid = threadIdx.x;
  if (tid == 0) fail = 0;
  for (int e = tid; e < kCb * kCb; e += blockDim.x) {
    const int i = e / kCb, l = e % kCb;
    D[i][l] = (i < b && l <= i) ? G[(size_t)(j0 + i) * ldg + j0 + l] : 0.0;
  }
  __syncthreads();
  // unblocked right-looking factorisation of D by warp 0 (lane i owns row i)
  if (tid < 32) {
    const int i = tid;
    for (int j = 0; j < b; ++j) {
      if (i == j) {
        const double d = D[j][j];
        if (!(d > 0.0) || !isfinite(d)) fail = 1;
        D[j][j] = (d > 0.0 && isfinite(d)) ? sqrt(d) : 1.0;
      }
      __syncwarp();
      if (i > j && i < b) D[i][j] /= D[j][j];
      __syncwarp();
      if (i > j && i < b)
        for (int l = j + 1; l <= i; ++l) D[i][l] -= D[i][j] * D[l][j];
      __syncwarp();
    }
  }
  __syncthreads();
  if (fail) {
    if (blockIdx.x == 0 && tid == 0) atomicExch(status, SLRF_ECHOL);
    return;
  }
  if (blockIdx.x == 0)
    for (int e = tid; e < b * b; e += blockDim.x) {
      const int i = e / b, l = e % b;
      if (l <= i) G[(size_t)(j0 + i) * ldg + j0 + l] = D[i][l];
    }
  // panel rows of this CTA: forward substitution with D^T, one row per thread
  const int j1 = j0 + b;
  const int r = j1 + (int)blockIdx.x * kCb + tid;
  if (tid < kCb && r < k) {
    double x[kCb];
    double *row = G + (size_t)r * ldg + j0;
#pragma unroll
    for (int c = 0; c < kCb; ++c) x[c] = c < b ? row[c] : 0.0;
#pragma unroll
    for (int c = 0; c < kCb; ++c) {
      if (c < b) {
        double v = x[c];
#pragma unroll
        for (int l = 0; l < c; ++l) v -= x[l] * D[c][l];
        x[c] = v / D[c][c];
      }
    }
#pragma unroll
    for (int c = 0; c < kCb; ++c)
      if (c < b) row[c] = x[c];
  }
}
__global__ void __launch_bounds__(256) chol_syrk_kernel(int k, double *G, int ldg, int j0, int b, int *status,
                                                        const int *run_if) {
  if (chol_skip(status, run_if)) return;
  // tile (ti, tj), ti >= tj, from the linear block index
  int t = (int)blockIdx.x, ti = 0;
  while (t > ti) { t -= ti + 1; ++ti; }
  const int tj = t;
  const int j1 = j0 + b;
  const int i0 = j1 + ti * 32, l0 = j1 + tj * 32;
  __shared__ double Pi[32][kCb + 1], Pl[32][kCb + 1];
  for (int e = threadIdx.x; e < 32 * kCb; e += blockDim.x) {
    const int rr = e / kCb, c = e % kCb;
    Pi[rr][c] = (i0 + rr < k && c < b) ? G[(size_t)(i0 + rr) * ldg + j0 + c] : 0.0;
    Pl[rr][c] = (l0 + rr < k && c < b) ? G[(size_t)(l0 + rr) * ldg + j0 + c] : 0.0;
  }
  __syncthreads();
  // thread: row i0 + (tid / 8), columns l0 + (tid % 8) + 8 u
  const int ri = threadIdx.x >> 3, cl = threadIdx.x & 7;
  const int i = i0 + ri;
  if (i >= k) return;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int lc = cl + 8 * u, l = l0 + lc;
    if (l > i || l >= k) continue;
    double s = 0.0;
#pragma unroll 8
    for (int c = 0; c < kCb; ++c) s = fma(Pi[ri][c], Pl[lc][c], s);
    G[(size_t)i * ldg + l] -= s;
  }
}
__global__ void __launch_bounds__(256) tri_inv_kernel(int k, const double *G, int ldg, double *Rinv, int ldr,
                                                      int *status, const int *run_if) {
  if (chol_skip(status, run_if)) return;
  extern __shared__ __align__(16) unsigned char tri_smem[];
  double *X = reinterpret_cast<double *>(tri_smem);  // [k][kCi]: X[i][cc], column c0 + cc
  const int c0 = (int)blockIdx.x * kCi;
  const int tid = threadIdx.x;
  const int nt = blockDim.x;
  for (int e = tid; e < k * kCi; e += nt) X[e] = 0.0;
  __syncthreads();
  // thread -> (row ri of the row block, column cc); kCi x kCi outputs, split sums over 4 lanes
  const int cc = tid % kCi, ri = (tid / kCi) % kCi, part = tid / (kCi * kCi);
  constexpr int kParts = 256 / (kCi * kCi);
  __shared__ double S[kParts][kCi][kCi];
  __shared__ double Ld[kCi][kCi + 1];  // the row block's diagonal block of L
  for (int i0 = c0; i0 < k; i0 += kCi) {
    const int bi = min(kCi, k - i0);
    // S = L[I][c0 .. i0) X[c0 .. i0)[C]  (independent loads: several in flight per thread)
    double s = 0.0;
    const int i = i0 + ri;
    if (ri < bi) {
      const double *gi = G + (size_t)i * ldg;
#pragma unroll 4
      for (int l = c0 + part; l < i0; l += kParts) s = fma(gi[l], X[(size_t)l * kCi + cc], s);
    }
    S[part][ri][cc] = s;
    if (tid < kCi * kCi) {
      const int a = tid / kCi, b = tid % kCi;
      Ld[a][b] = (a < bi && b <= a) ? G[(size_t)(i0 + a) * ldg + i0 + b] : 0.0;
    }
    __syncthreads();
    // forward substitution inside the block (one thread per column)
    if (tid < kCi) {
      const int c = tid, col = c0 + c;
      for (int rr = 0; rr < bi; ++rr) {
        const int row = i0 + rr;
        double v = row == col ? 1.0 : 0.0;
#pragma unroll
        for (int q = 0; q < kParts; ++q) v -= S[q][rr][c];
        for (int l = 0; l < rr; ++l) v -= Ld[rr][l] * X[(size_t)(i0 + l) * kCi + c];
        X[(size_t)row * kCi + c] = row < col ? 0.0 : v / Ld[rr][rr];
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < kCi * k; e += nt) {
    const int c = e / k, i = e % k, col = c0 + c;
    if (col < k) Rinv[(size_t)col * ldr + i] = i < col ? 0.0 : X[(size_t)i * kCi + c];
  }
}
static void chol_inv_blocked(int k, double *G, int ldg, double *Rinv, int ldr, int *status, cudaStream_t st,
                             const int *run_if) {
  for (int j0 = 0; j0 < k; j0 += kCb) {
    const int b = std::min(kCb, k - j0);
    const int rest = k - j0 - b;
    const int pb = std::max(1, (rest + kCb - 1) / kCb);
    chol_panel_kernel<<<pb, 256, 0, st>>>(k, G, ldg, j0, status, run_if);
    if (rest > 0) {
      const int T = (rest + 31) / 32;
      chol_syrk_kernel<<<T * (T + 1) / 2, 256, 0, st>>>(k, G, ldg, j0, b, status, run_if);
    }
  }
  const size_t smem = (size_t)k * kCi * sizeof(double);
  tri_inv_kernel<<<(k + kCi - 1) / kCi, 256, smem, st>>>(k, G, ldg, Rinv, ldr, status, run_if);
}

void chol_inv(int k, double *G, int ldg, double *Rinv, int ldr, int *status, cudaStream_t st, const int *run_if,
              bool fp32) {
  static bool attrs = false;
  if (!attrs) {
    cudaFuncSetAttribute(chol_inv_smem_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCholSmemMax);
    cudaFuncSetAttribute(chol_inv_smem_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCholSmemMax);
    attrs = true;
  }
  const size_t b64 = ((size_t)k * k + 3 * k) * sizeof(double), b32 = ((size_t)k * k + 3 * k) * sizeof(float);
  if (k >= kCholBlockedMin && (size_t)k * kCi * sizeof(double) <= kCholSmemMax) {
    static bool tri_attr = false;
    if (!tri_attr) {
      cudaFuncSetAttribute(tri_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCholSmemMax);
      tri_attr = true;
    }
    chol_inv_blocked(k, G, ldg, Rinv, ldr, status, st, run_if);
  } else if (fp32 && b32 <= kCholSmemMax)
    chol_inv_smem_kernel<float><<<1, 1024, b32, st>>>(k, G, ldg, Rinv, ldr, status, run_if);
  else if (b64 <= kCholSmemMax)
    chol_inv_smem_kernel<double><<<1, 1024, b64, st>>>(k, G, ldg, Rinv, ldr, status, run_if);
  else
    chol_inv_kernel<<<1, 1024, 0, st>>>(k, G, ldg, Rinv, ldr, status, run_if);
}

// ------------------------------------------------------------------------------ Jacobi
// Two-sided cyclic Jacobi with the round-robin (circle) ordering, which makes the kk/2
// rotations of one round disjoint.  One block per pair: every block computes all rotations
// of the round (cheap 2x2 problems), then rewrites the rows p, q of J^T A J and of V^T for
// its own pair; one grid barrier per round.  The rotation inputs of a round (a_pp, a_qq,
// a_pq of every pair) are not read from A, whose rows the owning blocks rewrite during the
// round, but from a small table that the owners of the previous round filled (two copies,
// alternating by round), and the block's own rows load together with them: a round costs
// one L2 round trip, the rotation arithmetic and the barrier.  The sweep loop stops once
// every off-diagonal met in a sweep is below 1e-8 of its diagonal scale (quadratic
// convergence leaves them at rounding level after that sweep).
__device__ __forceinline__ void rr_pair(int kk, int r, int b, int &p, int &q) {
  const int M = kk - 1;
  int a0, a1;
  if (b == 0) { a0 = r; a1 = kk - 1; }
  else { a0 = (r + b) % M; a1 = (r - b + M) % M; }
  p = a0 < a1 ? a0 : a1;
  q = a0 < a1 ? a1 : a0;
}
__device__ __forceinline__ int rr_partner(int kk, int r, int x) {
  const int M = kk - 1;
  if (x == kk - 1) return r;
  if (x == r) return kk - 1;
  return ((2 * r - x) % M + M) % M;
}

// Rotation (c, s) that annihilates a_pq: t = tan(phi) is the smaller root of
// t^2 + 2 tau t - 1 = 0 with tau = (a_qq - a_pp) / (2 a_pq), written as
// t = sgn(th) ph / (|th| + sqrt(th^2 + ph^2)) with th = a_qq - a_pp, ph = 2 a_pq
// (t = 1 when th = 0), then c = 1 / sqrt(1 + t^2), s = t c.
__device__ __forceinline__ void jacobi_rotation(double app, double aqq, double apq, double &c, double &sn) {
  const double th = aqq - app, ph = 2.0 * apq;
  double t;
  if (fmax(fabs(th), fabs(ph)) < 1e150) {
    const double num = th > 0.0 ? ph : (th < 0.0 ? -ph : fabs(ph));
    t = num / (fabs(th) + sqrt(th * th + ph * ph));
  } else {  // squares would overflow
    const double tau = th / ph;
    t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
  }
  c = rsqrt(1.0 + t * t);
  sn = t * c;
}

constexpr int kJacobiThreads = 128;
constexpr int kJacobiPer = 512 / kJacobiThreads;  // row entries per thread (kk <= 512)

__global__ void __launch_bounds__(kJacobiThreads) jacobi_kernel(int k, int kk, const double *H, int ldh,
                                                                double *theta, double *S, int lds, JacobiWork w,
                                                                int max_sweeps) {
  const unsigned nb = gridDim.x;  // == kk / 2: block b owns pair b of every round
  GridBarrier gb{w.bar, w.err};
  unsigned epoch = 0;
  double *A = w.A, *Vt = w.Vt;
  double *const rdiag = w.rot, *const roff = w.rot + 2 * kk;  // [2][kk] each
  // init: A = H (padded), Vt = I
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)kk * kk;
       t += (int64_t)nb * blockDim.x) {
    const int i = (int)(t / kk), j = (int)(t % kk);
    const double h = (i < k && j < k) ? H[(size_t)i * ldh + j] : 0.0;
    A[t] = h;
    Vt[t] = (i == j) ? 1.0 : 0.0;
    // the round-0 table: diagonal, and a_pq of every round-0 pair (p < q) at index p
    if (i == j) rdiag[i] = h;
    else if (i < j && rr_partner(kk, 0, i) == j) roff[i] = h;
  }
  if (!grid_sync(gb, nb, epoch)) return;
  __shared__ double rp[512], rq[512];  // rows p, q of A
  __shared__ double cs[512][2];        // rotation (c, s) of every index for this round
  const int b0 = blockIdx.x;
  int par = 0;  // table copy of the current round
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    // has this thread met |a_pq| >= 1e-8 sqrt(|a_pp a_qq|) this sweep?  (identical in every
    // block, since every block computes every rotation)
    int unconv = 0;
    for (int r = 0; r < kk - 1; ++r) {
      int p, q;
      rr_pair(kk, r, b0, p, q);
      // this block's rows of A and V^T, in flight while the rotation inputs load
      double ap[kJacobiPer], aq[kJacobiPer], vp[kJacobiPer], vq[kJacobiPer];
#pragma unroll
      for (int u = 0; u < kJacobiPer; ++u) {
        const int x = threadIdx.x + u * kJacobiThreads;
        if (x < kk) {
          ap[u] = __ldcg(&A[(size_t)p * kk + x]);
          aq[u] = __ldcg(&A[(size_t)q * kk + x]);
          vp[u] = __ldcg(&Vt[(size_t)p * kk + x]);
          vq[u] = __ldcg(&Vt[(size_t)q * kk + x]);
        }
      }
      // every block computes every rotation of the round (kk/2 independent 2x2 problems),
      // so no barrier is needed between the rotation and the update phase
      for (int b = threadIdx.x; b < kk / 2; b += blockDim.x) {
        int pb, qb;
        rr_pair(kk, r, b, pb, qb);
        const double app = __ldcg(&rdiag[par * kk + pb]), aqq = __ldcg(&rdiag[par * kk + qb]),
                     apq = __ldcg(&roff[par * kk + pb]);
        const double a2 = apq * apq, sc2 = fabs(app * aqq);
        unconv |= (apq != 0.0 && a2 >= 1e-16 * sc2);
        double c = 1.0, sn = 0.0;
        if (apq != 0.0 && a2 > 1e-30 * sc2) jacobi_rotation(app, aqq, apq, c, sn);
        cs[pb][0] = c; cs[pb][1] = sn;
        cs[qb][0] = c; cs[qb][1] = sn;
      }
#pragma unroll
      for (int u = 0; u < kJacobiPer; ++u) {
        const int x = threadIdx.x + u * kJacobiThreads;
        if (x < kk) { rp[x] = ap[u]; rq[x] = aq[u]; }
      }
      __syncthreads();
      const double c = cs[p][0], sn = cs[p][1];
      // next round: partners of p and q, and the table copy it reads
      const int r1 = r + 1 < kk - 1 ? r + 1 : 0, nxt = par ^ 1;
      const int pn = rr_partner(kk, r1, p), qn = rr_partner(kk, r1, q);
#pragma unroll
      for (int u = 0; u < kJacobiPer; ++u) {
        const int x = threadIdx.x + u * kJacobiThreads;
        if (x < kk) {
          const int y = rr_partner(kk, r, x);
          const double c2 = cs[x][0], s2 = cs[x][1];
          const bool first = x < y;  // the smaller index is p of its pair
          // (A J)[row][x] for rows p and q
          double ajp, ajq;
          if (first) { ajp = c2 * rp[x] - s2 * rp[y]; ajq = c2 * rq[x] - s2 * rq[y]; }
          else { ajp = s2 * rp[y] + c2 * rp[x]; ajq = s2 * rq[y] + c2 * rq[x]; }
          double np = c * ajp - sn * ajq, nq = sn * ajp + c * ajq;
          if (x == q) np = 0.0;  // annihilated entry
          if (x == p) nq = 0.0;
          A[(size_t)p * kk + x] = np;
          A[(size_t)q * kk + x] = nq;
          Vt[(size_t)p * kk + x] = c * vp[u] - sn * vq[u];
          Vt[(size_t)q * kk + x] = sn * vp[u] + c * vq[u];
          if (x == p) rdiag[nxt * kk + p] = np;
          if (x == q) rdiag[nxt * kk + q] = nq;
          if (x == pn && p < pn) roff[nxt * kk + p] = np;
          if (x == qn && q < qn) roff[nxt * kk + q] = nq;
        }
      }
      par = nxt;
      if (!grid_sync(gb, nb, epoch)) return;
    }
    if (!__syncthreads_or(unconv)) break;
  }
  // sort ascending (stable by index) and write theta, S (column i = eigenvector i)
  if (blockIdx.x == 0) {
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
      const double di = __ldcg(&A[(size_t)i * kk + i]);
      int rank = 0;
      for (int j = 0; j < k; ++j) {
        const double dj = __ldcg(&A[(size_t)j * kk + j]);
        rank += (dj < di) || (dj == di && j < i);
      }
      theta[rank] = di;
      for (int x = 0; x < k; ++x) S[(size_t)x * lds + rank] = __ldcg(&Vt[(size_t)i * kk + x]);
    }
  }
}

size_t jacobi_work_doubles(int k) {
  const int kk = k + (k & 1);
  return 2 * (size_t)kk * kk + 4 * (size_t)kk;
}

int jacobi_eig(int k, const double *H, int ldh, double *theta, double *S, int lds, JacobiWork w, cudaStream_t st) {
  int kk = k + (k & 1);
  if (kk < 2) kk = 2;
  if (kk > 512) return SLRF_EINVAL;
  int dev = 0, per_sm = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_kernel, kJacobiThreads, 0);
  const int nb = kk / 2;  // one block per rotation pair, all co-resident
  if (per_sm < 1 || nb > per_sm * sms) return SLRF_ECUDA;
  cudaMemsetAsync(w.bar, 0, sizeof(unsigned), st);
  cudaMemsetAsync(w.err, 0, sizeof(int), st);
  int max_sweeps = 40;
  void *args[] = {&k, &kk, (void *)&H, &ldh, &theta, &S, &lds, &w, &max_sweeps};
  cudaError_t e = cudaLaunchCooperativeKernel((void *)jacobi_kernel, dim3(nb), dim3(kJacobiThreads), args, 0, st);
  return e == cudaSuccess ? SLRF_OK : SLRF_ECUDA;
}

// ------------------------------------------------------------------------------ residuals
// Per column c over rows: s0 = sum (AV - theta BV)^2, s1 = sum AV^2, s2 = sum V BV,
// and (max |V|, its row, its sign) for the sign convention.  Partials per row chunk.
constexpr int kRRows = 512;

__global__ void ritz_partial_kernel(int64_t n, int k, const double *V, const double *AV, const double *BV, int ld,
                                    const double *theta, double *work) {
  const int c = blockIdx.y * blockDim.x + threadIdx.x;
  if (c >= k) return;
  const int64_t r0 = (int64_t)blockIdx.x * kRRows;
  const int64_t r1 = (r0 + kRRows < n) ? r0 + kRRows : n;
  const double th = theta[c];
  double s0 = 0, s1 = 0, s2 = 0, amax = -1.0, sgn = 1.0, arow = 0;
  for (int64_t i = r0; i < r1; ++i) {
    const double av = AV[i * ld + c], bv = BV[i * ld + c], v = V[i * ld + c];
    const double rr = fma(-th, bv, av);
    s0 = fma(rr, rr, s0);
    s1 = fma(av, av, s1);
    s2 = fma(v, bv, s2);
    if (fabs(v) > amax) { amax = fabs(v); sgn = v < 0 ? -1.0 : 1.0; arow = (double)i; }
  }
  double *o = work + ((size_t)blockIdx.x * k + c) * 6;
  o[0] = s0; o[1] = s1; o[2] = s2; o[3] = amax; o[4] = sgn; o[5] = arow;
}

__global__ void ritz_final_kernel(int k, int nchunks, const double *theta, const double *work, double *res,
                                  double *res_paper, double *sgn) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= k) return;
  double s0 = 0, s1 = 0, s2 = 0, amax = -1.0, sg = 1.0;
  for (int z = 0; z < nchunks; ++z) {
    const double *o = work + ((size_t)z * k + c) * 6;
    s0 += o[0]; s1 += o[1]; s2 += o[2];
    if (o[3] > amax) { amax = o[3]; sg = o[4]; }  // strict: the first row wins ties
  }
  const double rn = sqrt(s0);
  res[c] = s1 > 0 ? rn / sqrt(s1) : INFINITY;
  if (res_paper) res_paper[c] = (s2 > 0 && theta[c] != 0) ? rn / (fabs(theta[c]) * sqrt(s2)) : INFINITY;
  if (sgn) sgn[c] = sg;
}

size_t ritz_work_doubles(int64_t n, int k) { return (size_t)((n + kRRows - 1) / kRRows) * k * 6; }

void ritz_residuals(int64_t n, int k, const double *V, const double *AV, const double *BV, int ld,
                    const double *theta, double *res, double *res_paper, double *sgn, double *work, cudaStream_t st) {
  if (k <= 0) return;
  const int nchunks = (int)((n + kRRows - 1) / kRRows);
  dim3 grid(nchunks, (k + 127) / 128);
  ritz_partial_kernel<<<grid, 128, 0, st>>>(n, k, V, AV, BV, ld, theta, work);
  ritz_final_kernel<<<(k + 127) / 128, 128, 0, st>>>(k, nchunks, theta, work, res, res_paper, sgn);
}

// ------------------------------------------------------------------------------ locking
__global__ void lock_decide_kernel(int k, const double *theta, const double *res, double gamma, double tol,
                                   int lock, int cap, int *info, int *dst_x, int *dst_v, double *Theta,
                                   double *Res, double *theta_act, int *unresolved) {
  if (threadIdx.x != 0) return;
  int n_conv = info[0];
  int newly = 0, nact = 0, pending = 0;
  double low_th = INFINITY, low_res = 0.0;  // lowest active Ritz pair
  for (int c = 0; c < k; ++c) {
    const double th = theta[c];
    const bool conv = (res[c] <= tol) && (th > 0.0) && (th <= gamma);
    if (!(lock && conv) && th < low_th) { low_th = th; low_res = res[c]; }
    if (lock && conv) {
      const int slot = n_conv + newly;
      dst_x[c] = slot < cap ? slot : -1;
      dst_v[c] = -1;
      if (slot < cap) { Theta[slot] = th; Res[slot] = res[c]; }
      ++newly;
    } else {
      dst_x[c] = -1;
      dst_v[c] = nact;
      theta_act[nact] = th;
      ++nact;
      if (lock) {
        if (th <= gamma) pending = 1;
      } else if (th > 0.0 && th <= gamma && !conv) {
        pending = 1;
      }
    }
  }
  // with locking, the stop test counts only once the subspace resolves the spectrum next
  // to gamma: the lowest active Ritz pair has a relative residual <= 1e-2
  const bool unres = lock && nact > 0 && !(low_res <= 1e-2);
  if (unres) pending = 1;
  if (unresolved != nullptr) *unresolved = unres ? 1 : 0;
  info[0] = n_conv + newly;
  info[1] = nact;
  info[2] = pending;
  info[3] = newly;
}

void lock_decide(int k, const double *theta, const double *res, double gamma, double tol, int lock, int cap,
                 int *info, int *dst_x, int *dst_v, double *Theta, double *Res, double *theta_act, cudaStream_t st,
                 int *unresolved) {
  lock_decide_kernel<<<1, 32, 0, st>>>(k, theta, res, gamma, tol, lock, cap, info, dst_x, dst_v, Theta, Res,
                                       theta_act, unresolved);
}

__global__ void lock_gather_kernel(int64_t n, int k, const double *V, const double *AV, const double *BV, int ld,
                                   const double *sgn, const int *dst_x, const int *dst_v, double *X, double *BX,
                                   int ldx, double *Vn, double *AVn, double *BVn, int ldn) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * k) return;
  const int64_t i = t / k;
  const int c = (int)(t % k);
  const double s = sgn[c];
  const int dx = dst_x[c], dv = dst_v[c];
  if (dx >= 0) {
    X[i * ldx + dx] = s * V[i * ld + c];
    BX[i * ldx + dx] = s * BV[i * ld + c];
  } else if (dv >= 0) {
    Vn[i * ldn + dv] = s * V[i * ld + c];
    AVn[i * ldn + dv] = s * AV[i * ld + c];
    BVn[i * ldn + dv] = s * BV[i * ld + c];
  }
}

void lock_gather(int64_t n, int k, const double *V, const double *AV, const double *BV, int ld, const double *sgn,
                 const int *dst_x, const int *dst_v, double *X, double *BX, int ldx, double *Vn, double *AVn,
                 double *BVn, int ldn, cudaStream_t st) {
  const int64_t tot = n * k;
  if (tot <= 0) return;
  lock_gather_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, k, V, AV, BV, ld, sgn, dst_x, dst_v, X, BX,
                                                                    ldx, Vn, AVn, BVn, ldn);
}

// ------------------------------------------------------------------------------ RNG
// Philox4x32-10 (Salmon et al., SC'11) keyed by the seed, counter = element index,
// and Box-Muller on two 32-bit uniforms -> one standard normal per element.
__device__ __forceinline__ void philox10(uint32_t ctr[4], uint32_t key[2]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  for (int r = 0; r < 10; ++r) {
    const uint32_t h0 = __umulhi(M0, ctr[0]), l0 = M0 * ctr[0];
    const uint32_t h1 = __umulhi(M1, ctr[2]), l1 = M1 * ctr[2];
    const uint32_t n0 = h1 ^ ctr[1] ^ key[0], n2 = h0 ^ ctr[3] ^ key[1];
    ctr[0] = n0; ctr[1] = l1; ctr[2] = n2; ctr[3] = l0;
    key[0] += W0; key[1] += W1;
  }
}

__global__ void gaussian_kernel(int64_t n, int k, uint64_t seed, double *V, int ld) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * k) return;
  uint32_t ctr[4] = {(uint32_t)t, (uint32_t)(t >> 32), 0u, 0u};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  philox10(ctr, key);
  const double u1 = ((double)ctr[0] + 1.0) / 4294967297.0;  // (0, 1)
  const double u2 = (double)ctr[1] / 4294967296.0;
  const double z = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
  V[(t / k) * ld + (t % k)] = z;
}

void gaussian_block(int64_t n, int k, uint64_t seed, double *V, int ld, cudaStream_t st) {
  const int64_t tot = n * k;
  if (tot <= 0) return;
  gaussian_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, k, seed, V, ld);
}

// ------------------------------------------------------------------------------ poles
// sigma_j = gamma x_j (1 + alpha i), x_j = (j - 1/2)/m; weights minimise
// sum_t (Phi(t) - 1[t <= gamma])^2 + beta ||w/gamma||^2 on 3000 uniform samples of (0, 1]
// and 3000 geometric samples of [band, 51] (normalised axis), via the normal equations.
__global__ void __launch_bounds__(256) design_poles_kernel(int m, int mp, double gamma, double alpha, double beta,
                                                           double band, double2 *sig, double2 *wt, int *status) {
  __shared__ double Nm[64][65];
  __shared__ double rhs[64];
  __shared__ double2 sh[32];
  constexpr int kCh = 16;            // samples per chunk
  __shared__ double Gs[kCh][65];     // design rows of one chunk (+ target in column n2)
  const int n2 = 2 * m, nc = n2 + 1;
  const int nin = 3000, nout = 3000;
  if (threadIdx.x < m) {
    const double x = (threadIdx.x + 0.5) / m;
    sh[threadIdx.x] = make_double2(x, alpha * x);
  }
  // design matrix column a at sample t:  a < m: 2 Re C_a(t); a >= m: -2 Im C_{a-m}(t); column
  // n2 is the target (1 in the pass band, 0 in the stop band).  Each thread owns the entries
  // e = threadIdx.x + 256 q of the n2 x (n2 + 1) normal equations and sums them over the
  // samples in order.
  double acc[17];
#pragma unroll
  for (int q = 0; q < 17; ++q) acc[q] = 0.0;
  const int nent = n2 * nc;
  for (int t0 = 0; t0 < nin + nout; t0 += kCh) {
    __syncthreads();
    for (int e = threadIdx.x; e < kCh * nc; e += blockDim.x) {
      const int tl = e / nc, a = e % nc, t = t0 + tl;
      double v = 0.0;
      if (t < nin + nout) {
        double tt, f;
        if (t < nin) { tt = (t + 0.5) / nin; f = 1.0; }
        else { tt = band * pow(51.0 / band, (double)(t - nin) / (nout - 1)); f = 0.0; }
        if (a == n2) v = f;
        else {
          const int ja = a < m ? a : a - m;
          const double dr = tt - sh[ja].x, di = -sh[ja].y;  // t - sigma
          const double den = dr * dr + di * di;
          v = a < m ? 2.0 * dr / den : 2.0 * di / den;
        }
      }
      Gs[tl][a] = v;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 17; ++q) {
      const int e = threadIdx.x + 256 * q;
      if (e < nent) {
        const int a = e / nc, b = e % nc;
        double s = acc[q];
        for (int tl = 0; tl < kCh; ++tl) s = fma(Gs[tl][a], Gs[tl][b], s);
        acc[q] = s;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 17; ++q) {
    const int e = threadIdx.x + 256 * q;
    if (e < nent) {
      const int a = e / nc, b = e % nc;
      if (b == n2) rhs[a] = acc[q];
      else Nm[a][b] = acc[q] + (a == b ? beta : 0.0);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // Cholesky solve of the SPD normal equations
    int ok = 1;
    for (int j = 0; j < n2 && ok; ++j) {
      double d = Nm[j][j];
      for (int l = 0; l < j; ++l) d -= Nm[j][l] * Nm[j][l];
      if (!(d > 0)) { ok = 0; break; }
      Nm[j][j] = sqrt(d);
      for (int i = j + 1; i < n2; ++i) {
        double s = Nm[i][j];
        for (int l = 0; l < j; ++l) s -= Nm[i][l] * Nm[j][l];
        Nm[i][j] = s / Nm[j][j];
      }
    }
    if (ok) {
      double y[64];
      for (int i = 0; i < n2; ++i) {
        double s = rhs[i];
        for (int l = 0; l < i; ++l) s -= Nm[i][l] * y[l];
        y[i] = s / Nm[i][i];
      }
      for (int i = n2 - 1; i >= 0; --i) {
        double s = y[i];
        for (int l = i + 1; l < n2; ++l) s -= Nm[l][i] * y[l];
        y[i] = s / Nm[i][i];
      }
      for (int j = 0; j < mp; ++j) {
        if (j < m) {
          sig[j] = make_double2(gamma * sh[j].x, gamma * sh[j].y);
          wt[j] = make_double2(gamma * y[j], gamma * y[m + j]);
        } else {
          sig[j] = make_double2(gamma, gamma);  // padding pole: never active, weight 0
          wt[j] = make_double2(0.0, 0.0);
        }
      }
    }
    *status = ok ? 0 : SLRF_EINVAL;
  }
}

void design_poles(int m, int mp, double gamma, double alpha, double beta, double band, double2 *sig, double2 *wt,
                  int *status, cudaStream_t st) {
  design_poles_kernel<<<1, 256, 0, st>>>(m, mp, gamma, alpha, beta, band, sig, wt, status);
}

}  // namespace slrf
