// FP64 kernels of the outer iteration: real SpMM, tall-skinny products, small dense
// factorisations, Ritz residuals and locking (arXiv 2510.17334, Alg. 2: B-orthonormalisation, Rayleigh-Ritz, locking).
#pragma once

#include "common.cuh"

namespace slrf {

// YA = A X and/or YB = B X for a real row-major block X (n x k).  Either output may be null.
void spmm_real(int64_t n, const int64_t *rowptr, const int32_t *col, const double *valA,
               const double *valB, const double *X, int ldx, int k, double *YA, double *YB, int ldy,
               cudaStream_t st, const int *run_if = nullptr);
// YB = B X in FP32 arithmetic (FP64 storage): input of an FP32 Gram matrix.
void spmm_b32(int64_t n, const int64_t *rowptr, const int32_t *col, const double *valB, const double *X, int ldx,
              int k, double *YB, int ldy, cudaStream_t st);

// YA = A X and YB = B X in FP32 arithmetic (FP64 storage): the start of the FP32 solves.
void spmm_ab32(int64_t n, const int64_t *rowptr, const int32_t *col, const double *valA, const double *valB,
               const double *X, int ldx, int k, double *YA, double *YB, int ldy, cudaStream_t st);
// Jacobi preconditioner D = diag(A): dsc = D^-1/2 (*flag = 1 if a diagonal entry is missing or
// not positive) and the values of D^-1/2 A D^-1/2, D^-1/2 B D^-1/2 on the same pattern.
void jacobi_scaling(int64_t n, const int64_t *rowptr, const int32_t *col, const double *valA, const double *valB,
                    double *dsc, double *valAs, double *valBs, int *flag, cudaStream_t st);
// CSR sanity check before any kernel gathers through a caller's pattern: rowptr[0] = 0,
// non-decreasing, rowptr[n] = nnz, 0 <= col < n; sets *flag = 1 otherwise (grid of blocks x 256).
void validate_csr(int64_t n, int64_t nnz, const int64_t *rowptr, const int32_t *col, int *flag, int blocks,
                  cudaStream_t st);
// One bounded wait that cannot complete (kind 0: grid barrier, 1: mbarrier); sets *err.
// count and err: zeroed device words.
void wait_selftest(int kind, unsigned *count, int *err, cudaStream_t st);
// X[i][:] *= s[i] (row-major n x k, leading dimension ldx).
void row_scale(int64_t n, int k, const double *s, double *X, int ldx, cudaStream_t st);

// R = AV - theta .* BV (column-wise theta), row-major n x k.
void shifted_residual(int64_t n, int k, const double *AV, const double *BV, int ld, const double *theta,
                      double *R, int ldr, cudaStream_t st);

// C (k1 x k2, row-major, ldc) = X^T Y for X (n x k1), Y (n x k2).  sym: X == Y, k1 == k2,
// only upper tiles are computed and mirrored.  work must hold gram_work_doubles(...) doubles.
size_t gram_work_doubles(int64_t n, int k1, int k2);
// fp32: FP32 inputs and accumulation within row chunks (for passes whose error a later
// FP64 pass removes); run_if: device flag, the launch does nothing while *run_if == 0.
void gram(int64_t n, const double *X, int ldx, int k1, const double *Y, int ldy, int k2, double *C, int ldc,
          bool sym, double *work, cudaStream_t st, bool fp32 = false, const int *run_if = nullptr);

// Z = alpha X S + beta Z;  X n x k1, S k1 x k2 (row-major, lds), Z n x k2.  upper: S is
// upper triangular.  Z must not alias X.
void gemm_nn(int64_t n, const double *X, int ldx, int k1, const double *S, int lds, int k2, double *Z, int ldz,
             double alpha, double beta, bool upper, cudaStream_t st);

// G = R^T R (lower Cholesky L = R^T of the symmetric k x k G, using its lower triangle);
// Rinv (k x k row-major, upper) = R^{-1}.  *status is set to SLRF_ECHOL on failure and never
// cleared (device int).  G may be overwritten.  fp32: factor in FP32 (first Cholesky-QR
// pass).  In shared memory when k^2 values fit, else in global memory (FP64).
void chol_inv(int k, double *G, int ldg, double *Rinv, int ldr, int *status, cudaStream_t st,
              const int *run_if = nullptr, bool fp32 = false);

// Symmetric eigen-decomposition of H (k x k) by parallel cyclic Jacobi:
// theta ascending (k), S (k x k row-major, column i = eigenvector i).
struct JacobiWork {
  double *A;        // kk x kk
  double *Vt;       // kk x kk
  double *rot;      // 4 * kk: diagonal and pair entries of the next round, two copies
  int *flags;       // [4]
  unsigned *bar;    // [2] barrier counters
  int *err;         // [1]
};
size_t jacobi_work_doubles(int k);
int jacobi_eig(int k, const double *H, int ldh, double *theta, double *S, int lds, JacobiWork w,
               cudaStream_t st);

// Column statistics of the Ritz block: res = ||AV - theta BV|| / ||AV||,
// res_paper = ||AV - theta BV|| / (theta sqrt(v^T B v)), sgn = sign of the largest |v|.
void ritz_residuals(int64_t n, int k, const double *V, const double *AV, const double *BV, int ld,
                    const double *theta, double *res, double *res_paper, double *sgn, double *work,
                    cudaStream_t st);
size_t ritz_work_doubles(int64_t n, int k);

// Lock / compact decision (one block).  Writes dst_x[c] (>= 0: locked slot), dst_v[c]
// (>= 0: active slot), appends theta/res of locked columns to Theta/Res, writes the
// active theta to theta_act, and updates info[0..3] = {n_conv, n_act, pending, newly}.
void lock_decide(int k, const double *theta, const double *res, double gamma, double tol, int lock,
                 int cap, int *info, int *dst_x, int *dst_v, double *Theta, double *Res, double *theta_act,
                 cudaStream_t st, int *unresolved = nullptr);
// Move columns: V/AV/BV (times sgn) to X/BX (dst_x) or to Vn/AVn/BVn (dst_v).
void lock_gather(int64_t n, int k, const double *V, const double *AV, const double *BV, int ld,
                 const double *sgn, const int *dst_x, const int *dst_v, double *X, double *BX, int ldx,
                 double *Vn, double *AVn, double *BVn, int ldn, cudaStream_t st);

// Gaussian block from a counter-based generator (Philox4x32-10 + Box-Muller).
void gaussian_block(int64_t n, int k, uint64_t seed, double *V, int ld, cudaStream_t st);

// SLRF pole/weight design on the device (one block): writes mp poles and weights.
void design_poles(int m, int mp, double gamma, double alpha, double beta, double band, double2 *sig,
                  double2 *wt, int *status, cudaStream_t st);

// Elementwise helpers.
void copy_block(int64_t n, int k, const double *src, int lds, double *dst, int ldd, cudaStream_t st);
void check_finite(int64_t count, const double *x, int *flag, cudaStream_t st);

}  // namespace slrf
