// FP64-accurate tall-skinny products on the bf16 tensor cores (tcgen05 + TMEM), by the
// Ozaki splitting.  These are the Gram and projection products of the B-orthonormalisation
// and Rayleigh-Ritz steps of Alg. 2 (arXiv 2510.17334): X^T B U, U^T B U, U^T A U, U R^{-1}, U S.
//
// Splitting.  Every operand row i (the index that survives the product) gets an exponent
// E_i with |x| < 2^E_i over the row; x 2^(56-E_i), rounded to an integer, is written in 7
// balanced base-256 digits d_0..d_6 (d_0 in [0, 256], the others in [-128, 127]) and stored
// as bf16 values D_s = d_s 2^(-8s), which are exact.  Then x = 2^(E_i - 8) sum_s D_s up to
// 2^-56 |max_i|, and x y = 2^(E_a + F_b - 16) sum_{s,t} D_s E_t.
//
// Exactness.  The products D_s E_t of level l = s + t are integers times 2^(-8l); summed over
// 128 rows (one chunk) every level l <= 4 stays below 2^24 units, so the FP32 tensor-core
// accumulation of each such level is exact.  Levels 5 and 6 share one accumulator (their
// weight is below 2^-40 of the leading term); levels above 6 are dropped (below 2^-56).
// Chunk results of the exact levels are combined in 64-bit integers, so the per-block sums
// are exact and deterministic; blocks of rows are summed in FP64 in a fixed order.
#pragma once

#include "common.cuh"

namespace slrf {

// Bytes of device workspace that oz_gram / oz_gemm need for operands up to n x k1, n x k2
// (and k1 x k2 for the small factor of oz_gemm).
size_t oz_work_bytes(int64_t n, int k1, int k2);

// C (k1 x k2, row-major, ldc) = X^T Y for X (n x k1, ldx), Y (n x k2, ldy), all FP64.
// sym: C is symmetric (k1 == k2, e.g. X^T B X with Y = B X); only tiles touching the upper
// triangle are computed and the lower triangle mirrors the upper one.  run_if: device flag, no work while *run_if == 0.
// work: work_bytes >= oz_work_bytes(n, k1, k2) of device memory; a call whose layout does not
// fit sets *err and does nothing.  err: device int, set nonzero if an internal wait ran out
// or the workspace is too small (never in normal use).
void oz_gram(int64_t n, const double *X, int ldx, int k1, const double *Y, int ldy, int k2, double *C, int ldc,
             bool sym, void *work, size_t work_bytes, int *err, cudaStream_t st, const int *run_if = nullptr);

// Z (n x k2, ldz) = alpha X S + beta Z for X (n x k1, ldx), S (k1 x k2, row-major, lds).
// k1 <= 512.  Z must not alias X.
void oz_gemm(int64_t n, const double *X, int ldx, int k1, const double *S, int lds, int k2, double *Z, int ldz,
             double alpha, double beta, void *work, size_t work_bytes, int *err, cudaStream_t st);

}  // namespace slrf
