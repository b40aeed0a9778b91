// COCG kernels for all (pole, column) systems (A - sigma_j B) d = r0 of one filter apply.
#pragma once

#include "common.cuh"

namespace slrf {

// Per-(pole, column) COCG scalars, FP64 in both precisions.
struct WScal {
  double2 alpha;   // step length for the next update
  double2 beta;    // p <- r + beta p for the next SpMM
  double2 rho;     // r^T r (unconjugated)
  double r0n2;     // ||r0||^2
  double rn2;      // ||r||^2 after the last update
  int active;      // 1 while the column still iterates
  int iters;       // updates performed in the current solve
  int brk;         // breakdown flag
  int iters_total; // updates over all refinement steps of the filter apply
};

constexpr int kThreads = 256;  // threads per COCG block (8 warps)
constexpr int kWarps = kThreads / 32;
constexpr int kNQ = 6;         // doubles per partial slot

template <typename R>
struct CocgArgs {
  int64_t n;
  const int64_t *rowptr;
  const int32_t *col;
  const R *valA;
  const R *valB;
  int W;        // complex entries per row: kpad * mp, a multiple of 32 * vec
  int vec;      // complex entries per lane (the tile is 32 vec entries): FP64 1; FP32 2
                // with the plain CSR SpMM, 4 with the grouped one (cocg_vec_csr / _grp)
  int k;        // real columns in the block
  int m;        // poles in use
  int mp;       // poles padded to a power of two (<= 32)
  int rows_per_block;
  int nrb;      // row blocks (gridDim.x)
  cx_t<R> *d;   // correction  (solution = y0 + d)
  cx_t<R> *r;   // residual
  cx_t<R> *p;   // search direction
  cx_t<R> *q;   // (A - sigma B) p
  const cx_t<R> *sig;  // mp poles
  double *partial;     // [nrb][W][kNQ]
  unsigned *counters;  // [ntiles]
  WScal *ws;           // [W]
  double tol2;         // tol_inner^2
  // right-hand side:  r0 = c_w g,  q0 = c_w (A g - sigma B g)  (real FP64 blocks, ld = ldg)
  const double *g, *Ag, *Bg;
  int ldg;
  const double2 *cfac;  // [W] factor c_w
  const double *gscale; // [k] or null: the FP32 path solves for g * gscale (no underflow),
                        // and the pole sum is divided by gscale again
  // accumulation U = coefV .* V + sum_j 2 Re(w_j d_j)
  const double2 *wt;    // mp weights (FP64, zero for padded poles)
  const double *V;
  int ldv;
  const double *coefV;  // [k]
  double *U;
  int ldu;
  // iterative refinement (FP32 path, refine_max >= 2): FP64 correction accumulator
  // D [n][W] in the scaled units of the first step, the FP64 pattern values and poles
  // for the FP64 residual, and ||r0||^2 of the first step per w
  double2 *D64;
  const double *valA64, *valB64;
  const double2 *sig64;
  double *r00;
  int it_cap;  // > 0: a column stops after this many updates (per-problem It_max in a batch)
  // Grouped-row SpMM (G > 1): rows [G g, G g + G) share one sorted union column list.  Record
  // e of group g (gptr[g] <= e < gptr[g + 1]) is grec_bytes<R, G>() bytes: the G rows' A
  // values, then their B values (one value each in the working precision), then the column
  // (int32, at grec_col<R, G>()); zero where a row has no entry.
  // The records of a group reach shared memory by 1-D bulk copies (TMA engine).
  int G;                     // rows per group; 1 = plain CSR
  int64_t ngroups;
  const int64_t *gptr;       // [ngroups + 1]
  const unsigned char *grec; // records, 16-byte aligned
  int bdiag;                 // 1: B-diagonal records (G = 3, see grec_col)
  int *err;                  // 1: a bounded wait gave up (SLRF_ETIMEOUT); 2, 3: group records
                             // inconsistent; 4: update buffers missing (SLRF_EINVAL)
  // Jacobi preconditioner D = diag(A): the value arrays above are those of
  // D^-1/2 A D^-1/2 and D^-1/2 B D^-1/2, g is D^-1/2 g, and dsc[i] = D_ii^-1/2 turns the
  // scaled solutions back (y = D^-1/2 z) in the pole sum; null: no preconditioner
  const double *dsc;
  // kAccU accumulator: [tile][row][32 VEC / mp columns] of R (n x kpad entries)
  void *uacc;
};

// Record of the grouped-row SpMM: 2 G values and the column, rounded up to 16 bytes (G = 3:
// 64 B in FP64, 32 B in FP32).  SLRF_GRP_SPLAT = 1 stores each FP32 value twice (the (a, a)
// operand of the packed FMA ready-made, 64 B records); 0 stores it once and pairs it in
// registers.
#ifndef SLRF_GRP_SPLAT
#define SLRF_GRP_SPLAT 0
#endif
//
// B-diagonal records (BD, 3-row groups only): vector-valued FEM pencils whose B couples a dof
// only with the same dof of a neighbour node (a mass matrix M (x) I_3) have, in a node's group,
// one nonzero B value per column c -- the row c mod 3.  When every group's columns come in
// aligned node triples (3J, 3J + 1, 3J + 2), a record holds the 3 A values, that one B value
// and the column (FP32 32 B, FP64 48 B), and the walk knows the B row from the record's place
// in its triple: one B product per record instead of three.  Checked on the device when the
// records are built (grp_bd_detect); otherwise the general records are kept.
template <typename R, int G, bool BD = false> __host__ __device__ constexpr int grec_col() {
  return BD ? 4 * (int)sizeof(R) : ((sizeof(R) == 8 || SLRF_GRP_SPLAT) ? 16 * G : 8 * G);
}
template <typename R, int G, bool BD = false> __host__ __device__ constexpr int grec_bytes() {
  return (grec_col<R, G, BD>() + 4 + 15) / 16 * 16;
}
inline int grec_bytes_rt(int G, bool fp32, bool bd = false) {
  const int col = bd ? (fp32 ? 16 : 32) : ((!fp32 || SLRF_GRP_SPLAT) ? 16 * G : 8 * G);
  return (col + 4 + 15) / 16 * 16;
}
// Records per staged chunk (one bulk copy): 64 (2 KB of 32-byte FP32 records, 4 KB in FP64).
#ifndef SLRF_GRP_CHUNK32
#define SLRF_GRP_CHUNK32 64
#endif
#ifndef SLRF_GRP_CHUNK64
#define SLRF_GRP_CHUNK64 64
#endif
// B-diagonal records: whole node triples per chunk (a multiple of 3).
#ifndef SLRF_GRP_CHUNK_BD
#define SLRF_GRP_CHUNK_BD 81
#endif
template <typename R, bool BD = false> __host__ __device__ constexpr int grp_chunk() {
  return BD ? SLRF_GRP_CHUNK_BD : (sizeof(R) == 4 ? SLRF_GRP_CHUNK32 : SLRF_GRP_CHUNK64);
}
// Dynamic shared memory of the grouped SpMM: two chunk buffers per warp.
template <typename R, int G, bool BD = false> __host__ __device__ constexpr int grp_smem_bytes() {
  return kWarps * 2 * grp_chunk<R, BD>() * grec_bytes<R, G, BD>();
}

// Final-update modes: how the last COCG update of a solve delivers its correction.
// kAccU: an update of a solve without refinement adds its step to the accumulator (no d
// array); kAccUEnd: the last one, which also writes U.
enum FinalMode {
  kFinalNone = 0, kFinalU = 1, kFinalStoreD = 2, kFinalAddD = 3, kFinalUFromD = 4, kAccU = 5, kAccUEnd = 6
};
// Whether the buffers an update in mode `fm` writes or reads are present (the refinement
// modes need D64, the accumulator modes uacc, the modes that write U need U, V, coefV).
// The launchers skip a launch that fails this and record code 4 in *a.err.
template <typename R> inline bool cocg_mode_ok(const CocgArgs<R> &a, int fm) {
  const bool needs_d64 = fm == kFinalStoreD || fm == kFinalAddD || fm == kFinalUFromD;
  const bool needs_acc = fm == kAccU || fm == kAccUEnd;
  const bool writes_u = fm == kFinalU || fm == kFinalUFromD || fm == kAccUEnd;
  if (fm < kFinalNone || fm > kAccUEnd) return false;
  if (needs_d64 && a.D64 == nullptr) return false;
  if (needs_acc && a.uacc == nullptr) return false;
  if (writes_u && (a.U == nullptr || a.V == nullptr || a.coefV == nullptr)) return false;
  return true;
}

// Launchers (defined in cocg.cu).  All enqueue on `st`.
template <typename R> void cocg_init(const CocgArgs<R> &a, cudaStream_t st);
// update of tiles [tile0, tile0 + ntiles) (ntiles = 0: every tile)
template <typename R> void cocg_update(const CocgArgs<R> &a, bool first, int final_mode, cudaStream_t st,
                                      int tile0 = 0, int ntiles = 0);
// one launch: SpMM of tiles [s0, s0 + ns) and update of tiles [u0, u0 + nu)
template <typename R> void cocg_dual(const CocgArgs<R> &a, int s0, int ns, int u0, int nu, bool first, int fm,
                                    cudaStream_t st);
template <typename R> void cocg_spmm(const CocgArgs<R> &a, cudaStream_t st, bool fresh = false);
// refinement step s >= 2: r = r0 - (A - sigma B) D (FP64), new COCG scalars per w
template <typename R> void cocg_residual(const CocgArgs<R> &a, cudaStream_t st);
// Complex entries per lane (CocgArgs::vec): one 16-byte value in FP64; in FP32 two (one
// 16-byte load) with the plain CSR SpMM and four (two loads) with the grouped-row SpMM,
// whose staged records then serve twice the columns.  Measured on GB300: four entries make
// the grouped SpMM of the 64 x 64 x 32 elasticity box 16 % faster and the plain CSR SpMM of
// the 41^3 Laplacian 20 % slower.
template <typename R> __host__ __device__ constexpr int cocg_vec_csr() { return sizeof(R) == 8 ? 1 : 2; }
template <typename R> __host__ __device__ constexpr int cocg_vec_grp() { return sizeof(R) == 8 ? 1 : 4; }
template <typename R> __host__ __device__ constexpr int cocg_vec_max() { return sizeof(R) == 8 ? 1 : 4; }
// resident blocks per SM the COCG kernels are compiled for (sets their register budget)
#ifndef SLRF_F32_MINB
#define SLRF_F32_MINB 4
#endif
#ifndef SLRF_F32_MINB4
#define SLRF_F32_MINB4 3
#endif
template <typename R, int V> __host__ __device__ constexpr int cocg_minb() {
  return sizeof(R) == 8 ? 4 : (V >= 4 ? SLRF_F32_MINB4 : SLRF_F32_MINB);
}
// Lane width and row length the kernels can use (else the launchers refuse, code 4).
template <typename R> inline bool cocg_layout_ok(const CocgArgs<R> &a) {
  const bool v = sizeof(R) == 8 ? a.vec == 1 : (a.vec == 2 || a.vec == 4);
  return v && a.W > 0 && a.W % (32 * a.vec) == 0;
}

// gscale[c] = 1 / max |g[:, c]| (tmp: k words of scratch)
void col_scale(int64_t n, int k, const double *g, int ld, unsigned long long *tmp, double *gscale, cudaStream_t st);

// Batched launches: one persistent grid over the work items (row block, tile) of P
// problems; args (device, P entries) and prefix (device, P + 1 item offsets).
template <typename R> void cocg_init_batched_launch(const CocgArgs<R> *args, const int *prefix, int P, int total,
                                                    cudaStream_t st);
template <typename R> void cocg_update_batched_launch(const CocgArgs<R> *args, const int *prefix, int P, int total,
                                                      bool first, int fm, cudaStream_t st);
template <typename R> void cocg_spmm_batched_launch(const CocgArgs<R> *args, const int *prefix, int P, int total,
                                                    bool fresh, cudaStream_t st);
template <typename R> void cocg_residual_batched_launch(const CocgArgs<R> *args, const int *prefix, int P, int total,
                                                        cudaStream_t st);

// Raise the dynamic shared-memory limit of the grouped SpMM kernels (once per process;
// call before the first launch and outside stream capture).
void cocg_kernel_attrs();
// Records of the grouped format checked once after the build (columns in [0, n), offsets
// non-decreasing); *flag = 1 otherwise.
template <typename R>
void grp_check(int64_t n, int G, int64_t ngroups, const int64_t *gptr, const unsigned char *rec, int *flag,
               int blocks, cudaStream_t st, bool bd = false);
// B-diagonal records (see grec_col): *flag = 1 unless every group of 3 rows has its records
// in aligned column triples and B vanishes off the row c mod 3 (general records as input).
template <typename R>
void grp_bd_detect(int64_t n, int64_t ngroups, const int64_t *gptr, const unsigned char *rec, int *flag, int blocks,
                   cudaStream_t st);
// General records -> B-diagonal records (nrec of them).
template <typename R>
void grp_bd_convert(int64_t nrec, const unsigned char *rec, unsigned char *bdrec, cudaStream_t st);
// FP64 real products through FP64 B-diagonal records of 3-row groups: YA = A X and/or YB = B X
// (either may be null), X first copied to x64 ([n][grp_real64_ld(k)], padding zero) with row i
// multiplied by xscale[i] (null: 1), output row i by yscale[i] (null: 1).
int grp_real64_ld(int k);
void spmm_grp_real64(int64_t n, int64_t ngroups, const int64_t *gptr, const unsigned char *grec, int *err, int nrb,
                     const double *X, int ldx, int k, const double *xscale, double *x64, double *YA, double *YB,
                     int ldy, const double *yscale, cudaStream_t st);
// Resident blocks per SM of the grouped SpMM of height G (after cocg_kernel_attrs; 0 on error).
int grp_blocks_per_sm(int G, bool fp32, bool bd = false);

// Real products through the FP32 grouped records (G > 1): YA = A X and/or YB = B X (either
// output may be null) for a real FP64 block X of k columns, in FP32 products and sums.  X is
// first copied to x32 in FP32 ([n][grp_real32_ld(k)], padding zero), row i multiplied by
// xscale[i] (null: 1); output row i is multiplied by yscale[i] (null: 1).  The records'
// values are those the records were built from (the Jacobi-scaled ones when the
// preconditioner is on).  nrb row blocks per column tile; *err as for the COCG SpMM.
int grp_real32_ld(int k);
void spmm_grp_real32(int64_t n, int G, int64_t ngroups, const int64_t *gptr, const unsigned char *grec, int *err,
                     int nrb, const double *X, int ldx, int k, const double *xscale, float *x32, double *YA,
                     double *YB, int ldy, const double *yscale, cudaStream_t st, bool bd = false);


// Grouped-row format: cnt[g] = number of distinct columns of rows [G g, G g + G) (grp_count),
// then the records of every group at the offsets gptr (grp_fill, R = float or double).
void grp_count(int64_t n, int G, const int64_t *rowptr, const int32_t *col, int *cnt, cudaStream_t st);
template <typename R>
void grp_fill(int64_t n, int G, const int64_t *rowptr, const int32_t *col, const double *valA, const double *valB,
              const int64_t *gptr, unsigned char *rec, cudaStream_t st);

// prepare per-w factors: warm start c = 1/(sigma_j - theta_c), else 1; coefV = Phi(theta_c)
void cocg_prepare(int W, int k, int m, int mp, const double2 *sig, const double2 *wt,
                  const double *theta, double2 *cfac, double *coefV, WScal *ws, cudaStream_t st);

}  // namespace slrf
