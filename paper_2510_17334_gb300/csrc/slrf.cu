// C ABI and host orchestration of the enhanced ParaSLRF (arXiv 2510.17334, Alg. 2) on one GPU.
//
// The paper's two parallel levels (poles across process groups, each solve across the
// processes of a group; Sec. 2.1) become one grid: every (pole, column) system of a
// filter apply is in flight in the same COCG launches, and the paper's sum-reduce of
// the Y_j (the filter sum of Alg. 2) is the in-register pole sum of the last COCG update.
// The host drives the outer loop; the only device->host transfer per outer iteration is
// a handful of integers for the lock decision (the locking step of Alg. 2).
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "../../include/slrf.h"
#include "cocg.cuh"
#include "dense.cuh"
#include "ozaki.cuh"

using namespace slrf;

namespace slrf {
int eig_grad_values(int64_t n, const int64_t *rowptr, const int32_t *col, int k, const double *evals,
                    const double *X, int ldx, const double *g, double *gA, double *gB, cudaStream_t st);
struct MinresScal;
struct AdjBuffers {
  double *b, *y, *v, *r1, *r2, *w, *w2, *x, *AV, *BV, *YA, *YB, *work, *work2;
  MinresScal *scal;
  int *flag;
};
int eig_grad_vectors(int64_t n, const int64_t *rowptr, const int32_t *col, const double *valA, const double *valB,
                     int k, const double *evals, const double *X, const double *g_eval, const double *g_X,
                     double *gA, double *gB, AdjBuffers bf, int maxit, double tol, int *h_active, int *notconv,
                     cudaStream_t st);
size_t adj_work_doubles(int64_t n, int k);
}

struct slrf_ctx {
  int status = SLRF_OK;  // sticky
  cudaStream_t st = nullptr;   // library stream (all work, graph capture)
  cudaStream_t ust = nullptr;  // caller's stream (NULL = legacy default stream)
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  int dev = 0;
  int64_t n = 0, nnz = 0;
  double gamma = 0;
  int L = 0;
  slrf_opts o{};
  int m = 0, mp = 0;
  bool mixed = false;
  // matrices (library copies, padded)
  int64_t *rowptr = nullptr;
  int32_t *col = nullptr;
  double *valA = nullptr, *valB = nullptr;
  float *valA32 = nullptr, *valB32 = nullptr;  // FP32 copies of the values the COCG uses
  // Jacobi preconditioner (opts.precond): D^-1/2 per row and the scaled FP64 values the
  // COCG and its starting sweep use (valA / valB stay the pencil's own values)
  double *dsc = nullptr, *valAs = nullptr, *valBs = nullptr;
  // grouped-row format of the COCG SpMM (grp > 1 rows per group)
  int grp = 1;
  int64_t ngroups = 0;
  int64_t *gptr = nullptr;
  unsigned char *grec = nullptr;
  int sm_count = 0;  // multiprocessors of the device (grid sizing), queried at setup
  // pole table
  double2 *sig = nullptr, *wt = nullptr;
  float2 *sig32 = nullptr;
  double h_sig[64] = {}, h_wt[64] = {};
  // COCG working set
  int vec = 1;
  size_t Wmax = 0;
  void *cd = nullptr, *cr = nullptr, *cp = nullptr, *cq = nullptr;
  double *partial = nullptr;
  unsigned *counters = nullptr;
  WScal *ws = nullptr;
  double2 *cfac = nullptr;
  double *coefV = nullptr;
  double *gscale = nullptr;          // FP32 path: per-column right-hand-side scale
  unsigned long long *gmax = nullptr;
  double2 *D64 = nullptr;            // FP32 path with refinement: FP64 correction [n][Wmax]
  double *uacc = nullptr;            // filter accumulator of the updates without refinement [n][Wmax/mp]
  float *x32 = nullptr;              // FP32 copy of a real block for the grouped real SpMM [n][ld32(L)]
  double *dsqrt = nullptr;           // D^1/2 (Jacobi preconditioner): unscaled products from scaled records
  double *r00 = nullptr;             // ||r0||^2 of the first refinement step, per w
  int last_k = 0, last_W = 0;
  int64_t launches = 0;              // kernels enqueued by the orchestration (statistics)
  int64_t rpb_tuned = 0;             // autotuned COCG rows per block (0 = default)
  int grp_bpsm = 0;                  // resident blocks per SM of the grouped SpMM in use
  int bdiag = 0;                     // the grouped records are B-diagonal (see grec_col)
  unsigned char *grec64 = nullptr;   // mixed path: FP64 B-diagonal records of the same groups
  double *x64 = nullptr;             // padded FP64 copy of a real block for the grouped FP64 products
  // real n x L blocks (ld = L)
  double *V = nullptr, *AV = nullptr, *BV = nullptr, *G = nullptr, *AG = nullptr, *BG = nullptr;
  double *U = nullptr, *U2 = nullptr, *BU = nullptr, *Vt = nullptr, *AVt = nullptr, *BVt = nullptr;
  double *X = nullptr, *BX = nullptr;
  // small
  double *Gm = nullptr, *Rinv = nullptr, *Hm = nullptr, *Sm = nullptr, *Wm = nullptr;
  double *theta = nullptr, *theta_act = nullptr, *res = nullptr, *res_paper = nullptr, *sgn = nullptr;
  double *Theta = nullptr, *Res = nullptr;
  double *work = nullptr;
  size_t work_doubles = 0;
  unsigned char *ozwork = nullptr;  // split-bf16 product workspace (opts.dense = 1)
  size_t ozwork_bytes = 0;
  int *dst_x = nullptr, *dst_v = nullptr, *iflags = nullptr;  // iflags: [0..3] lock info, [4] chol, [5] nan
  int *h_iflags = nullptr;                                    // pinned mirror
  JacobiWork jw{};
  cudaEvent_t ev[4] = {};
  // graph cache of the inner loop
  cudaGraphExec_t gexec = nullptr;
  int g_k = -1, g_warm = -1, g_itm = -1;
  int it_cur = 0;  // It_max of the next filter apply (opts.it_adapt: grows per problem)
  int unres_streak = 0;  // consecutive outer steps with the lowest active Ritz pair unresolved
  std::vector<void *> allocs;
};

// ----------------------------------------------------------------------------- helpers
#define CK(call)                                  \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) {                      \
      if (ctx) ctx->status = SLRF_ECUDA;          \
      return SLRF_ECUDA;                          \
    }                                             \
  } while (0)
#define CKL()                                     \
  do {                                            \
    cudaError_t e_ = cudaGetLastError();          \
    if (e_ != cudaSuccess) {                      \
      ctx->status = SLRF_ECUDA;                   \
      return SLRF_ECUDA;                          \
    }                                             \
  } while (0)

template <typename T> static int dalloc(slrf_ctx *ctx, T **p, size_t count) {
  void *q = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc(&q, count * sizeof(T) + 64);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? SLRF_ENOMEM : SLRF_ECUDA;
  }
  ctx->allocs.push_back(q);
  *p = reinterpret_cast<T *>(q);
  return SLRF_OK;
}

static void dfree(slrf_ctx *ctx, void *p) {
  if (!p) return;
  auto it = std::find(ctx->allocs.begin(), ctx->allocs.end(), p);
  if (it != ctx->allocs.end()) ctx->allocs.erase(it);
  cudaFree(p);
}

static int pow2_at_least(int m) {
  int p = 1;
  while (p < m) p <<= 1;
  return p;
}

// columns padded so that k * mp is a multiple of the warp tile (32 * vec complex entries)
static int kpad_of(int k, int mp, int vec) {
  const int tile = 32 * vec;
  const int W = ((k * mp + tile - 1) / tile) * tile;
  return W / mp;
}

// FP64 values of the shifted systems the COCG solves (scaled when preconditioned).
static const double *cocg_valA(const slrf_ctx *c) { return c->dsc ? c->valAs : c->valA; }
static const double *cocg_valB(const slrf_ctx *c) { return c->dsc ? c->valBs : c->valB; }


__global__ void recip_kernel(int64_t count, const double *a, double *b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) b[i] = 1.0 / a[i];
}
__global__ void to_float_kernel(int64_t count, const double *a, float *b) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < count) b[t] = (float)a[t];
}
__global__ void to_float2_kernel(int count, const double2 *a, float2 *b) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < count) b[t] = make_float2((float)a[t].x, (float)a[t].y);
}
// out[0] += breakdowns, out[1] += COCG updates of the last filter apply
__global__ void count_iters_kernel(int W, const WScal *ws, int *out) {
  int c = 0, it = 0;
  for (int w = threadIdx.x; w < W; w += blockDim.x) { c += ws[w].brk; it += ws[w].iters_total; }
  c = warp_sum(c);
  it = warp_sum(it);
  if ((threadIdx.x & 31) == 0) { atomicAdd(out, c); atomicAdd(out + 1, it); }
}

// Fork the library stream from the caller's stream on entry, join it back on exit.
struct StreamScope {
  slrf_ctx *c;
  explicit StreamScope(slrf_ctx *ctx) : c(ctx) {
    cudaEventRecord(c->ev_in, c->ust);
    cudaStreamWaitEvent(c->st, c->ev_in, 0);
  }
  ~StreamScope() {
    cudaEventRecord(c->ev_out, c->st);
    cudaStreamWaitEvent(c->ust, c->ev_out, 0);
  }
};
// final sort of the locked pairs: rank by Theta ascending (ties: lock order)
__global__ void final_rank_kernel(int nconv, const double *Theta, int *rank) {
  for (int i = threadIdx.x; i < nconv; i += blockDim.x) {
    const double di = Theta[i];
    int r = 0;
    for (int j = 0; j < nconv; ++j) {
      const double dj = Theta[j];
      r += (dj < di) || (dj == di && j < i);
    }
    rank[i] = r;
  }
}
__global__ void final_gather_kernel(int64_t n, int nconv, int cnt, const int *rank, const double *Theta,
                                    const double *Res, const double *X, int ldx, double *evals, double *Xo,
                                    int ldo, double *resid) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * nconv) return;
  const int64_t i = t / nconv;
  const int c = (int)(t % nconv);
  const int r = rank[c];
  if (r >= cnt) return;
  if (Xo) Xo[i * ldo + r] = X[i * ldx + c];
  if (i == 0) {
    if (evals) evals[r] = Theta[c];
    if (resid) resid[r] = Res[c];
  }
}

// ----------------------------------------------------------------------------- grouped rows
// The COCG SpMM's grouped-row format (CocgArgs): rows [G g, G g + G) share one union
// column list.  group_counts returns the union sizes for a G; build_groups writes the
// offsets and the records of the working precision; choose_group picks G.
static int group_counts(slrf_ctx *ctx, int G, std::vector<int> &cnt) {
  const int64_t ng = (ctx->n + G - 1) / G;
  int *d = nullptr;
  if (cudaMalloc(&d, (size_t)ng * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return SLRF_ENOMEM;
  }
  grp_count(ctx->n, G, ctx->rowptr, ctx->col, d, ctx->st);
  cnt.resize((size_t)ng);
  cudaError_t e = cudaMemcpyAsync(cnt.data(), d, (size_t)ng * sizeof(int), cudaMemcpyDeviceToHost, ctx->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
  cudaFree(d);
  return e == cudaSuccess ? SLRF_OK : SLRF_ECUDA;
}
static int grec_size(int G, bool fp32) { return grec_bytes_rt(G, fp32); }
static void drop_groups(slrf_ctx *ctx) {
  dfree(ctx, ctx->gptr);
  dfree(ctx, ctx->grec);
  dfree(ctx, ctx->grec64);
  ctx->grec64 = nullptr;
  ctx->gptr = nullptr;
  ctx->grec = nullptr;
  ctx->grp = 1;
  ctx->ngroups = 0;
  ctx->grp_bpsm = 0;
  ctx->bdiag = 0;
  ctx->vec = ctx->mixed ? cocg_vec_csr<float>() : cocg_vec_csr<double>();
}
static int build_groups(slrf_ctx *ctx, int G) {
  drop_groups(ctx);
  if (G <= 1) return SLRF_OK;
  std::vector<int> cnt;
  int rc = group_counts(ctx, G, cnt);
  if (rc != SLRF_OK) return rc;
  const int64_t ng = (int64_t)cnt.size();
  std::vector<int64_t> off((size_t)ng + 1, 0);
  for (int64_t g = 0; g < ng; ++g) off[g + 1] = off[g] + cnt[g];
  // gptr[ng + 1] (one spare word) holds the record check's flag
  if ((rc = dalloc(ctx, &ctx->gptr, (size_t)ng + 2)) != SLRF_OK) return rc;
  if ((rc = dalloc(ctx, &ctx->grec, (size_t)off[ng] * grec_size(G, ctx->mixed) + 16)) != SLRF_OK) return rc;
  if (cudaMemcpyAsync(ctx->gptr, off.data(), off.size() * sizeof(int64_t), cudaMemcpyHostToDevice, ctx->st) !=
      cudaSuccess)
    return SLRF_ECUDA;
  if (ctx->mixed)
    grp_fill<float>(ctx->n, G, ctx->rowptr, ctx->col, cocg_valA(ctx), cocg_valB(ctx), ctx->gptr, ctx->grec, ctx->st);
  else
    grp_fill<double>(ctx->n, G, ctx->rowptr, ctx->col, cocg_valA(ctx), cocg_valB(ctx), ctx->gptr, ctx->grec, ctx->st);
  // the SpMM trusts the record columns (no per-record check): check every record once
  int *dflag = reinterpret_cast<int *>(ctx->gptr + ng + 1);
  int bad = 0;
  if (cudaMemsetAsync(dflag, 0, sizeof(int), ctx->st) != cudaSuccess) return SLRF_ECUDA;
  if (ctx->mixed)
    grp_check<float>(ctx->n, G, ng, ctx->gptr, ctx->grec, dflag, ctx->sm_count * 4, ctx->st);
  else
    grp_check<double>(ctx->n, G, ng, ctx->gptr, ctx->grec, dflag, ctx->sm_count * 4, ctx->st);
  if (cudaMemcpyAsync(&bad, dflag, sizeof(int), cudaMemcpyDeviceToHost, ctx->st) != cudaSuccess ||
      cudaStreamSynchronize(ctx->st) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return SLRF_ECUDA;
  if (bad) {
    drop_groups(ctx);
    return SLRF_EINVAL;
  }
  // 3-row groups of a vector-valued pencil whose B couples only equal dofs: B-diagonal records
  int bd = 0;
  if (G == 3 && ctx->o.bdiag) {
    int nbd = 0;
    if (cudaMemsetAsync(dflag, 0, sizeof(int), ctx->st) != cudaSuccess) return SLRF_ECUDA;
    if (ctx->mixed)
      grp_bd_detect<float>(ctx->n, ng, ctx->gptr, ctx->grec, dflag, ctx->sm_count * 4, ctx->st);
    else
      grp_bd_detect<double>(ctx->n, ng, ctx->gptr, ctx->grec, dflag, ctx->sm_count * 4, ctx->st);
    if (cudaMemcpyAsync(&nbd, dflag, sizeof(int), cudaMemcpyDeviceToHost, ctx->st) != cudaSuccess ||
        cudaStreamSynchronize(ctx->st) != cudaSuccess || cudaGetLastError() != cudaSuccess)
      return SLRF_ECUDA;
    if (nbd == 0) {
      unsigned char *bdrec = nullptr;
      if ((rc = dalloc(ctx, &bdrec, (size_t)off[ng] * grec_bytes_rt(3, ctx->mixed, true) + 16)) != SLRF_OK) return rc;
      if (ctx->mixed) grp_bd_convert<float>(off[ng], ctx->grec, bdrec, ctx->st);
      else grp_bd_convert<double>(off[ng], ctx->grec, bdrec, ctx->st);
      if (cudaMemsetAsync(dflag, 0, sizeof(int), ctx->st) != cudaSuccess) return SLRF_ECUDA;
      if (ctx->mixed) grp_check<float>(ctx->n, 3, ng, ctx->gptr, bdrec, dflag, ctx->sm_count * 4, ctx->st, true);
      else grp_check<double>(ctx->n, 3, ng, ctx->gptr, bdrec, dflag, ctx->sm_count * 4, ctx->st, true);
      if (cudaMemcpyAsync(&bad, dflag, sizeof(int), cudaMemcpyDeviceToHost, ctx->st) != cudaSuccess ||
          cudaStreamSynchronize(ctx->st) != cudaSuccess || cudaGetLastError() != cudaSuccess)
        return SLRF_ECUDA;
      if (bad) {
        dfree(ctx, bdrec);
        drop_groups(ctx);
        return SLRF_EINVAL;
      }
      dfree(ctx, ctx->grec);
      ctx->grec = bdrec;
      bd = 1;
      if (ctx->mixed) {
        // FP64 B-diagonal records of the same groups for the FP64 real products of the outer step
        unsigned char *gen64 = nullptr, *bd64 = nullptr;
        if ((rc = dalloc(ctx, &gen64, (size_t)off[ng] * grec_bytes_rt(3, false) + 16)) != SLRF_OK) return rc;
        if ((rc = dalloc(ctx, &bd64, (size_t)off[ng] * grec_bytes_rt(3, false, true) + 16)) != SLRF_OK) return rc;
        grp_fill<double>(ctx->n, 3, ctx->rowptr, ctx->col, cocg_valA(ctx), cocg_valB(ctx), ctx->gptr, gen64, ctx->st);
        grp_bd_convert<double>(off[ng], gen64, bd64, ctx->st);
        if (cudaMemsetAsync(dflag, 0, sizeof(int), ctx->st) != cudaSuccess) return SLRF_ECUDA;
        grp_check<double>(ctx->n, 3, ng, ctx->gptr, bd64, dflag, ctx->sm_count * 4, ctx->st, true);
        if (cudaMemcpyAsync(&bad, dflag, sizeof(int), cudaMemcpyDeviceToHost, ctx->st) != cudaSuccess ||
            cudaStreamSynchronize(ctx->st) != cudaSuccess || cudaGetLastError() != cudaSuccess)
          return SLRF_ECUDA;
        dfree(ctx, gen64);
        if (bad) dfree(ctx, bd64);
        else ctx->grec64 = bd64;
      }
    }
  }
  ctx->bdiag = bd;
  ctx->grp = G;
  ctx->ngroups = ng;
  ctx->vec = ctx->mixed ? cocg_vec_grp<float>() : cocg_vec_grp<double>();
  ctx->grp_bpsm = grp_blocks_per_sm(G, ctx->mixed, bd != 0);
  return SLRF_OK;
}
// Candidate G from the pattern.  FP64: the SpMM is bound by the FP64 pipe, so only groups
// that add no zero products qualify (union x rows == entries), the largest such G.  FP32:
// a cost per row, in units of one plain-CSR entry, fitted to GB300 timings of the 41^3
// Laplacian (27 entries/row) and the 64x64x32 elasticity box (81): a record of a G-row
// group costs about 1.2 + 0.25 G entries (the gather, the staged record, 8 G packed FMAs).
static int choose_group(slrf_ctx *ctx, int &G) {
  G = 1;
  double best = (double)ctx->nnz / ctx->n;
  for (int g = (ctx->mixed ? 2 : 4); ctx->mixed ? g <= 4 : g >= 2; g += ctx->mixed ? 1 : -1) {
    std::vector<int> cnt;
    int rc = group_counts(ctx, g, cnt);
    if (rc != SLRF_OK) return rc;
    double recs = 0, slots = 0;
    for (size_t i = 0; i < cnt.size(); ++i) {
      recs += cnt[i];
      slots += (double)cnt[i] * (double)std::min<int64_t>(g, ctx->n - (int64_t)i * g);
    }
    if (!ctx->mixed) {
      if (slots <= (double)ctx->nnz) { G = g; return SLRF_OK; }
      continue;
    }
    const double cost = recs / ctx->n * (1.2 + 0.25 * g);
    if (cost < best) { best = cost; G = g; }
  }
  return SLRF_OK;
}
static int setup_groups(slrf_ctx *ctx) {
  int G = ctx->o.group;
  if (G == 0) {
    int rc = choose_group(ctx, G);
    if (rc != SLRF_OK) return rc;
  }
  return build_groups(ctx, G);
}

// ----------------------------------------------------------------------------- filter
// U = sum_j 2 Re(w_j Y_j), (A - sigma_j B) Y_j = B X, in correction form (see cocg.cu).
// AXp/BXp: A X and B X if already known (warm start), else computed here.

// Optional per-kernel timing of one filter apply (measurement hook, direct launches).
struct FilterTiming {
  double ms_init = 0, ms_spmm = 0, ms_update = 0;
  int n_spmm = 0, n_update = 0;
};

// Row blocks per column tile before autotuning.  Plain CSR: about as many as the GPU
// holds resident (SMs x 4 blocks), so that the blocks in flight at any time all belong to
// one or two tiles (the tile index varies slowest) and the gathered rows of those tiles stay
// in L2.  Grouped SpMM: exactly one resident wave of that kernel, whose blocks take
// interleaved stripes of groups and so sweep the rows of a tile together.
static int64_t row_blocks(const slrf_ctx *ctx) {
  const int per_sm = (ctx->grp > 1 && ctx->grp_bpsm > 0) ? std::min(ctx->grp_bpsm, 4) : 4;
  return (int64_t)ctx->sm_count * per_sm;
}
// FP64 B-diagonal records of the context, or null: an FP64 context's own records, or the extra
// FP64 records of a mixed context
static const unsigned char *rec64(const slrf_ctx *ctx) {
  if (ctx->grp != 3 || !ctx->bdiag) return nullptr;
  return ctx->mixed ? ctx->grec64 : ctx->grec;
}
// FP64 products A X, B X (either output may be null) with the stored matrices: through the FP64
// B-diagonal records when the context has them (scaled back by D^1/2 when they hold the
// Jacobi-scaled values), else the CSR kernel.
static void real_products64(slrf_ctx *ctx, const double *X, int ldx, int k, double *YA, double *YB, int ldy,
                            cudaStream_t st);

// row blocks of the grouped real SpMM: one resident wave, no more than there are stripes
static int grp_real_blocks(const slrf_ctx *ctx) {
  const int64_t stripes = (ctx->ngroups + kWarps - 1) / kWarps;
  return (int)std::max<int64_t>(1, std::min<int64_t>(row_blocks(ctx), stripes));
}
static void real_products64(slrf_ctx *ctx, const double *X, int ldx, int k, double *YA, double *YB, int ldy,
                            cudaStream_t st) {
  const unsigned char *r64 = rec64(ctx);
  if (r64 != nullptr && ctx->x64 != nullptr)
    spmm_grp_real64(ctx->n, ctx->ngroups, ctx->gptr, r64, ctx->iflags + 15, grp_real_blocks(ctx), X, ldx, k,
                    ctx->dsqrt, ctx->x64, YA, YB, ldy, ctx->dsqrt, st);
  else
    spmm_real(ctx->n, ctx->rowptr, ctx->col, ctx->valA, ctx->valB, X, ldx, k, YA, YB, ldy, st);
}

// COCG arguments of one filter apply of this context (k columns, optional warm start).
template <typename R>
static CocgArgs<R> build_cocg_args(slrf_ctx *ctx, const double *X, int ldx, int k, double *U, int ldu, int &nref) {
  const int vec = ctx->vec;  // lane width of the SpMM format in use
  const int kp = kpad_of(k, ctx->mp, vec);
  const int W = kp * ctx->mp;
  // row blocks per tile (row_blocks); an autotuned row count (slrf_opts.autotune) replaces it
  const int64_t rblocks = row_blocks(ctx);
  int64_t rpb = std::max<int64_t>(16, (ctx->n + rblocks - 1) / rblocks);
  if (ctx->rpb_tuned > 0) rpb = std::max<int64_t>(rpb, ctx->rpb_tuned);
  // whole groups per row block, the same number for every warp of the block
  const int64_t unit = (int64_t)ctx->grp * kWarps;
  rpb = (rpb + unit - 1) / unit * unit;
  const int nrb = (int)((ctx->n + rpb - 1) / rpb);
  CocgArgs<R> a{};
  a.n = ctx->n;
  a.rowptr = ctx->rowptr;
  a.col = ctx->col;
  if constexpr (sizeof(R) == 8) {
    a.valA = cocg_valA(ctx); a.valB = cocg_valB(ctx); a.sig = ctx->sig;
  } else {
    a.valA = ctx->valA32; a.valB = ctx->valB32; a.sig = ctx->sig32;
  }
  a.G = ctx->grp;
  a.ngroups = ctx->ngroups;
  a.gptr = ctx->gptr;
  a.grec = ctx->grec;
  a.bdiag = ctx->bdiag;
  a.err = ctx->iflags + 15;
  a.dsc = ctx->dsc;
  a.uacc = ctx->uacc;
  a.W = W; a.vec = vec; a.k = k; a.m = ctx->m; a.mp = ctx->mp;
  a.rows_per_block = (int)rpb; a.nrb = nrb;
  a.d = (cx_t<R> *)ctx->cd; a.r = (cx_t<R> *)ctx->cr; a.p = (cx_t<R> *)ctx->cp; a.q = (cx_t<R> *)ctx->cq;
  a.partial = ctx->partial; a.counters = ctx->counters; a.ws = ctx->ws;
  a.tol2 = ctx->o.tol_inner * ctx->o.tol_inner;
  a.g = ctx->G; a.Ag = ctx->AG; a.Bg = ctx->BG; a.ldg = ctx->L;
  a.cfac = ctx->cfac; a.wt = ctx->wt;
  a.gscale = sizeof(R) == 4 ? ctx->gscale : nullptr;
  a.V = X; a.ldv = ldx; a.coefV = ctx->coefV; a.U = U; a.ldu = ldu;
  // refinement steps: the FP32 path repeats (FP64 residual, fresh FP32 solve) refine_max times
  nref = (sizeof(R) == 4 && ctx->D64 != nullptr) ? std::max(1, ctx->o.refine_max) : 1;
  if (nref > 1) {
    a.D64 = ctx->D64;
    a.valA64 = cocg_valA(ctx);
    a.valB64 = cocg_valB(ctx);
    a.sig64 = ctx->sig;
    a.r00 = ctx->r00;
  }
  ctx->last_k = k;
  ctx->last_W = W;
  return a;
}

// Update modes of refinement step `step` of `nref`: the middle updates and the last one.
// FP32 without refinement: every update adds its step to the accumulator (kAccU, no d
// array); in FP64 the extra complex product per entry costs more on the FP64 pipe than the
// d traffic it saves, so the FP64 path keeps d and its last update writes U (kFinalU).
template <typename R> static void update_modes(int nref, int step, int &fm_mid, int &fm_last) {
  const bool accu = nref == 1 && sizeof(R) == 4;
  fm_mid = accu ? kAccU : kFinalNone;
  fm_last = accu        ? kAccUEnd
            : nref == 1 ? kFinalU
            : step == 1 ? kFinalStoreD
                        : (step < nref ? kFinalAddD : kFinalUFromD);
}

template <typename R>
static int run_cocg(slrf_ctx *ctx, const double *X, int ldx, int k, const double *theta, double *U, int ldu,
                    bool capture_ok, FilterTiming *tm) {
  int nref = 1;
  CocgArgs<R> a = build_cocg_args<R>(ctx, X, ldx, k, U, ldu, nref);
  const int W = a.W;
  const int itm = ctx->it_cur > 0 ? ctx->it_cur : ctx->o.it_max;
  const int T = W / (32 * a.vec);  // column tiles
  // Two-group schedule (graph and direct paths, FP32 path): the tiles are split into two
  // groups that run one launch apart, so that each launch carries the SpMM of one group and
  // the update of the other (cocg_dual); each group still alternates update and SpMM in
  // order.  Measured on the 41^3 workload: -3 % filter time in FP32; in FP64 both kernels
  // load the FP64 pipe (the update does ~11 FP64 FMAs per entry), so there it is not used.
  const bool dual_ok = sizeof(R) == 4 && T >= 2 && itm >= 2 && ctx->grp == 1;
  ctx->launches += 2 * itm + 1 + (sizeof(R) == 4 ? 3 : 0) + (int64_t)(nref - 1) * (2 * itm + 1) +
                   (dual_ok && tm == nullptr ? nref : 0);
  // one launch sequence for the graph, the direct and the timed path; `kind` tags each
  // launch for the timing hook (0 other, 1 SpMM, 2 update, 3 init, 4 SpMM + update)
  auto body = [&](cudaStream_t s, auto &&launch, bool dual) {
    launch(0, [&] { cocg_prepare(W, k, ctx->m, ctx->mp, ctx->sig, ctx->wt, theta, ctx->cfac, ctx->coefV, ctx->ws, s); });
    if (sizeof(R) == 4)
      launch(0, [&] { col_scale(ctx->n, k, ctx->G, ctx->L, ctx->gmax, ctx->gscale, s); });
    launch(3, [&] { cocg_init<R>(a, s); });
    for (int step = 1; step <= nref; ++step) {
      if (step > 1) {
        if constexpr (sizeof(R) == 4) launch(0, [&] { cocg_residual<R>(a, s); });
        launch(1, [&] { cocg_spmm<R>(a, s, true); });
      }
      int fm_mid, fm_last;
      update_modes<R>(nref, step, fm_mid, fm_last);
      if (dual && dual_ok) {
        const int n0 = T / 2, n1 = T - n0;  // group 0: tiles [0, n0), group 1: [n0, T)
        launch(2, [&] { cocg_update<R>(a, true, fm_mid, s, 0, n0); });  // U_1 of group 0
        for (int t = 1; t < itm; ++t) {
          // S_t of group 0 with U_t of group 1, then S_t of group 1 with U_{t+1} of group 0
          launch(4, [&] { cocg_dual<R>(a, 0, n0, n0, n1, t == 1, fm_mid, s); });
          launch(4, [&] { cocg_dual<R>(a, n0, n1, 0, n0, false, t + 1 == itm ? fm_last : fm_mid, s); });
        }
        launch(2, [&] { cocg_update<R>(a, false, fm_last, s, n0, n1); });  // U_itm of group 1
      } else {
        for (int it = 1; it <= itm; ++it) {
          launch(2, [&] { cocg_update<R>(a, it == 1, it == itm ? fm_last : fm_mid, s); });
          if (it < itm) launch(1, [&] { cocg_spmm<R>(a, s); });
        }
      }
    }
  };
  auto plain = [](int, auto &&fn) { fn(); };
  if (tm != nullptr) {
    // same launches, each bracketed by events on the library stream
    cudaStream_t s = ctx->st;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> evs;
    auto timed = [&](int kind, auto &&fn) {
      cudaEvent_t e0, e1;
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      cudaEventRecord(e0, s);
      fn();
      cudaEventRecord(e1, s);
#if SLRF_CHECKS
      {  // debug build: run launch by launch and report the first one that fails
        const cudaError_t e = cudaStreamSynchronize(s);
        fprintf(stderr, "slrf timed launch %zu kind %d: %s\n", evs.size(), kind, cudaGetErrorString(e));
      }
#endif
      evs.push_back({kind, {e0, e1}});
    };
    body(s, timed, false);
    CKL();
    CK(cudaStreamSynchronize(s));
    for (auto &e : evs) {
      float t = 0;
      cudaEventElapsedTime(&t, e.second.first, e.second.second);
      if (e.first == 1) { tm->ms_spmm += t; tm->n_spmm++; }
      else if (e.first == 2) { tm->ms_update += t; tm->n_update++; }
      else if (e.first == 3) tm->ms_init += t;
      cudaEventDestroy(e.second.first);
      cudaEventDestroy(e.second.second);
    }
  } else if (capture_ok && ctx->o.use_graph) {
    const int warm = theta != nullptr;
    if (!(ctx->gexec && ctx->g_k == k && ctx->g_warm == warm && ctx->g_itm == itm)) {
      if (ctx->gexec) { cudaGraphExecDestroy(ctx->gexec); ctx->gexec = nullptr; }
      cudaGraph_t g;
      CK(cudaStreamBeginCapture(ctx->st, cudaStreamCaptureModeThreadLocal));
      body(ctx->st, plain, true);
      CK(cudaStreamEndCapture(ctx->st, &g));
      cudaError_t e = cudaGraphInstantiate(&ctx->gexec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) { ctx->status = SLRF_ECUDA; return SLRF_ECUDA; }
      ctx->g_k = k;
      ctx->g_warm = warm;
      ctx->g_itm = itm;
    }
    CK(cudaGraphLaunch(ctx->gexec, ctx->st));
  } else {
    body(ctx->st, plain, true);
  }
  CKL();
  return SLRF_OK;
}

// The real FP64 sweep that starts every pole (Proposition (i), Sec. 4):
//   zero guess:  g = B X;   warm start:  g = A X - theta B X;   then A g and B g.
static int filter_prep(slrf_ctx *ctx, const double *X, int ldx, int k, const double *theta, const double *AXp,
                       const double *BXp) {
  const cudaStream_t st = ctx->st;
  const int L = ctx->L;
  if (theta == nullptr) {
    real_products64(ctx, X, ldx, k, nullptr, ctx->G, L, st);
    ctx->launches += 1;
  } else {
    const double *AX = AXp, *BX = BXp;
    int ldab = L;
    if (AX == nullptr || BX == nullptr) {
      real_products64(ctx, X, ldx, k, ctx->AG, ctx->BG, L, st);
      AX = ctx->AG;
      BX = ctx->BG;
      ctx->launches += 1;
    }
    shifted_residual(ctx->n, k, AX, BX, ldab, theta, ctx->G, L, st);
    ctx->launches += 1;
  }
  // preconditioned: the solves start from D^-1/2 g and the scaled matrices
  if (ctx->dsc != nullptr) {
    row_scale(ctx->n, k, ctx->dsc, ctx->G, L, st);
    ctx->launches += 1;
  }
  // A g and B g only start the COCG recurrences (q0); in the mixed path those run in FP32
  if (ctx->mixed && ctx->grp > 1)  // the records hold exactly the values the solves use
    spmm_grp_real32(ctx->n, ctx->grp, ctx->ngroups, ctx->gptr, ctx->grec, ctx->iflags + 15, grp_real_blocks(ctx),
                    ctx->G, L, k, nullptr, ctx->x32, ctx->AG, ctx->BG, L, nullptr, st, ctx->bdiag != 0);
  else if (ctx->mixed)
    spmm_ab32(ctx->n, ctx->rowptr, ctx->col, cocg_valA(ctx), cocg_valB(ctx), ctx->G, L, k, ctx->AG, ctx->BG, L, st);
  else if (rec64(ctx) != nullptr && ctx->x64 != nullptr)  // records hold the values the solves use
    spmm_grp_real64(ctx->n, ctx->ngroups, ctx->gptr, rec64(ctx), ctx->iflags + 15, grp_real_blocks(ctx), ctx->G, L, k,
                    nullptr, ctx->x64, ctx->AG, ctx->BG, L, nullptr, st);
  else
    spmm_real(ctx->n, ctx->rowptr, ctx->col, cocg_valA(ctx), cocg_valB(ctx), ctx->G, L, k, ctx->AG, ctx->BG, L, st);
  ctx->launches += 1;
  CKL();
  return SLRF_OK;
}

static int filter_impl(slrf_ctx *ctx, const double *X, int ldx, int k, const double *theta, const double *AXp,
                       const double *BXp, double *U, int ldu, bool capture_ok, FilterTiming *tm = nullptr) {
  int rc = filter_prep(ctx, X, ldx, k, theta, AXp, BXp);
  if (rc != SLRF_OK) return rc;
  if (ctx->mixed) return run_cocg<float>(ctx, X, ldx, k, theta, U, ldu, capture_ok, tm);
  return run_cocg<double>(ctx, X, ldx, k, theta, U, ldu, capture_ok, tm);
}

// Autotuner: time the fused SpMM (best of three launches) on a Gaussian block of the full
// width (after the usual initialisation) for each group height of the grouped-row format
// (when opts.group = 0), then for each candidate rows-per-block, and keep the fastest.
template <typename R>
static int autotune_rows(slrf_ctx *ctx) {
  const cudaStream_t st = ctx->st;
  const int L = ctx->L;
  gaussian_block(ctx->n, L, ctx->o.seed + 7, ctx->V, L, st);
  int rc = filter_prep(ctx, ctx->V, L, L, nullptr, nullptr, nullptr);
  if (rc != SLRF_OK) return rc;
  auto base_rows = [&]() {
    const int64_t rblocks = row_blocks(ctx);
    return std::max<int64_t>(16, (ctx->n + rblocks - 1) / rblocks);
  };
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  // best of three SpMM launches with the current group height and rows per block
  auto time_spmm = [&](float &t) -> int {
    int nref = 1;
    CocgArgs<R> a = build_cocg_args<R>(ctx, ctx->V, L, L, ctx->U, L, nref);
    cocg_prepare(a.W, L, ctx->m, ctx->mp, ctx->sig, ctx->wt, nullptr, ctx->cfac, ctx->coefV, ctx->ws, st);
    if (sizeof(R) == 4) col_scale(ctx->n, L, ctx->G, L, ctx->gmax, ctx->gscale, st);
    cocg_init<R>(a, st);
    t = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(e0, st);
      cocg_spmm<R>(a, st);
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) return SLRF_ECUDA;
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      t = std::min(t, ms);
    }
    return SLRF_OK;
  };
  float best = 1e30f, t = 0;
  if (ctx->o.group == 0) {
    // group height: plain CSR and every grouped format the precision admits (FP64: the
    // no-fill height the pattern model found, if any; FP32: 2, 3 and 4)
    const int g_model = ctx->grp;
    int best_g = 1;
    for (int g = 1; g <= 4; ++g) {
      if (g > 1 && !ctx->mixed && g != g_model) continue;
      if ((rc = build_groups(ctx, g)) != SLRF_OK) break;
      ctx->rpb_tuned = 0;
      if ((rc = time_spmm(t)) != SLRF_OK) break;
      if (t < best) { best = t; best_g = g; }
    }
    if (rc == SLRF_OK) rc = build_groups(ctx, best_g);
    if (rc != SLRF_OK) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return rc;
    }
  }
  const int64_t base = base_rows();
  const int64_t cand[] = {base, 32, 64, 128, 256};
  best = 1e30f;
  int64_t best_r = 0;
  for (int64_t c : cand) {
    if (c < base || c > ctx->n) continue;
    ctx->rpb_tuned = c;
    if ((rc = time_spmm(t)) != SLRF_OK) break;
    if (t < best) { best = t; best_r = c; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != SLRF_OK) return rc;
  ctx->rpb_tuned = best_r;
  CKL();
  return SLRF_OK;
}

// opts.it_adapt: after three consecutive outer steps whose lowest active Ritz pair is still
// unresolved (relative residual > 1e-2), the problem's It_max doubles, up to 8 opts.it_max.
static void adapt_it(slrf_ctx *c, bool unresolved) {
  if (!c->o.it_adapt) return;
  if (!unresolved) { c->unres_streak = 0; return; }
  if (++c->unres_streak >= 3) {
    c->it_cur = std::min(2 * c->it_cur, 8 * c->o.it_max);
    c->unres_streak = 0;
  }
}

// ----------------------------------------------------------------------------- products
// Tall-skinny products of the outer update: split-bf16 tensor-core products with the error
// of an FP64 product (opts.dense = 1) or FP64 FMA on the CUDA cores.  FP32 first passes
// stay on the CUDA cores, and so do tall products (n > 4096) below kOzMinWork = n k1 k2
// multiply-adds, where the FP64 product (~2 n k1 k2 / 1e12 s) beats the fixed ~80 us of the
// split path's launches (the small k x k products keep the split path: the FP64 kernels
// would run on a handful of blocks).  Each adds the kernels it launches to ctx->launches.
constexpr double kOzMinWork = 5e7;
static bool use_split(const slrf_ctx *ctx, int64_t n, int k1, int k2) {
  return ctx->ozwork != nullptr && (n <= 4096 || (double)n * k1 * k2 >= kOzMinWork);
}
static void tsgram(slrf_ctx *ctx, int64_t n, const double *X, int ldx, int k1, const double *Y, int ldy, int k2,
                   double *C, int ldc, bool sym, bool fp32 = false, const int *run_if = nullptr) {
  if (!fp32 && use_split(ctx, n, k1, k2)) {
    const bool same = X == Y && ldx == ldy && k1 == k2;
    oz_gram(n, X, ldx, k1, Y, ldy, k2, C, ldc, sym, ctx->ozwork, ctx->ozwork_bytes, ctx->iflags + 13, ctx->st,
            run_if);
    ctx->launches += same ? 4 : 6;
  } else {
    gram(n, X, ldx, k1, Y, ldy, k2, C, ldc, sym, ctx->work, ctx->st, fp32, run_if);
    ctx->launches += 2;
  }
}
static void tsgemm(slrf_ctx *ctx, int64_t n, const double *X, int ldx, int k1, const double *S, int lds, int k2,
                   double *Z, int ldz, double alpha, double beta, bool upper) {
  if (use_split(ctx, n, k1, k2)) {
    oz_gemm(n, X, ldx, k1, S, lds, k2, Z, ldz, alpha, beta, ctx->ozwork, ctx->ozwork_bytes, ctx->iflags + 13,
            ctx->st);
    ctx->launches += 4;
  } else {
    gemm_nn(n, X, ldx, k1, S, lds, k2, Z, ldz, alpha, beta, upper, ctx->st);
    ctx->launches += 1;
  }
}

// ----------------------------------------------------------------------------- RR step
// U (n x k, ld L) -> B-orth vs X (CGS2) -> Cholesky-QR2 -> Rayleigh-Ritz -> Vt, AVt, BVt,
// theta, res, res_paper, sgn.  The second CholQR pass is folded into the projection:
//   U1 = U R1^{-1};  G2 = U1^T B U1 = R2^T R2;  H = R2^{-T} (U1^T A U1) R2^{-1} = S Theta S^T;
//   V = U1 (R2^{-1} S)
// which equals projecting on U2 = U1 R2^{-1} without forming U2 (one n x k^2 product and
// one SpMM fewer).  With want_basis, U2 is formed into U as well.  Cholesky failure is
// reported through iflags[4].
static int rr_impl(slrf_ctx *ctx, double *U, int k, const double *X, const double *BX, int nconv, int ldx,
                   bool want_basis = false) {
  const cudaStream_t st = ctx->st;
  const int64_t n = ctx->n;
  const int L = ctx->L;
  ctx->launches += 9;  // 3 SpMMs (FP32 B U, gated FP64 B U, A U1 + B U1), 3 Cholesky, Jacobi, 2 residual
                      // kernels; the products count themselves
  // First passes in FP32 (mixed-precision CGS2 and Cholesky-QR): their Gram matrices only
  // have to bring U close to the target; the FP64 second passes remove the FP32 error.
  if (nconv > 0) {
    for (int pass = 0; pass < 2; ++pass) {
      tsgram(ctx, n, BX, ldx, nconv, U, L, k, ctx->Wm, k, false, pass == 0);
      tsgemm(ctx, n, X, ldx, nconv, ctx->Wm, k, k, U, L, -1.0, 1.0, false);
    }
  }
  double *U1 = ctx->U2, *AU1 = ctx->AG;
  // pass 1: U1 = U R1^{-1}, R1 from the FP32 Gram; if that Gram is not numerically
  // positive definite (kappa(U) beyond ~1e3), iflags[11] triggers the FP64 Gram instead
  // FP32 B U: feeds the FP32 Gram.  Through the FP32 records when there are any; with the
  // preconditioner they hold D^-1/2 B D^-1/2, so B U = D^1/2 (D^-1/2 B D^-1/2) (D^1/2 U)
  if (ctx->mixed && ctx->grp > 1)
    spmm_grp_real32(n, ctx->grp, ctx->ngroups, ctx->gptr, ctx->grec, ctx->iflags + 15, grp_real_blocks(ctx), U, L,
                    k, ctx->dsqrt, ctx->x32, nullptr, ctx->BU, L, ctx->dsqrt, st, ctx->bdiag != 0);
  else
    spmm_b32(n, ctx->rowptr, ctx->col, ctx->valB, U, L, k, ctx->BU, L, st);
  cudaMemsetAsync(ctx->iflags + 11, 0, sizeof(int), st);
  tsgram(ctx, n, U, L, k, ctx->BU, L, k, ctx->Gm, k, true, true);
  chol_inv(k, ctx->Gm, k, ctx->Rinv, k, ctx->iflags + 11, st, nullptr, true);
  spmm_real(n, ctx->rowptr, ctx->col, ctx->valA, ctx->valB, U, L, k, nullptr, ctx->BU, L, st, ctx->iflags + 11);
  tsgram(ctx, n, U, L, k, ctx->BU, L, k, ctx->Gm, k, true, false, ctx->iflags + 11);
  chol_inv(k, ctx->Gm, k, ctx->Rinv, k, ctx->iflags + 4, st, ctx->iflags + 11);
  tsgemm(ctx, n, U, L, k, ctx->Rinv, k, k, U1, L, 1.0, 0.0, true);
  // pass 2 and projection
  real_products64(ctx, U1, L, k, AU1, ctx->BU, L, st);
  tsgram(ctx, n, U1, L, k, ctx->BU, L, k, ctx->Gm, k, true);
  tsgram(ctx, n, U1, L, k, AU1, L, k, ctx->Hm, k, true);
  chol_inv(k, ctx->Gm, k, ctx->Rinv, k, ctx->iflags + 4, st);
  tsgemm(ctx, k, ctx->Hm, k, k, ctx->Rinv, k, k, ctx->Wm, k, 1.0, 0.0, true);  // T = H1 R2^{-1}
  tsgram(ctx, k, ctx->Rinv, k, k, ctx->Wm, k, k, ctx->Gm, k, true);           // H = R2^{-T} T
  CKL();
  int rc = jacobi_eig(k, ctx->Gm, k, ctx->theta, ctx->Sm, k, ctx->jw, st);
  if (rc != SLRF_OK) { ctx->status = rc; return rc; }
  tsgemm(ctx, k, ctx->Rinv, k, k, ctx->Sm, k, k, ctx->Wm, k, 1.0, 0.0, false);  // Z = R2^{-1} S
  tsgemm(ctx, n, U1, L, k, ctx->Wm, k, k, ctx->Vt, L, 1.0, 0.0, false);         // V = U1 Z
  if (want_basis) tsgemm(ctx, n, U1, L, k, ctx->Rinv, k, k, U, L, 1.0, 0.0, true);
  if (!want_basis && use_split(ctx, n, k, k)) {
    // inside the solve: A V = (A U1) Z and B V = (B U1) Z, two tensor-core products instead
    // of an FP64 SpMM (they differ from A and B times the stored V by u |A| |V|, far below
    // the lock tolerance); slrf_rayleigh_ritz reports the residuals of the V it returns
    tsgemm(ctx, n, AU1, L, k, ctx->Wm, k, k, ctx->AVt, L, 1.0, 0.0, false);
    tsgemm(ctx, n, ctx->BU, L, k, ctx->Wm, k, k, ctx->BVt, L, 1.0, 0.0, false);
  } else {
    real_products64(ctx, ctx->Vt, L, k, ctx->AVt, ctx->BVt, L, st);
    ctx->launches += 1;
  }
  ritz_residuals(n, k, ctx->Vt, ctx->AVt, ctx->BVt, L, ctx->theta, ctx->res, ctx->res_paper, ctx->sgn, ctx->work, st);
  CKL();
  return SLRF_OK;
}


// ----------------------------------------------------------------------------- batched
struct slrf_batch {
  int P = 0;
  std::vector<slrf_ctx *> c;
  cudaStream_t st = nullptr, ust = nullptr;
  cudaEvent_t ev_in = nullptr, ev_b = nullptr, ev_t0 = nullptr, ev_t1 = nullptr;
  cudaEvent_t ev_f0 = nullptr, ev_f1 = nullptr;  // around the batched COCG of an outer step
  std::vector<cudaEvent_t> ev_p;
  bool mixed = false;
  void *dargs = nullptr, *hargs = nullptr;
  int *dprefix = nullptr, *hprefix = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int g_P = -1, g_total = -1, g_itm = -1;
};

static void batch_free(slrf_batch *b) {
  if (!b) return;
  if (b->st) cudaStreamSynchronize(b->st);
  for (auto *c : b->c) slrf_destroy(c);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  for (auto e : b->ev_p) if (e) cudaEventDestroy(e);
  for (auto e : {b->ev_in, b->ev_b, b->ev_t0, b->ev_t1, b->ev_f0, b->ev_f1}) if (e) cudaEventDestroy(e);
  if (b->dargs) cudaFree(b->dargs);
  if (b->dprefix) cudaFree(b->dprefix);
  if (b->hargs) cudaFreeHost(b->hargs);
  if (b->hprefix) cudaFreeHost(b->hprefix);
  if (b->st) cudaStreamDestroy(b->st);
  delete b;
}

// One persistent batched COCG pass over the active problems (args/prefix already on the
// device): init, then refine_max x (It_max updates and SpMMs), on the batch stream.
template <typename R>
static void batch_cocg(slrf_batch *b, int P, int total, int nref, int itm, cudaStream_t s) {
  const CocgArgs<R> *args = reinterpret_cast<const CocgArgs<R> *>(b->dargs);
  const int *pre = b->dprefix;
  cocg_init_batched_launch<R>(args, pre, P, total, s);
  for (int step = 1; step <= nref; ++step) {
    if (step > 1) {
      if constexpr (sizeof(R) == 4) cocg_residual_batched_launch<R>(args, pre, P, total, s);
      cocg_spmm_batched_launch<R>(args, pre, P, total, true, s);
    }
    int fm_mid, fm_last;
    update_modes<R>(nref, step, fm_mid, fm_last);
    for (int it = 1; it <= itm; ++it) {
      cocg_update_batched_launch<R>(args, pre, P, total, it == 1, it == itm ? fm_last : fm_mid, s);
      if (it < itm) cocg_spmm_batched_launch<R>(args, pre, P, total, false, s);
    }
  }
}

template <typename R>
static int batch_outer_filter(slrf_batch *b, const std::vector<int> &act, const std::vector<int> &kk,
                              const std::vector<char> &warm, int64_t &launches) {
  slrf_ctx *ctx = nullptr;  // for CK
  const int vec = cocg_vec_csr<R>();  // the batched kernels run the plain CSR lane width
  CocgArgs<R> *ha = reinterpret_cast<CocgArgs<R> *>(b->hargs);
  int nref = 1, total = 0, itm = 0;
  const int P = (int)act.size();
  b->hprefix[0] = 0;
  for (int i = 0; i < P; ++i) {
    slrf_ctx *c = b->c[act[i]];
    const int k = kk[act[i]];
    const double *th = warm[act[i]] ? c->theta_act : nullptr;
    int rc = filter_prep(c, c->V, c->L, k, th, warm[act[i]] ? c->AV : nullptr, warm[act[i]] ? c->BV : nullptr);
    if (rc != SLRF_OK) return rc;
    ha[i] = build_cocg_args<R>(c, c->V, c->L, k, c->U, c->L, nref);
    ha[i].it_cap = c->o.it_adapt ? c->it_cur : 0;  // per-problem It_max inside the shared loop
    if (ha[i].vec != vec || ha[i].G != 1) return SLRF_EINVAL;  // the batched setup forces group = 1
    for (int step = 1; step <= nref; ++step) {  // the batched kernels read these buffers unchecked
      int fm_mid, fm_last;
      update_modes<R>(nref, step, fm_mid, fm_last);
      if (!cocg_mode_ok(ha[i], fm_mid) || !cocg_mode_ok(ha[i], fm_last)) return SLRF_EINVAL;
    }
    itm = std::max(itm, c->it_cur > 0 ? c->it_cur : c->o.it_max);
    cocg_prepare(ha[i].W, k, c->m, c->mp, c->sig, c->wt, th, c->cfac, c->coefV, c->ws, c->st);
    if (sizeof(R) == 4) col_scale(c->n, k, c->G, c->L, c->gmax, c->gscale, c->st);
    launches += 1 + (sizeof(R) == 4 ? 2 : 0);
    total += ha[i].nrb * (ha[i].W / (32 * vec));
    b->hprefix[i + 1] = total;
    CK(cudaEventRecord(b->ev_p[act[i]], c->st));
    CK(cudaStreamWaitEvent(b->st, b->ev_p[act[i]], 0));
  }
  CK(cudaMemcpyAsync(b->dargs, b->hargs, P * sizeof(CocgArgs<R>), cudaMemcpyHostToDevice, b->st));
  CK(cudaMemcpyAsync(b->dprefix, b->hprefix, (P + 1) * sizeof(int), cudaMemcpyHostToDevice, b->st));
  launches += 1 + (int64_t)nref * (2 * itm - 1) + (nref - 1) * (sizeof(R) == 4 ? 2 : 1);
  CK(cudaEventRecord(b->ev_f0, b->st));
  if (b->c[act[0]]->o.use_graph) {
    if (!(b->gexec && b->g_P == P && b->g_total == total && b->g_itm == itm)) {
      if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
      cudaGraph_t g;
      CK(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
      batch_cocg<R>(b, P, total, nref, itm, b->st);
      CK(cudaStreamEndCapture(b->st, &g));
      cudaError_t e = cudaGraphInstantiate(&b->gexec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return SLRF_ECUDA;
      b->g_P = P;
      b->g_total = total;
      b->g_itm = itm;
    }
    CK(cudaGraphLaunch(b->gexec, b->st));
  } else {
    batch_cocg<R>(b, P, total, nref, itm, b->st);
  }
  if (cudaGetLastError() != cudaSuccess) return SLRF_ECUDA;
  CK(cudaEventRecord(b->ev_f1, b->st));
  CK(cudaEventRecord(b->ev_b, b->st));
  for (int i = 0; i < P; ++i) CK(cudaStreamWaitEvent(b->c[act[i]]->st, b->ev_b, 0));
  return SLRF_OK;
}

// ----------------------------------------------------------------------------- ABI
extern "C" {

int slrf_opts_default(slrf_opts *o) {
  if (!o) return SLRF_EINVAL;
  memset(o, 0, sizeof(*o));
  o->m = 8;
  o->alpha = 1.0;
  o->beta = 0.01;
  o->band = 1.3;
  o->it_max = 40;
  o->refine_max = 1;
  o->outer_max = 100;
  o->tol_inner = 1e-10;
  o->tol_eig = 1e-8;
  o->precision = 0;
  o->warm_start = 1;
  o->lock = 1;
  o->use_graph = 1;
  o->nev = 0;
  o->seed = 1;
  o->dense = 1;
  o->bdiag = 1;
  return SLRF_OK;
}

int slrf_wait_selftest(int kind, void *stream) {
  if (kind < 0 || kind > 1) return SLRF_EINVAL;
  const cudaStream_t st = (cudaStream_t)stream;
  void *buf = nullptr;
  if (cudaMalloc(&buf, 16) != cudaSuccess) {
    cudaGetLastError();
    return SLRF_ENOMEM;
  }
  int herr = 0;
  cudaError_t e = cudaMemsetAsync(buf, 0, 16, st);
  if (e == cudaSuccess) {
    wait_selftest(kind, reinterpret_cast<unsigned *>(buf), reinterpret_cast<int *>(buf) + 1, st);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, reinterpret_cast<int *>(buf) + 1, sizeof(int),
                                            cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(buf);
  if (e != cudaSuccess) return SLRF_ECUDA;
  return herr != 0 ? SLRF_ETIMEOUT : SLRF_OK;
}

const char *slrf_strerror(int s) {
  switch (s) {
    case SLRF_OK: return "ok";
    case SLRF_EINVAL: return "invalid argument";
    case SLRF_ENOMEM: return "not enough device memory";
    case SLRF_ECUDA: return "CUDA runtime error";
    case SLRF_EBREAKDOWN: return "COCG breakdown";
    case SLRF_ETIMEOUT: return "bounded device wait timed out";
    case SLRF_ECHOL: return "Gram matrix not positive definite (Cholesky failed)";
    case SLRF_ENOCONV: return "outer iteration cap reached";
    case SLRF_ENAN: return "non-finite value";
    case SLRF_ETRUNC: return "output capacity too small";
    case SLRF_ESTATE: return "context in failed state";
    default: return "unknown status";
  }
}

int slrf_last_error(const slrf_ctx *ctx) { return ctx ? ctx->status : SLRF_EINVAL; }

// ----------------------------------------------------------------------------- products (ABI)
static int ts_prologue(int64_t n, int k1, int k2, int mode, cudaStream_t st, void **work, int **err,
                       size_t bytes) {
  if (n < 0 || k1 < 1 || k2 < 1 || k1 > 512 || k2 > 512 || (mode != 0 && mode != 1)) return SLRF_EINVAL;
  if (cudaMallocAsync(work, bytes + 64, st) != cudaSuccess) { cudaGetLastError(); return SLRF_ENOMEM; }
  if (cudaMallocAsync(reinterpret_cast<void **>(err), sizeof(int), st) != cudaSuccess) {
    cudaGetLastError();
    cudaFreeAsync(*work, st);
    return SLRF_ENOMEM;
  }
  cudaMemsetAsync(*err, 0, sizeof(int), st);
  return SLRF_OK;
}
static int ts_epilogue(cudaStream_t st, void *work, int *err) {
  int h = 0;
  cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(work, st);
  cudaFreeAsync(err, st);
  if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) return SLRF_ECUDA;
  return h != 0 ? SLRF_ETIMEOUT : SLRF_OK;
}

int slrf_tsgram(int64_t n, const double *X, int ldx, int k1, const double *Y, int ldy, int k2, double *C, int ldc,
                int mode, void *stream) {
  if ((n > 0 && (!X || !Y)) || !C || ldx < k1 || ldy < k2 || ldc < k2) return SLRF_EINVAL;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t bytes = mode == 1 ? oz_work_bytes(n, k1, k2)
                                 : std::max<size_t>(gram_work_doubles(n, k1, k2), 1) * sizeof(double);
  void *work = nullptr;
  int *err = nullptr;
  int rc = ts_prologue(n, k1, k2, mode, st, &work, &err, bytes);
  if (rc != SLRF_OK) return rc;
  if (mode == 1) oz_gram(n, X, ldx, k1, Y, ldy, k2, C, ldc, false, work, bytes, err, st);
  else gram(n, X, ldx, k1, Y, ldy, k2, C, ldc, false, static_cast<double *>(work), st);
  return ts_epilogue(st, work, err);
}

int slrf_tsgemm(int64_t n, const double *X, int ldx, int k1, const double *S, int lds, int k2, double *Z, int ldz,
                double alpha, double beta, int mode, void *stream) {
  if ((n > 0 && (!X || !Z)) || !S || ldx < k1 || lds < k2 || ldz < k2 || (n > 0 && X == Z)) return SLRF_EINVAL;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  void *work = nullptr;
  int *err = nullptr;
  const size_t bytes = mode == 1 ? oz_work_bytes(n, k1, k2) : 64;
  int rc = ts_prologue(n, k1, k2, mode, st, &work, &err, bytes);
  if (rc != SLRF_OK) return rc;
  if (mode == 1) oz_gemm(n, X, ldx, k1, S, lds, k2, Z, ldz, alpha, beta, work, bytes, err, st);
  else gemm_nn(n, X, ldx, k1, S, lds, k2, Z, ldz, alpha, beta, false, st);
  return ts_epilogue(st, work, err);
}

void slrf_destroy(slrf_ctx *ctx) {
  if (!ctx) return;
  if (ctx->st) cudaStreamSynchronize(ctx->st);
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  for (auto &e : ctx->ev)
    if (e) cudaEventDestroy(e);
  if (ctx->ev_in) cudaEventDestroy(ctx->ev_in);
  if (ctx->ev_out) cudaEventDestroy(ctx->ev_out);
  if (ctx->st) cudaStreamDestroy(ctx->st);
  for (void *p : ctx->allocs) cudaFree(p);
  if (ctx->h_iflags) cudaFreeHost(ctx->h_iflags);
  delete ctx;
}

int slrf_setup(slrf_ctx **out, const slrf_csr_pair *pc, double gamma, int block_L, const slrf_opts *opts,
               void *stream) {
  if (!out) return SLRF_EINVAL;
  *out = nullptr;
  if (!pc || !pc->rowptr || !pc->col || !pc->valA || !pc->valB || pc->n < 1 || pc->nnz < 1) return SLRF_EINVAL;
  if (!(gamma > 0) || block_L < 1 || block_L > pc->n) return SLRF_EINVAL;
  slrf_opts o;
  if (opts) o = *opts;
  else slrf_opts_default(&o);
  if (o.m < 1 || o.m > 32 || o.it_max < 1 || o.outer_max < 1 || o.refine_max < 1 || o.dense < 0 || o.dense > 1 ||
      o.it_adapt < 0 || o.it_adapt > 1 || o.precond < 0 || o.precond > 1 || o.group < 0 || o.group > 4 || o.bdiag < 0 ||
      o.bdiag > 1)
    return SLRF_EINVAL;
  if (block_L > 510) return SLRF_EINVAL;  // the projected eigensolver holds two rows of <= 512 in shared memory
  if (!(o.tol_inner >= 0) || !(o.tol_eig > 0)) return SLRF_EINVAL;
  if (pc->n > (int64_t)INT32_MAX) return SLRF_EINVAL;  // int32 column indices
  slrf_ctx *ctx = new (std::nothrow) slrf_ctx();
  if (!ctx) return SLRF_ENOMEM;
  auto fail = [&](int rc) {
    slrf_destroy(ctx);
    return rc;
  };
  ctx->ust = (cudaStream_t)stream;
  cudaGetDevice(&ctx->dev);
  if (cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, ctx->dev) != cudaSuccess ||
      ctx->sm_count < 1)
    return fail(SLRF_ECUDA);
  cocg_kernel_attrs();
  if (cudaStreamCreateWithFlags(&ctx->st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_out, cudaEventDisableTiming) != cudaSuccess)
    return fail(SLRF_ECUDA);
  // inputs may have been produced on the caller's stream
  cudaEventRecord(ctx->ev_in, ctx->ust);
  cudaStreamWaitEvent(ctx->st, ctx->ev_in, 0);
  ctx->n = pc->n;
  ctx->nnz = pc->nnz;
  ctx->gamma = gamma;
  ctx->L = block_L;
  ctx->o = o;
  ctx->m = o.m;
  ctx->mp = pow2_at_least(o.m);
  ctx->mixed = o.precision == 1;
  ctx->vec = ctx->mixed ? cocg_vec_csr<float>() : cocg_vec_csr<double>();  // until groups are built
  const int64_t n = ctx->n;
  const int L = block_L;
  // state sized for the widest lane layout (the grouped SpMM may be chosen below)
  const int kp = kpad_of(L, ctx->mp, ctx->mixed ? cocg_vec_max<float>() : cocg_vec_max<double>());
  ctx->Wmax = (size_t)kp * ctx->mp;
  // working-set estimate against free memory
  const size_t csz = ctx->mixed ? 8 : 16;
  const size_t state = 4 * (size_t)n * ctx->Wmax * csz;
  const size_t ntiles_max = ctx->Wmax / (32 * (ctx->mixed ? cocg_vec_csr<float>() : cocg_vec_csr<double>()));
  // run_cocg uses at most 4 row blocks per SM for any k <= L
  const size_t partial = (size_t)ctx->sm_count * 4 * ctx->Wmax * kNQ;
  const size_t blocks = 16 * sizeof(double) * (size_t)n * L;
  const size_t matrix = (size_t)ctx->nnz * (4 + 16 + (ctx->mixed ? 8 : 0)) + 8 * (size_t)(n + 1);
  const size_t refine = (ctx->mixed && o.refine_max > 1) ? 16 * (size_t)n * ctx->Wmax : 0;
  const size_t uacc = 8 * (size_t)n * (ctx->Wmax / ctx->mp) + (ctx->mixed ? 4 * (size_t)n * grp_real32_ld(L) : 0) +
                      8 * (size_t)n * grp_real64_ld(L);
  const size_t need = (state + blocks + matrix + refine + uacc) + 8 * partial + (64u << 20);
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return fail(SLRF_ECUDA);
  if (need > fr) return fail(SLRF_ENOMEM);
  int rc;
#define AL(p, c)                                \
  if ((rc = dalloc(ctx, &(p), (c))) != SLRF_OK) \
  return fail(rc)
  AL(ctx->rowptr, (size_t)n + 1);
  AL(ctx->col, (size_t)ctx->nnz + 8);
  AL(ctx->valA, (size_t)ctx->nnz + 4);
  AL(ctx->valB, (size_t)ctx->nnz + 4);
  if (cudaMemcpyAsync(ctx->rowptr, pc->rowptr, (n + 1) * sizeof(int64_t), cudaMemcpyDefault, ctx->st) != cudaSuccess ||
      cudaMemcpyAsync(ctx->col, pc->col, ctx->nnz * sizeof(int32_t), cudaMemcpyDefault, ctx->st) != cudaSuccess ||
      cudaMemcpyAsync(ctx->valA, pc->valA, ctx->nnz * sizeof(double), cudaMemcpyDefault, ctx->st) != cudaSuccess ||
      cudaMemcpyAsync(ctx->valB, pc->valB, ctx->nnz * sizeof(double), cudaMemcpyDefault, ctx->st) != cudaSuccess)
    return fail(SLRF_ECUDA);
  {
    // reject a malformed pattern before any kernel gathers through it
    int bad = 0;
    cudaMemsetAsync(ctx->valA + ctx->nnz, 0, sizeof(double), ctx->st);
    int *dflag = reinterpret_cast<int *>(ctx->valA + ctx->nnz);
    validate_csr(n, ctx->nnz, ctx->rowptr, ctx->col, dflag, ctx->sm_count * 4, ctx->st);
    if (cudaMemcpyAsync(&bad, dflag, sizeof(int), cudaMemcpyDeviceToHost, ctx->st) != cudaSuccess ||
        cudaStreamSynchronize(ctx->st) != cudaSuccess)
      return fail(SLRF_ECUDA);
    if (bad) return fail(SLRF_EINVAL);
  }
  AL(ctx->sig, 32);
  AL(ctx->wt, 32);
  AL(ctx->sig32, 32);
  if (o.precond) {
    // Jacobi preconditioner: D^-1/2 and the scaled values of both matrices
    AL(ctx->dsc, (size_t)n);
    AL(ctx->valAs, (size_t)ctx->nnz + 4);
    AL(ctx->valBs, (size_t)ctx->nnz + 4);
    int bad = 0;
    int *dflag = reinterpret_cast<int *>(ctx->valAs + ctx->nnz);
    cudaMemsetAsync(dflag, 0, sizeof(int), ctx->st);
    jacobi_scaling(n, ctx->rowptr, ctx->col, ctx->valA, ctx->valB, ctx->dsc, ctx->valAs, ctx->valBs, dflag, ctx->st);
    if (cudaMemcpyAsync(&bad, dflag, sizeof(int), cudaMemcpyDeviceToHost, ctx->st) != cudaSuccess ||
        cudaStreamSynchronize(ctx->st) != cudaSuccess)
      return fail(SLRF_ECUDA);
    if (bad) return fail(SLRF_EINVAL);
  }
  if (ctx->mixed) {
    AL(ctx->valA32, (size_t)ctx->nnz + 4);
    AL(ctx->valB32, (size_t)ctx->nnz + 4);
    const unsigned gb = (unsigned)((ctx->nnz + 255) / 256);
    to_float_kernel<<<gb, 256, 0, ctx->st>>>(ctx->nnz, cocg_valA(ctx), ctx->valA32);
    to_float_kernel<<<gb, 256, 0, ctx->st>>>(ctx->nnz, cocg_valB(ctx), ctx->valB32);
  }
  if ((rc = setup_groups(ctx)) != SLRF_OK) return fail(rc);
  AL(ctx->iflags, 16);
  if (cudaMallocHost(&ctx->h_iflags, 16 * sizeof(int)) != cudaSuccess) return fail(SLRF_ENOMEM);
  cudaMemsetAsync(ctx->iflags, 0, 16 * sizeof(int), ctx->st);
  // pole table
  if (o.poles && o.weights) {
    double2 hs[32], hw[32];
    for (int j = 0; j < ctx->mp; ++j) {
      if (j < o.m) {
        hs[j] = make_double2(o.poles[2 * j], o.poles[2 * j + 1]);
        hw[j] = make_double2(o.weights[2 * j], o.weights[2 * j + 1]);
      } else {
        hs[j] = make_double2(gamma, gamma);
        hw[j] = make_double2(0, 0);
      }
    }
    if (cudaMemcpy(ctx->sig, hs, ctx->mp * sizeof(double2), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(ctx->wt, hw, ctx->mp * sizeof(double2), cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(SLRF_ECUDA);
  } else {
    design_poles(o.m, ctx->mp, gamma, o.alpha, o.beta, o.band, ctx->sig, ctx->wt, ctx->iflags + 8, ctx->st);
  }
  to_float2_kernel<<<1, 32, 0, ctx->st>>>(ctx->mp, ctx->sig, ctx->sig32);
  {
    double2 hs[32], hw[32];
    int hst[16];
    if (cudaMemcpyAsync(hs, ctx->sig, ctx->mp * sizeof(double2), cudaMemcpyDeviceToHost, ctx->st) != cudaSuccess ||
        cudaMemcpyAsync(hw, ctx->wt, ctx->mp * sizeof(double2), cudaMemcpyDeviceToHost, ctx->st) != cudaSuccess ||
        cudaMemcpyAsync(hst, ctx->iflags, 16 * sizeof(int), cudaMemcpyDeviceToHost, ctx->st) != cudaSuccess ||
        cudaStreamSynchronize(ctx->st) != cudaSuccess)
      return fail(SLRF_ECUDA);
    if (hst[8] != 0) return fail(SLRF_EINVAL);
    for (int j = 0; j < ctx->m; ++j) {
      ctx->h_sig[2 * j] = hs[j].x; ctx->h_sig[2 * j + 1] = hs[j].y;
      ctx->h_wt[2 * j] = hw[j].x; ctx->h_wt[2 * j + 1] = hw[j].y;
    }
  }
  // COCG state
  AL(ctx->cd, n * ctx->Wmax * csz);
  AL(ctx->cr, n * ctx->Wmax * csz);
  AL(ctx->cp, n * ctx->Wmax * csz);
  AL(ctx->cq, n * ctx->Wmax * csz);
  AL(ctx->partial, partial);
  AL(ctx->counters, ntiles_max + 32);
  cudaMemsetAsync(ctx->counters, 0, (ntiles_max + 32) * sizeof(unsigned), ctx->st);
  AL(ctx->ws, ctx->Wmax);
  AL(ctx->cfac, ctx->Wmax);
  AL(ctx->coefV, (size_t)L);
  AL(ctx->gscale, (size_t)L);
  AL(ctx->gmax, (size_t)L);
  if (ctx->mixed && o.refine_max > 1) {
    AL(ctx->D64, (size_t)n * ctx->Wmax);
    AL(ctx->r00, ctx->Wmax);
  }
  AL(ctx->uacc, (size_t)n * (ctx->Wmax / ctx->mp));
  if (ctx->mixed) AL(ctx->x32, (size_t)n * grp_real32_ld(L));
  AL(ctx->x64, (size_t)n * grp_real64_ld(L));
  if (ctx->dsc != nullptr) {
    AL(ctx->dsqrt, (size_t)n);
    recip_kernel<<<(unsigned)((n + 255) / 256), 256, 0, ctx->st>>>(n, ctx->dsc, ctx->dsqrt);
  }
  // real blocks
  const size_t nb = (size_t)n * L;
  AL(ctx->V, nb); AL(ctx->AV, nb); AL(ctx->BV, nb);
  AL(ctx->G, nb); AL(ctx->AG, nb); AL(ctx->BG, nb);
  AL(ctx->U, nb); AL(ctx->U2, nb); AL(ctx->BU, nb);
  AL(ctx->Vt, nb); AL(ctx->AVt, nb); AL(ctx->BVt, nb);
  AL(ctx->X, nb); AL(ctx->BX, nb);
  const size_t LL = (size_t)L * L;
  AL(ctx->Gm, LL); AL(ctx->Rinv, LL); AL(ctx->Hm, LL); AL(ctx->Sm, LL); AL(ctx->Wm, LL);
  AL(ctx->theta, L); AL(ctx->theta_act, L); AL(ctx->res, L); AL(ctx->res_paper, L); AL(ctx->sgn, L);
  AL(ctx->Theta, L); AL(ctx->Res, L);
  AL(ctx->dst_x, L); AL(ctx->dst_v, L);
  // gram() splits rows into at most 64 chunks of k1 x k2 <= L x L partial tiles
  ctx->work_doubles = std::max({(size_t)64 * L * L, ritz_work_doubles(n, L), (size_t)4 * L});
  AL(ctx->work, ctx->work_doubles);
  if (o.dense) {
    ctx->ozwork_bytes = oz_work_bytes(n, L, L);
    AL(ctx->ozwork, ctx->ozwork_bytes);
  }
  {
    const int kk = L + (L & 1) < 2 ? 2 : L + (L & 1);
    AL(ctx->jw.A, (size_t)kk * kk);
    AL(ctx->jw.Vt, (size_t)kk * kk);
    AL(ctx->jw.rot, 4 * (size_t)kk);
    AL(ctx->jw.flags, 4);
    AL(ctx->jw.bar, 4);
    ctx->jw.err = ctx->iflags + 9;
  }
#undef AL
  for (auto &e : ctx->ev)
    if (cudaEventCreate(&e) != cudaSuccess) return fail(SLRF_ECUDA);
  if (o.autotune) {
    const int arc = ctx->mixed ? autotune_rows<float>(ctx) : autotune_rows<double>(ctx);
    if (arc != SLRF_OK) return fail(arc);
  }
  if (cudaStreamSynchronize(ctx->st) != cudaSuccess || cudaGetLastError() != cudaSuccess) return fail(SLRF_ECUDA);
  *out = ctx;
  return SLRF_OK;
}

int slrf_get_poles(slrf_ctx *ctx, int *m_out, double *sigma, double *w) {
  if (!ctx) return SLRF_EINVAL;
  if (m_out) *m_out = ctx->m;
  if (sigma) memcpy(sigma, ctx->h_sig, 2 * ctx->m * sizeof(double));
  if (w) memcpy(w, ctx->h_wt, 2 * ctx->m * sizeof(double));
  return SLRF_OK;
}

int slrf_filter_apply(slrf_ctx *ctx, const double *X, int k, const double *theta, double *U) {
  if (!ctx) return SLRF_EINVAL;
  if (ctx->status != SLRF_OK) return SLRF_ESTATE;
  if (!X || !U || k < 1 || k > ctx->L || X == U) return SLRF_EINVAL;
  StreamScope sc(ctx);
  return filter_impl(ctx, X, k, k, theta, nullptr, nullptr, U, k, false);
}

int slrf_format(const slrf_ctx *ctx, int *group, int *bdiag, int *lane_width) {
  if (!ctx) return SLRF_EINVAL;
  if (group) *group = ctx->grp;
  if (bdiag) *bdiag = ctx->bdiag;
  if (lane_width) *lane_width = ctx->vec;
  return SLRF_OK;
}

int slrf_apply(slrf_ctx *ctx, const double *X, int k, double *AX, double *BX, int fp32) {
  if (!ctx) return SLRF_EINVAL;
  if (ctx->status != SLRF_OK) return SLRF_ESTATE;
  if (!X || k < 1 || k > ctx->L || (!AX && !BX) || X == AX || X == BX || AX == BX) return SLRF_EINVAL;
  StreamScope sc(ctx);
  const int64_t n = ctx->n;
  if (fp32 && ctx->mixed && ctx->grp > 1) {
    // FP32 records (Jacobi-scaled values when the preconditioner is on: scale both sides by D^1/2)
    spmm_grp_real32(n, ctx->grp, ctx->ngroups, ctx->gptr, ctx->grec, ctx->iflags + 15, grp_real_blocks(ctx), X, k,
                    k, ctx->dsqrt, ctx->x32, AX, BX, k, ctx->dsqrt, ctx->st, ctx->bdiag != 0);
  } else if (fp32) {
    spmm_ab32(n, ctx->rowptr, ctx->col, ctx->valA, ctx->valB, X, k, k, AX, BX, k, ctx->st);
  } else {
    real_products64(ctx, X, k, k, AX, BX, k, ctx->st);
  }
  CKL();
  return SLRF_OK;
}

int slrf_filter_timing(slrf_ctx *ctx, const double *X, int k, const double *theta, double *U, double *ms,
                       int *launches) {
  if (!ctx) return SLRF_EINVAL;
  if (ctx->status != SLRF_OK) return SLRF_ESTATE;
  if (!X || !U || !ms || k < 1 || k > ctx->L || X == U) return SLRF_EINVAL;
  StreamScope sc(ctx);
  FilterTiming tm;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  cudaEventRecord(e0, ctx->st);
  const int rc = filter_impl(ctx, X, k, k, theta, nullptr, nullptr, U, k, false, &tm);
  cudaEventRecord(e1, ctx->st);
  CK(cudaEventSynchronize(e1));
  float tot = 0;
  cudaEventElapsedTime(&tot, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != SLRF_OK) return rc;
  ms[0] = tot;
  ms[1] = tm.ms_spmm;
  ms[2] = tm.ms_update;
  ms[3] = tm.ms_init;
  if (launches) {
    launches[0] = tm.n_spmm;
    launches[1] = tm.n_update;
  }
  return SLRF_OK;
}

int slrf_filter_stats(slrf_ctx *ctx, int *iters, double *relres, int *breakdown) {
  if (!ctx) return SLRF_EINVAL;
  if (ctx->status != SLRF_OK) return SLRF_ESTATE;
  const int W = ctx->last_W, k = ctx->last_k;
  if (W == 0) return SLRF_EINVAL;
  StreamScope sc(ctx);
  std::vector<WScal> h(W);
  CK(cudaMemcpyAsync(h.data(), ctx->ws, W * sizeof(WScal), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  for (int c = 0; c < k; ++c)
    for (int j = 0; j < ctx->m; ++j) {
      const WScal &s = h[c * ctx->mp + j];
      const int o = j * k + c;
      if (iters) iters[o] = s.iters;
      if (relres) relres[o] = s.r0n2 > 0 ? std::sqrt(s.rn2 / s.r0n2) : 0.0;
      if (breakdown) breakdown[o] = s.brk;
    }
  return SLRF_OK;
}

int slrf_rayleigh_ritz(slrf_ctx *ctx, double *U, int k, const double *X, const double *BX, int n_conv, int ldx,
                       double *V, double *theta, double *res) {
  if (!ctx) return SLRF_EINVAL;
  if (ctx->status != SLRF_OK) return SLRF_ESTATE;
  if (!U || !V || !theta || !res || k < 1 || k > ctx->L || n_conv < 0) return SLRF_EINVAL;
  if (n_conv > 0 && (!X || !BX || ldx < n_conv)) return SLRF_EINVAL;
  const int64_t n = ctx->n;
  const int L = ctx->L;
  StreamScope sc(ctx);
  // stage into library buffers with leading dimension L
  copy_block(n, k, U, k, ctx->U, L, ctx->st);
  if (n_conv > 0) {
    if (n_conv > L) return SLRF_EINVAL;
    copy_block(n, n_conv, X, ldx, ctx->X, L, ctx->st);
    copy_block(n, n_conv, BX, ldx, ctx->BX, L, ctx->st);
  }
  CK(cudaMemsetAsync(ctx->iflags + 4, 0, sizeof(int), ctx->st));
  int rc = rr_impl(ctx, ctx->U, k, ctx->X, ctx->BX, n_conv, L, true);
  if (rc != SLRF_OK) return rc;
  int hf[16];
  CK(cudaMemcpyAsync(hf, ctx->iflags, 16 * sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (hf[9] != 0 || hf[13] != 0) return SLRF_ETIMEOUT;
  if (hf[4] != 0) return SLRF_ECHOL;
  // apply the sign convention and hand out V, theta, res
  {
    // dst_v = identity, no locking: gather into Vt-sized outputs via lock_gather with cap 0
    std::vector<int> idv(k), idx(k, -1);
    for (int c = 0; c < k; ++c) idv[c] = c;
    CK(cudaMemcpyAsync(ctx->dst_v, idv.data(), k * sizeof(int), cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(ctx->dst_x, idx.data(), k * sizeof(int), cudaMemcpyHostToDevice, ctx->st));
    lock_gather(n, k, ctx->Vt, ctx->AVt, ctx->BVt, L, ctx->sgn, ctx->dst_x, ctx->dst_v, nullptr, nullptr, L, ctx->V,
                ctx->AV, ctx->BV, L, ctx->st);
    copy_block(n, k, ctx->V, L, V, k, ctx->st);
    copy_block(n, k, ctx->U, L, U, k, ctx->st);
    CK(cudaMemcpyAsync(theta, ctx->theta, k * sizeof(double), cudaMemcpyDeviceToDevice, ctx->st));
    CK(cudaMemcpyAsync(res, ctx->res, k * sizeof(double), cudaMemcpyDeviceToDevice, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
  }
  CKL();
  return SLRF_OK;
}

int slrf_solve(slrf_ctx *ctx, const double *V0, int cap, int *n_found, double *evals, double *Xo, double *resid,
               slrf_stats *stats) {
  if (!ctx) return SLRF_EINVAL;
  if (ctx->status != SLRF_OK) return SLRF_ESTATE;
  if (!n_found || cap < 0 || (cap > 0 && (!evals || !Xo || !resid))) return SLRF_EINVAL;
  *n_found = 0;
  StreamScope sc(ctx);
  const cudaStream_t st = ctx->st;
  const int64_t n = ctx->n;
  const int L = ctx->L;
  slrf_stats S{};
  if (V0) copy_block(n, L, V0, L, ctx->V, L, st);
  else gaussian_block(n, L, ctx->o.seed, ctx->V, L, st);
  CK(cudaMemsetAsync(ctx->iflags, 0, 16 * sizeof(int), st));
  if (V0) {
    check_finite((int64_t)n * L, ctx->V, ctx->iflags + 5, st);
    CK(cudaMemcpyAsync(ctx->h_iflags, ctx->iflags, 16 * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (ctx->h_iflags[5]) return SLRF_ENAN;
  }
  int k = L, nconv = 0, quiet = 0, status = SLRF_ENOCONV, outer = 0;
  ctx->launches = V0 ? 2 : 1;
  ctx->it_cur = ctx->o.it_max;
  ctx->unres_streak = 0;
  struct ItReset {
    slrf_ctx *c;
    ~ItReset() { c->it_cur = 0; }  // filter_apply outside a solve uses opts.it_max
  } it_reset{ctx};
  bool have_ritz = false;
  float ms_f = 0, ms_d = 0;
  CK(cudaEventRecord(ctx->ev[0], st));
  for (outer = 1; outer <= ctx->o.outer_max; ++outer) {
    const bool warm = have_ritz && ctx->o.warm_start;
    CK(cudaEventRecord(ctx->ev[1], st));
    int rc = filter_impl(ctx, ctx->V, L, k, warm ? ctx->theta_act : nullptr, warm ? ctx->AV : nullptr,
                         warm ? ctx->BV : nullptr, ctx->U, L, true);
    if (rc != SLRF_OK) return rc;
    CK(cudaEventRecord(ctx->ev[2], st));
    count_iters_kernel<<<1, 256, 0, st>>>(ctx->last_W, ctx->ws, ctx->iflags + 6);
    ctx->launches += 1 + 2;  // + lock_decide, lock_gather below
    S.column_solves += (int64_t)ctx->m * k;
    rc = rr_impl(ctx, ctx->U, k, ctx->X, ctx->BX, ctx->o.lock ? nconv : 0, L);
    if (rc != SLRF_OK) return rc;
    // lock decision, compaction (the locking step of Alg. 2)
    lock_decide(k, ctx->theta, ctx->res, ctx->gamma, ctx->o.tol_eig, ctx->o.lock, L, ctx->iflags, ctx->dst_x,
                ctx->dst_v, ctx->Theta, ctx->Res, ctx->theta_act, st, ctx->iflags + 14);
    lock_gather(n, k, ctx->Vt, ctx->AVt, ctx->BVt, L, ctx->sgn, ctx->dst_x, ctx->dst_v, ctx->X, ctx->BX, L, ctx->V,
                ctx->AV, ctx->BV, L, st);
    CKL();
    CK(cudaEventRecord(ctx->ev[3], st));
    CK(cudaMemcpyAsync(ctx->h_iflags, ctx->iflags, 16 * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    {
      float a = 0, b = 0;
      cudaEventElapsedTime(&a, ctx->ev[1], ctx->ev[2]);
      cudaEventElapsedTime(&b, ctx->ev[2], ctx->ev[3]);
      ms_f += a;
      ms_d += b;
    }
    const int *hf = ctx->h_iflags;
    // hf[15]: 1 a bounded wait gave up; 2-4 inconsistent group records or update buffers
    if (hf[9] != 0 || hf[13] != 0 || hf[15] == 1) { status = SLRF_ETIMEOUT; break; }
    if (hf[15] != 0) { status = SLRF_EINVAL; break; }
    if (hf[4] != 0) { status = SLRF_ECHOL; break; }
    nconv = hf[0];
    k = hf[1];
    const int pending = hf[2];
    have_ritz = true;
    adapt_it(ctx, hf[14] != 0);
    if (k < 1) { status = SLRF_OK; break; }
    quiet = pending ? 0 : quiet + 1;
    if (quiet >= 2 && (ctx->o.nev <= 0 || nconv >= ctx->o.nev)) { status = SLRF_OK; break; }
  }
  if (outer > ctx->o.outer_max) outer = ctx->o.outer_max;
  CK(cudaEventRecord(ctx->ev[3], st));
  CK(cudaEventSynchronize(ctx->ev[3]));
  {
    float tt = 0;
    cudaEventElapsedTime(&tt, ctx->ev[0], ctx->ev[3]);
    S.ms_total = tt;
  }
  S.ms_filter = ms_f;
  S.ms_dense = ms_d;
  S.outer_iters = outer;
  S.n_conv = nconv;
  S.breakdowns = ctx->h_iflags[6];
  S.column_iterations = ctx->h_iflags[7];
  S.kernel_launches = ctx->launches + (nconv > 0 ? 2 : 0);
  if (!ctx->o.lock && status == SLRF_OK) {
    // basic method: the wanted converged Ritz pairs of the last step are the result
    CK(cudaMemsetAsync(ctx->iflags, 0, sizeof(int), st));
    lock_decide(k, ctx->theta, ctx->res, ctx->gamma, ctx->o.tol_eig, 1, L, ctx->iflags, ctx->dst_x, ctx->dst_v,
                ctx->Theta, ctx->Res, ctx->theta_act, st);
    lock_gather(n, k, ctx->Vt, ctx->AVt, ctx->BVt, L, ctx->sgn, ctx->dst_x, ctx->dst_v, ctx->X, ctx->BX, L, ctx->U2,
                ctx->G, ctx->AG, L, st);
    CK(cudaMemcpyAsync(ctx->h_iflags, ctx->iflags, 16 * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    nconv = ctx->h_iflags[0];
    S.n_conv = nconv;
  }
  *n_found = nconv;
  const int cnt = std::min(nconv, cap);
  if (nconv > 0 && cnt > 0) {
    final_rank_kernel<<<1, 256, 0, st>>>(nconv, ctx->Theta, ctx->dst_x);
    const int64_t tot = n * nconv;
    final_gather_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, nconv, cnt, ctx->dst_x, ctx->Theta, ctx->Res,
                                                                       ctx->X, L, evals, Xo, cap, resid);
    CKL();
    CK(cudaStreamSynchronize(st));
  }
  if (stats) *stats = S;
  if (status != SLRF_OK) return status;
  if (nconv > cap) return SLRF_ETRUNC;
  return SLRF_OK;
}

int slrf_solve_host(const slrf_csr_pair *ph, double gamma, int block_L, const slrf_opts *opts, const double *V0,
                    int cap, int *n_found, double *evals, double *X, double *resid, slrf_stats *stats) {
  if (!ph || !ph->rowptr || !ph->col || !ph->valA || !ph->valB || ph->n < 1 || ph->nnz < 1 || !n_found)
    return SLRF_EINVAL;
  slrf_ctx *ctx = nullptr;  // for CK
  const int64_t n = ph->n, nnz = ph->nnz;
  cudaStream_t st;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return SLRF_ECUDA;
  void *buf = nullptr;
  const size_t bytes = (n + 1) * 8 + nnz * 4 + 2 * nnz * 8 + (V0 ? (size_t)n * block_L * 8 : 0) +
                       (size_t)cap * 8 * 2 + (size_t)n * cap * 8 + 256;
  if (cudaMalloc(&buf, bytes) != cudaSuccess) {
    cudaStreamDestroy(st);
    return SLRF_ENOMEM;
  }
  char *b = (char *)buf;
  auto take = [&](size_t s) { char *p = b; b += (s + 15) / 16 * 16; return p; };
  int64_t *drp = (int64_t *)take((n + 1) * 8);
  int32_t *dcol = (int32_t *)take(nnz * 4);
  double *dA = (double *)take(nnz * 8), *dB = (double *)take(nnz * 8);
  double *dV0 = V0 ? (double *)take((size_t)n * block_L * 8) : nullptr;
  double *dev_e = (double *)take((size_t)cap * 8), *dev_r = (double *)take((size_t)cap * 8);
  double *dX = (double *)take((size_t)n * cap * 8);
  int rc = SLRF_OK;
  if (cudaMemcpyAsync(drp, ph->rowptr, (n + 1) * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(dcol, ph->col, nnz * 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(dA, ph->valA, nnz * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(dB, ph->valB, nnz * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      (V0 && cudaMemcpyAsync(dV0, V0, (size_t)n * block_L * 8, cudaMemcpyHostToDevice, st) != cudaSuccess))
    rc = SLRF_ECUDA;
  slrf_csr_pair dp{n, nnz, drp, dcol, dA, dB};
  if (rc == SLRF_OK) rc = slrf_setup(&ctx, &dp, gamma, block_L, opts, st);
  if (rc == SLRF_OK) {
    rc = slrf_solve(ctx, dV0, cap, n_found, dev_e, dX, dev_r, stats);
    const int cnt = std::min(*n_found, cap);
    if ((rc == SLRF_OK || rc == SLRF_ETRUNC) && cnt > 0) {
      if (cudaMemcpyAsync(evals, dev_e, cnt * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaMemcpyAsync(resid, dev_r, cnt * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaMemcpyAsync(X, dX, (size_t)n * cap * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        rc = SLRF_ECUDA;
    }
  }
  slrf_destroy(ctx);
  cudaStreamSynchronize(st);
  cudaFree(buf);
  cudaStreamDestroy(st);
  return rc;
}

int slrf_setup_batched(slrf_batch **out, int P, const slrf_csr_pair *pencils, const double *gammas, const int *blocks,
                       const slrf_opts *opts, void *stream) {
  if (!out) return SLRF_EINVAL;
  *out = nullptr;
  if (P < 1 || !pencils || !gammas || !blocks) return SLRF_EINVAL;
  slrf_batch *b = new (std::nothrow) slrf_batch();
  if (!b) return SLRF_ENOMEM;
  b->P = P;
  b->ust = (cudaStream_t)stream;
  b->c.assign(P, nullptr);
  b->ev_p.assign(P, nullptr);
  // the persistent batched launches gather through the plain CSR pattern of each problem
  slrf_opts ob;
  if (opts) ob = *opts;
  else slrf_opts_default(&ob);
  ob.group = 1;
  for (int p = 0; p < P; ++p) {
    const int rc = slrf_setup(&b->c[p], &pencils[p], gammas[p], blocks[p], &ob, stream);
    if (rc != SLRF_OK) {
      batch_free(b);
      return rc;
    }
  }
  b->mixed = b->c[0]->mixed;
  const size_t asz = std::max(sizeof(CocgArgs<double>), sizeof(CocgArgs<float>));
  if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_b, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreate(&b->ev_t0) != cudaSuccess || cudaEventCreate(&b->ev_t1) != cudaSuccess ||
      cudaEventCreate(&b->ev_f0) != cudaSuccess || cudaEventCreate(&b->ev_f1) != cudaSuccess ||
      cudaMalloc(&b->dargs, P * asz) != cudaSuccess || cudaMalloc(&b->dprefix, (P + 1) * sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&b->hargs, P * asz) != cudaSuccess || cudaMallocHost(&b->hprefix, (P + 1) * sizeof(int)) != cudaSuccess) {
    batch_free(b);
    return SLRF_ECUDA;
  }
  for (int p = 0; p < P; ++p)
    if (cudaEventCreateWithFlags(&b->ev_p[p], cudaEventDisableTiming) != cudaSuccess) {
      batch_free(b);
      return SLRF_ECUDA;
    }
  *out = b;
  return SLRF_OK;
}

void slrf_destroy_batched(slrf_batch *b) { batch_free(b); }

int slrf_solve_batched(slrf_batch *b, const double *const *V0, const int *caps, int *n_found, double *const *evals,
                       double *const *Xo, double *const *resid, int *status, slrf_stats *stats) {
  if (!b || !caps || !n_found || !status) return SLRF_EINVAL;
  const int P = b->P;
  for (int p = 0; p < P; ++p) {
    if (b->c[p]->status != SLRF_OK) return SLRF_ESTATE;
    if (caps[p] < 0 || (caps[p] > 0 && (!evals || !Xo || !resid || !evals[p] || !Xo[p] || !resid[p]))) return SLRF_EINVAL;
  }
  slrf_ctx *ctx = nullptr;  // for CK
  // fork: every problem stream and the batch stream start after the caller's stream
  CK(cudaEventRecord(b->ev_in, b->ust));
  CK(cudaStreamWaitEvent(b->st, b->ev_in, 0));
  for (auto *c : b->c) CK(cudaStreamWaitEvent(c->st, b->ev_in, 0));
  CK(cudaEventRecord(b->ev_t0, b->st));
  std::vector<int> kk(P), nconv(P, 0), quiet(P, 0), outer_of(P, 0);
  std::vector<char> done(P, 0), warm(P, 0);
  std::vector<int> st_p(P, SLRF_ENOCONV);
  int64_t launches = 0;
  slrf_stats S{};
  for (int p = 0; p < P; ++p) {
    slrf_ctx *c = b->c[p];
    c->launches = 0;
    kk[p] = c->L;
    if (V0 && V0[p]) copy_block(c->n, c->L, V0[p], c->L, c->V, c->L, c->st);
    else gaussian_block(c->n, c->L, c->o.seed + p, c->V, c->L, c->st);
    CK(cudaMemsetAsync(c->iflags, 0, 16 * sizeof(int), c->st));
    c->it_cur = c->o.it_max;
    c->unres_streak = 0;
    launches += 1;
  }
  struct ItReset {
    slrf_batch *b;
    ~ItReset() { for (auto *c : b->c) c->it_cur = 0; }
  } it_reset{b};
  const int outer_max = b->c[0]->o.outer_max;
  int outer = 0;
  double ms_f = 0.0;  // device time of the batched COCG launches
  for (outer = 1; outer <= outer_max; ++outer) {
    std::vector<int> act;
    for (int p = 0; p < P; ++p)
      if (!done[p]) act.push_back(p);
    if (act.empty()) break;
    const int rc = b->mixed ? batch_outer_filter<float>(b, act, kk, warm, launches)
                            : batch_outer_filter<double>(b, act, kk, warm, launches);
    if (rc != SLRF_OK) return rc;
    for (int p : act) {
      slrf_ctx *c = b->c[p];
      const int k = kk[p];
      count_iters_kernel<<<1, 256, 0, c->st>>>(c->last_W, c->ws, c->iflags + 6);
      S.column_solves += (int64_t)c->m * k;
      int r2 = rr_impl(c, c->U, k, c->X, c->BX, c->o.lock ? nconv[p] : 0, c->L);
      if (r2 != SLRF_OK) return r2;
      lock_decide(k, c->theta, c->res, c->gamma, c->o.tol_eig, c->o.lock, c->L, c->iflags, c->dst_x, c->dst_v,
                  c->Theta, c->Res, c->theta_act, c->st, c->iflags + 14);
      lock_gather(c->n, k, c->Vt, c->AVt, c->BVt, c->L, c->sgn, c->dst_x, c->dst_v, c->X, c->BX, c->L, c->V, c->AV,
                  c->BV, c->L, c->st);
      CK(cudaMemcpyAsync(c->h_iflags, c->iflags, 16 * sizeof(int), cudaMemcpyDeviceToHost, c->st));
      launches += 3;
    }
    {
      float f = 0.f;
      CK(cudaEventSynchronize(b->ev_f1));
      if (cudaEventElapsedTime(&f, b->ev_f0, b->ev_f1) == cudaSuccess) ms_f += f;
    }
    for (int p : act) {
      slrf_ctx *c = b->c[p];
      CK(cudaStreamSynchronize(c->st));
      const int *hf = c->h_iflags;
      outer_of[p] = outer;
      if (hf[9] != 0 || hf[13] != 0 || hf[15] == 1) { st_p[p] = SLRF_ETIMEOUT; done[p] = 1; continue; }
      if (hf[15] != 0) { st_p[p] = SLRF_EINVAL; done[p] = 1; continue; }
      if (hf[4] != 0) { st_p[p] = SLRF_ECHOL; done[p] = 1; continue; }
      nconv[p] = hf[0];
      kk[p] = hf[1];
      warm[p] = c->o.warm_start ? 1 : 0;
      if (kk[p] < 1) { st_p[p] = SLRF_OK; done[p] = 1; continue; }
      adapt_it(c, hf[14] != 0);
      quiet[p] = hf[2] ? 0 : quiet[p] + 1;
      if (quiet[p] >= 2 && (c->o.nev <= 0 || nconv[p] >= c->o.nev)) { st_p[p] = SLRF_OK; done[p] = 1; }
    }
  }
  int worst = SLRF_OK;
  for (int p = 0; p < P; ++p) {
    slrf_ctx *c = b->c[p];
    n_found[p] = nconv[p];
    const int cnt = std::min(nconv[p], caps[p]);
    if (nconv[p] > 0 && cnt > 0) {
      final_rank_kernel<<<1, 256, 0, c->st>>>(nconv[p], c->Theta, c->dst_x);
      const int64_t tot = c->n * nconv[p];
      final_gather_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, c->st>>>(c->n, nconv[p], cnt, c->dst_x, c->Theta,
                                                                          c->Res, c->X, c->L, evals[p], Xo[p],
                                                                          caps[p], resid[p]);
      launches += 2;
    }
    if (st_p[p] == SLRF_OK && nconv[p] > caps[p]) st_p[p] = SLRF_ETRUNC;
    status[p] = st_p[p];
    if (st_p[p] != SLRF_OK && worst == SLRF_OK) worst = st_p[p];
    CK(cudaEventRecord(b->ev_p[p], c->st));
    CK(cudaStreamWaitEvent(b->st, b->ev_p[p], 0));
    S.column_iterations += c->h_iflags[7];
    S.breakdowns += c->h_iflags[6];
    S.n_conv += nconv[p];
    launches += c->launches;
  }
  CK(cudaEventRecord(b->ev_t1, b->st));
  CK(cudaStreamWaitEvent(b->ust, b->ev_t1, 0));
  CK(cudaEventSynchronize(b->ev_t1));
  float tt = 0;
  cudaEventElapsedTime(&tt, b->ev_t0, b->ev_t1);
  S.ms_total = tt;
  S.ms_filter = ms_f;  // the batched COCG; the per-problem starts and dense phases are the rest
  S.ms_dense = tt - ms_f;
  S.outer_iters = outer > outer_max ? outer_max : outer - 1;
  S.kernel_launches = launches;
  if (stats) *stats = S;
  return worst;
}

int slrf_eig_grad(slrf_ctx *ctx, int k, const double *evals, const double *X, int ldx, const double *g_eval,
                  const double *g_X, double *gA, double *gB) {
  if (!ctx) return SLRF_EINVAL;
  if (ctx->status != SLRF_OK) return SLRF_ESTATE;
  if (k < 1 || !evals || !X || ldx < k || !g_eval || !gA || !gB) return SLRF_EINVAL;
  StreamScope sc(ctx);
  if (g_X == nullptr) {
    const int rc = eig_grad_values(ctx->n, ctx->rowptr, ctx->col, k, evals, X, ldx, g_eval, gA, gB, ctx->st);
    if (rc != SLRF_OK) ctx->status = rc;
    return rc;
  }
  if (k > ctx->L) return SLRF_EINVAL;
  // eigenvector terms: scratch n x k blocks (leading dimension k) from the context
  const int64_t n = ctx->n;
  const double *Xk = X;
  if (ldx != k) {
    copy_block(n, k, X, ldx, ctx->BX, k, ctx->st);
    Xk = ctx->BX;
  }
  const size_t aw = adj_work_doubles(n, k);
  if (2 * aw > ctx->work_doubles) return SLRF_EINVAL;
  AdjBuffers bf{ctx->V, ctx->AV, ctx->BV, ctx->G, ctx->AG, ctx->BG, ctx->U, ctx->U2, ctx->BU, ctx->Vt, ctx->AVt,
                ctx->BVt, ctx->work, ctx->work + aw, reinterpret_cast<MinresScal *>(ctx->partial), ctx->iflags + 10};
  int notconv = 0;
  const double tol = std::max(ctx->o.tol_inner, 1e-12);
  const int rc = eig_grad_vectors(n, ctx->rowptr, ctx->col, ctx->valA, ctx->valB, k, evals, Xk, g_eval, g_X, gA, gB,
                                  bf, 20000, tol, ctx->h_iflags + 12, &notconv, ctx->st);
  if (rc != SLRF_OK) {
    ctx->status = rc;
    return rc;
  }
  return notconv ? SLRF_ENOCONV : SLRF_OK;
}

}  // extern "C"
