// slrf_filter_apply_static: the FP64 filter apply of slrf_filter_apply without a context
// and without any device allocation.
//
// Callers that cannot allocate device memory -- code running under a framework's own
// memory pool or budget, a plugin that may not call cudaMalloc after initialisation, or
// work enqueued from a context where allocation is forbidden -- still need the filter.
// This entry point keeps every scratch buffer (pole table, the real start sweep, the
// COCG state d, r, p, q, the reduction partials and per-column scalars) in one
// file-scope static device array, SLRF_STATIC_ARENA_BYTES large, that every GPU which
// loads the library holds until the process exits.  The caller passes the pencil, the
// block, the optional Ritz values and the output, all in device memory.
//
// Host code must not pass `arena` itself to a kernel: in host code that name is a
// host-side stand-in, not a device address.  The device address is obtained once per
// device with cudaGetSymbolAddress (with that device current) on the first call made
// on it, and cached.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "../../include/slrf.h"
#include "cocg.cuh"
#include "dense.cuh"

namespace slrf {

static __device__ __align__(256) unsigned char arena[SLRF_STATIC_ARENA_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_arena[kMaxDevices] = {};

// device address of `arena` for the current device (set-up on the first call)
int arena_address(unsigned char **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SLRF_ECUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_arena[dev] == nullptr) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, arena) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return SLRF_ECUDA;
    }
    g_arena[dev] = static_cast<unsigned char *>(p);
  }
  *out = g_arena[dev];
  return SLRF_OK;
}

struct Carver {
  unsigned char *base;
  size_t off = 0;
  template <typename T> T *take(size_t count) {
    off = (off + 255) / 256 * 256;
    T *p = reinterpret_cast<T *>(base + off);
    off += count * sizeof(T);
    return p;
  }
};

int pow2_at_least(int m) {
  int p = 1;
  while (p < m) p <<= 1;
  return p;
}
}  // namespace

}  // namespace slrf

using namespace slrf;

extern "C" int slrf_filter_apply_static(const slrf_csr_pair *pc, double gamma, const slrf_opts *opts,
                                        const double *X, int k, const double *theta, double *U, void *stream) {
  if (!pc || !pc->rowptr || !pc->col || !pc->valA || !pc->valB || pc->n < 1 || pc->nnz < 1) return SLRF_EINVAL;
  if (!X || !U || X == U || k < 1 || !(gamma > 0)) return SLRF_EINVAL;
  slrf_opts o;
  if (opts) o = *opts;
  else slrf_opts_default(&o);
  if (o.m < 1 || o.m > 32 || o.it_max < 1 || !(o.tol_inner >= 0)) return SLRF_EINVAL;
  if (o.precision != 0) return SLRF_EINVAL;  // FP64 only
  const cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = pc->n;
  const int m = o.m, mp = pow2_at_least(m);
  const int W = ((k * mp + 31) / 32) * 32;
  const int ntiles = W / 32;
  const int64_t rpb = std::max<int64_t>(16, (n + 152 * 4 - 1) / (152 * 4));
  const int nrb = (int)((n + rpb - 1) / rpb);
  // layout of the arena for this call
  Carver c{nullptr};
  c.take<double2>(32);
  c.take<double2>(32);
  c.take<int>(16);
  c.take<double>((size_t)n * k * 3);
  c.take<double2>((size_t)n * W * 4);
  c.take<double>((size_t)nrb * W * kNQ);
  c.take<unsigned>((size_t)ntiles + 32);
  c.take<WScal>((size_t)W);
  c.take<double2>((size_t)W);
  c.take<double>((size_t)k);
  if (c.off > (size_t)SLRF_STATIC_ARENA_BYTES) return SLRF_EINVAL;  // problem too large for the arena
  unsigned char *base = nullptr;
  int rc = arena_address(&base);
  if (rc != SLRF_OK) return rc;
  Carver a{base};
  double2 *sig = a.take<double2>(32), *wt = a.take<double2>(32);
  int *flags = a.take<int>(16);
  double *G = a.take<double>((size_t)n * k * 3);
  double *AG = G + (size_t)n * k, *BG = AG + (size_t)n * k;
  double2 *state = a.take<double2>((size_t)n * W * 4);
  double *partial = a.take<double>((size_t)nrb * W * kNQ);
  unsigned *counters = a.take<unsigned>((size_t)ntiles + 32);
  WScal *ws = a.take<WScal>((size_t)W);
  double2 *cfac = a.take<double2>((size_t)W);
  double *coefV = a.take<double>((size_t)k);
  // the arena keeps the previous call's contents: clear what must start at zero
  if (cudaMemsetAsync(counters, 0, ((size_t)ntiles + 32) * sizeof(unsigned), st) != cudaSuccess ||
      cudaMemsetAsync(flags, 0, 16 * sizeof(int), st) != cudaSuccess)
    return SLRF_ECUDA;
  if (o.poles && o.weights) {
    double2 hs[32], hw[32];
    for (int j = 0; j < mp; ++j) {
      hs[j] = j < m ? make_double2(o.poles[2 * j], o.poles[2 * j + 1]) : make_double2(gamma, gamma);
      hw[j] = j < m ? make_double2(o.weights[2 * j], o.weights[2 * j + 1]) : make_double2(0, 0);
    }
    if (cudaMemcpyAsync(sig, hs, mp * sizeof(double2), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(wt, hw, mp * sizeof(double2), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return SLRF_ECUDA;
  } else {
    int hflag = 0;
    design_poles(m, mp, gamma, o.alpha, o.beta, o.band, sig, wt, flags, st);
    if (cudaMemcpyAsync(&hflag, flags, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return SLRF_ECUDA;
    if (hflag != 0) return SLRF_EINVAL;
  }
  // the real FP64 sweep that starts every pole (zero guess: g = B X; warm: g = A X - theta B X)
  if (theta == nullptr) {
    spmm_real(n, pc->rowptr, pc->col, pc->valA, pc->valB, X, k, k, nullptr, G, k, st);
  } else {
    spmm_real(n, pc->rowptr, pc->col, pc->valA, pc->valB, X, k, k, AG, BG, k, st);
    shifted_residual(n, k, AG, BG, k, theta, G, k, st);
  }
  spmm_real(n, pc->rowptr, pc->col, pc->valA, pc->valB, G, k, k, AG, BG, k, st);
  CocgArgs<double> ca{};
  ca.n = n;
  ca.rowptr = pc->rowptr;
  ca.col = pc->col;
  ca.valA = pc->valA;
  ca.valB = pc->valB;
  ca.W = W;
  ca.k = k;
  ca.m = m;
  ca.mp = mp;
  ca.rows_per_block = (int)rpb;
  ca.nrb = nrb;
  ca.d = state;
  ca.r = state + (size_t)n * W;
  ca.p = state + 2 * (size_t)n * W;
  ca.q = state + 3 * (size_t)n * W;
  ca.sig = sig;
  ca.partial = partial;
  ca.counters = counters;
  ca.ws = ws;
  ca.tol2 = o.tol_inner * o.tol_inner;
  ca.g = G;
  ca.Ag = AG;
  ca.Bg = BG;
  ca.ldg = k;
  ca.cfac = cfac;
  ca.gscale = nullptr;
  ca.wt = wt;
  ca.V = X;
  ca.ldv = k;
  ca.coefV = coefV;
  ca.U = U;
  ca.ldu = k;
  cocg_prepare(W, k, m, mp, sig, wt, theta, cfac, coefV, ws, st);
  cocg_init<double>(ca, st);
  for (int it = 1; it <= o.it_max; ++it) {
    cocg_update<double>(ca, it == 1, it == o.it_max ? kFinalU : kFinalNone, st);
    if (it < o.it_max) cocg_spmm<double>(ca, st);
  }
  return cudaGetLastError() == cudaSuccess ? SLRF_OK : SLRF_ECUDA;
}
