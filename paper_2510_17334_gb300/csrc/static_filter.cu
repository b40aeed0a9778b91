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
// host-side stand-in, not a device address.  Every call looks the device address up with
// cudaGetSymbolAddress, with the caller's device current (a cheap query that allocates
// nothing, so the address stays right after a device reset too).
//
// Before any kernel gathers through the caller's pattern, the call checks it on the
// device (rowptr monotone from 0 to nnz, columns in [0, n)) and refuses a malformed one
// with SLRF_EINVAL, as slrf_setup does.  The designed pole table stays in the arena and
// is reused by the next call on the same device with the same (m, gamma, alpha, beta,
// band) -- the design is one small kernel of a few milliseconds.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <mutex>

#include "../../include/slrf.h"
#include "cocg.cuh"
#include "dense.cuh"

namespace slrf {

static __device__ __align__(256) unsigned char arena[SLRF_STATIC_ARENA_BYTES];

namespace {
constexpr int kMaxDevices = 64;
// Which designed pole table the arena of each device holds (host-side record).
struct PoleKey {
  bool valid = false;
  int m = 0;
  double gamma = 0, alpha = 0, beta = 0, band = 0;
  unsigned char *base = nullptr;
};
std::mutex g_mu;
PoleKey g_poles[kMaxDevices];

// device address of `arena` on the current device
int arena_address(unsigned char **out, int *dev_out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SLRF_ECUDA;
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, arena) != cudaSuccess || p == nullptr) {
    cudaGetLastError();
    return SLRF_ECUDA;
  }
  *out = static_cast<unsigned char *>(p);
  *dev_out = dev;
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
  if (pc->n > (int64_t)INT32_MAX) return SLRF_EINVAL;  // int32 column indices
  if (!X || !U || X == U || k < 1 || !(gamma > 0)) return SLRF_EINVAL;
  slrf_opts o;
  if (opts) o = *opts;
  else slrf_opts_default(&o);
  if (o.m < 1 || o.m > 32 || o.it_max < 1 || !(o.tol_inner >= 0)) return SLRF_EINVAL;
  if (o.precision != 0 || o.precond != 0) return SLRF_EINVAL;  // FP64, unpreconditioned only
  const cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = pc->n;
  const int m = o.m, mp = pow2_at_least(m);
  const int W = ((k * mp + 31) / 32) * 32;
  const int ntiles = W / 32;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return SLRF_ECUDA;
  const int64_t rpb = std::max<int64_t>(16, (n + (int64_t)sms * 4 - 1) / ((int64_t)sms * 4));
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
  int rc = arena_address(&base, &dev);
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
  // reject a malformed pattern before any kernel gathers through it (flags[1])
  validate_csr(n, pc->nnz, pc->rowptr, pc->col, flags + 1, sms * 4, st);
  double2 hs[32], hw[32];
  const bool user_table = o.poles && o.weights;
  bool designed = false;
  if (user_table) {
    for (int j = 0; j < mp; ++j) {
      hs[j] = j < m ? make_double2(o.poles[2 * j], o.poles[2 * j + 1]) : make_double2(gamma, gamma);
      hw[j] = j < m ? make_double2(o.weights[2 * j], o.weights[2 * j + 1]) : make_double2(0, 0);
    }
    if (cudaMemcpyAsync(sig, hs, mp * sizeof(double2), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(wt, hw, mp * sizeof(double2), cudaMemcpyHostToDevice, st) != cudaSuccess)
      return SLRF_ECUDA;
  } else {
    std::lock_guard<std::mutex> lk(g_mu);
    const PoleKey &pk = g_poles[dev];
    const bool hit = pk.valid && pk.base == base && pk.m == m && pk.gamma == gamma && pk.alpha == o.alpha &&
                     pk.beta == o.beta && pk.band == o.band;
    if (!hit) {
      design_poles(m, mp, gamma, o.alpha, o.beta, o.band, sig, wt, flags, st);
      designed = true;
    }
  }
  // one synchronisation: the pattern check, the pole design status and (user table) the
  // host arrays of the copies above
  int hflag[2] = {0, 0};
  if (cudaMemcpyAsync(hflag, flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return SLRF_ECUDA;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    PoleKey &pk = g_poles[dev];
    if (user_table || hflag[0] != 0) {
      pk.valid = false;  // the arena no longer holds a designed table
    } else if (designed) {
      pk.valid = true;
      pk.base = base;
      pk.m = m;
      pk.gamma = gamma;
      pk.alpha = o.alpha;
      pk.beta = o.beta;
      pk.band = o.band;
    }
  }
  if (hflag[1] != 0) return SLRF_EINVAL;
  if (hflag[0] != 0) return SLRF_EINVAL;
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
  ca.vec = 1;
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
