// COCG for every (pole, column) shifted system of one filter apply, all in one grid.
//
// Method: the warm-started solves of Alg. 2 (arXiv 2510.17334, Sec. 4) in their Cayley
// form (Proposition, Sec. 4): with y0 = v/(theta - sigma), the residual system is
// (A - sigma B) d = r0,  r0 = (A - theta B) v / (sigma - theta),  solution y0 + d.
// Here r0 = c_w g with a real block g (g = B v and c = 1 for the zero initial guess,
// g = (A - theta B) v and c = 1/(sigma - theta) for the warm start), so every pole's
// start comes from one real FP64 sweep.  COCG (van der Vorst & Melissen) runs with
// the unconjugated bilinear form; each column stops at ||r|| <= tol ||r0|| or It_max.
//
// Layout: complex state [row][column][pole] (w = column * mp + pole), W entries per row.
// A warp owns 32 * VEC consecutive w (one 16-byte load per lane per gathered row),
// every warp of a block works on the same tile of w for a range of rows, and blockIdx.y
// (the tile) varies slowest so that one tile's rows stay resident in L2 while they are
// gathered.  CSR entries of a row are read once per warp and broadcast by shuffles.
//
// Kernels per iteration (2 launches):
//   update : d += alpha p; r -= alpha q; reduce rho' = r^T r, ||r||^2   -> beta, stop mask
//   spmm   : s = (A - sigma B) r (gathers r); p = r + beta p; q = s + beta q;
//            reduce mu = p^T q                                         -> alpha = rho/mu
// (q = A p is carried by the recurrence q = A r + beta q, so one SpMM per iteration.)
// Block partial sums are written to a buffer and the last block of each tile reduces
// them in a fixed order (deterministic) and updates the per-column scalars.
#include "cocg.cuh"

#include <type_traits>

#ifndef SLRF_GATHER_UNROLL
#define SLRF_GATHER_UNROLL 8
#endif
// CSR entries of a row chunk from shared-memory records (1) or register shuffles (0):
// records win in FP64 (five shuffles per entry), shuffles by a little in FP32
#ifndef SLRF_SPMM_SREC64
#define SLRF_SPMM_SREC64 1
#endif
#ifndef SLRF_SPMM_SREC32
#define SLRF_SPMM_SREC32 0
#endif
// grouped-row SpMM: records in flight per warp, resident blocks per SM
#ifndef SLRF_GRP_UNROLL
#define SLRF_GRP_UNROLL 8
#endif
#ifndef SLRF_GRP_MINB
#define SLRF_GRP_MINB 2
#endif
#ifndef SLRF_GRP_UNROLL_BD
#define SLRF_GRP_UNROLL_BD 4
#endif
// Per-record check of the gathered column in the grouped SpMM (1), or none (0): the records
// are built on the device from a pattern validated at setup and checked once after the
// build (grp_check), and nothing writes them afterwards (the check costs 5 % of the SpMM).
#ifndef SLRF_GRP_COLCHECK
#define SLRF_GRP_COLCHECK 0
#endif
namespace slrf {
constexpr int kGatherUnroll = SLRF_GATHER_UNROLL;  // CSR entries of a row in flight per warp
constexpr int kGrpUnroll = SLRF_GRP_UNROLL;        // grouped records in flight per warp
constexpr int kGrpUnrollBD = SLRF_GRP_UNROLL_BD;   // node triples in flight per warp (B-diagonal)
}

namespace slrf {

// VEC complex entries of one lane (16-byte loads: one in FP64, VEC / 2 in FP32)
template <typename R, int V> struct Vec { cx_t<R> z[V]; };

// Where the lane's 16-byte pieces live.  The kernels index the complex state (r, p, q, d)
// logically -- lane l owns the entries [V l, V l + V) of a tile of 32 V -- and reach it only
// through ldv / stv at tile + V l.  With V > 2 (FP32, two pieces per lane) the pieces are
// stored 64 entries apart, piece j of lane l at tile + 64 j + 2 l, so that every load
// instruction of the warp covers 512 contiguous bytes (with the pieces side by side, each
// instruction would touch every sector of the 1 KB segment and use half of it).
template <typename R, int V> __device__ __forceinline__ const float4 *piece(const cx_t<R> *p, int j) {
  const int lane = threadIdx.x & 31;
  return reinterpret_cast<const float4 *>(p - (V - 2) * lane + 64 * j);
}
template <typename R, int V> __device__ __forceinline__ float4 *piece(cx_t<R> *p, int j) {
  const int lane = threadIdx.x & 31;
  return reinterpret_cast<float4 *>(p - (V - 2) * lane + 64 * j);
}

template <typename R, int V> __device__ __forceinline__ Vec<R, V> ldv(const cx_t<R> *p) {
  Vec<R, V> v;
  if constexpr (sizeof(R) == 8) {
    v.z[0] = *reinterpret_cast<const double2 *>(p);
  } else {
#pragma unroll
    for (int j = 0; j < V / 2; ++j) {
      const float4 t = *piece<R, V>(p, j);
      v.z[2 * j] = make_float2(t.x, t.y);
      v.z[2 * j + 1] = make_float2(t.z, t.w);
    }
  }
  return v;
}
template <typename R, int V> __device__ __forceinline__ void stv(cx_t<R> *p, const Vec<R, V> &v) {
  if constexpr (sizeof(R) == 8) {
    *reinterpret_cast<double2 *>(p) = v.z[0];
  } else {
#pragma unroll
    for (int j = 0; j < V / 2; ++j)
      *piece<R, V>(p, j) = make_float4(v.z[2 * j].x, v.z[2 * j].y, v.z[2 * j + 1].x, v.z[2 * j + 1].y);
  }
}

// Streaming (evict-first) loads and stores of the SpMM's own-row p and q: they are read
// and written once per launch, so they should not push the gathered rows of r out of L2.
#ifndef SLRF_SPMM_STREAM
#define SLRF_SPMM_STREAM 1
#endif
template <typename R, int V> __device__ __forceinline__ Vec<R, V> ldv_cs(const cx_t<R> *p) {
  if constexpr (SLRF_SPMM_STREAM == 0) {
    return ldv<R, V>(p);
  } else {
    Vec<R, V> v;
    if constexpr (sizeof(R) == 8) {
      v.z[0] = __ldcs(reinterpret_cast<const double2 *>(p));
    } else {
#pragma unroll
      for (int j = 0; j < V / 2; ++j) {
        const float4 t = __ldcs(piece<R, V>(p, j));
        v.z[2 * j] = make_float2(t.x, t.y);
        v.z[2 * j + 1] = make_float2(t.z, t.w);
      }
    }
    return v;
  }
}
template <typename R, int V> __device__ __forceinline__ void stv_cs(cx_t<R> *p, const Vec<R, V> &v) {
  if constexpr (SLRF_SPMM_STREAM == 0) {
    stv<R, V>(p, v);
  } else if constexpr (sizeof(R) == 8) {
    __stcs(reinterpret_cast<double2 *>(p), v.z[0]);
  } else {
#pragma unroll
    for (int j = 0; j < V / 2; ++j)
      __stcs(piece<R, V>(p, j), make_float4(v.z[2 * j].x, v.z[2 * j].y, v.z[2 * j + 1].x, v.z[2 * j + 1].y));
  }
}

template <typename R> __device__ __forceinline__ cx_t<R> to_c(double2 a) {
  cx_t<R> z; z.x = (R)a.x; z.y = (R)a.y; return z;
}

// Reduce the per-lane values acc[VEC][NQ] of all warps of the block into the block's
// partial slot, then (last block of the tile only) reduce all blocks' slots into out.
// Returns true in every thread of the last block; out is valid in threads t < TW of it.
template <int VEC, int NQ>
__device__ bool block_then_grid_reduce(double (&acc)[VEC][NQ], const int W, const int w_tile0,
                                       const int rb, const int nrb, double *partial,
                                       unsigned *counter, double (&out)[NQ], int &w_out) {
  constexpr int TW = 32 * VEC;
  __shared__ double sm[kWarps][TW][NQ];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int v = 0; v < VEC; ++v)
#pragma unroll
    for (int qq = 0; qq < NQ; ++qq) sm[warp][lane * VEC + v][qq] = acc[v][qq];
  __syncthreads();
  for (int t = threadIdx.x; t < TW * NQ; t += kThreads) {
    const int wl = t / NQ, qq = t % NQ;
    double s = 0.0;
#pragma unroll
    for (int wi = 0; wi < kWarps; ++wi) s += sm[wi][wl][qq];
    partial[((size_t)rb * W + w_tile0 + wl) * kNQ + qq] = s;
  }
  if (!last_block_arrive(counter, (unsigned)nrb)) return false;
  // last block: sum the nrb slots of this tile in a fixed order
  double a2[VEC][NQ];
#pragma unroll
  for (int v = 0; v < VEC; ++v)
#pragma unroll
    for (int qq = 0; qq < NQ; ++qq) a2[v][qq] = 0.0;
  for (int b = warp; b < nrb; b += kWarps) {
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
      const double *src = partial + ((size_t)b * W + w_tile0 + lane * VEC + v) * kNQ;
#pragma unroll
      for (int qq = 0; qq < NQ; ++qq) a2[v][qq] += __ldcg(src + qq);
    }
  }
  __syncthreads();
#pragma unroll
  for (int v = 0; v < VEC; ++v)
#pragma unroll
    for (int qq = 0; qq < NQ; ++qq) sm[warp][lane * VEC + v][qq] = a2[v][qq];
  __syncthreads();
  if (threadIdx.x < TW) {
    w_out = w_tile0 + threadIdx.x;
#pragma unroll
    for (int qq = 0; qq < NQ; ++qq) {
      double s = 0.0;
#pragma unroll
      for (int wi = 0; wi < kWarps; ++wi) s += sm[wi][threadIdx.x][qq];
      out[qq] = s;
    }
  }
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

// ------------------------------------------------------------------------------ init
// r0 = c g, p0 = r0, q0 = c (A g - sigma B g); reduce mu0 = p0^T q0, rho0 = r0^T r0, ||r0||^2.
template <typename R, int V>
__device__ __forceinline__ void cocg_init_body(const CocgArgs<R> &a, const int rb, const int tile) {
  constexpr int VEC = V;
  using C = cx_t<R>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int w_tile0 = tile * 32 * VEC;
  const int w0 = w_tile0 + lane * VEC;
  C sg[VEC], cf[VEC];
  int cidx[VEC];
  bool ok[VEC];
#pragma unroll
  for (int v = 0; v < VEC; ++v) {
    const int w = w0 + v;
    sg[v] = a.sig[w & (a.mp - 1)];
    cidx[v] = w / a.mp;
    ok[v] = cidx[v] < a.k;
    double2 c = a.cfac[w];
    if (a.gscale != nullptr && ok[v]) {
      const double gs = a.gscale[cidx[v]];
      c.x *= gs;
      c.y *= gs;
    }
    cf[v] = to_c<R>(c);
  }
  constexpr int NQ = 5;
  R acc[VEC][NQ];  // per-thread partial sums in the working precision
#pragma unroll
  for (int v = 0; v < VEC; ++v)
#pragma unroll
    for (int qq = 0; qq < NQ; ++qq) acc[v][qq] = R(0);
  const int64_t i0 = (int64_t)rb * a.rows_per_block;
  const int64_t i1 = (i0 + a.rows_per_block < a.n ? i0 + a.rows_per_block : a.n);
  for (int64_t i = i0 + warp; i < i1; i += kWarps) {
    Vec<R, VEC> rv, qv;
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
      R gv = 0, agv = 0, bgv = 0;
      if (ok[v]) {
        const size_t o = (size_t)i * a.ldg + cidx[v];
        if (CHK(1, o, (long long)a.n * a.ldg)) { gv = (R)a.g[o]; agv = (R)a.Ag[o]; bgv = (R)a.Bg[o]; }
      }
      C r0; r0.x = cf[v].x * gv; r0.y = cf[v].y * gv;
      C t; t.x = agv - sg[v].x * bgv; t.y = -sg[v].y * bgv;
      C q0 = cmul(cf[v], t);
      rv.z[v] = r0; qv.z[v] = q0;
      acc[v][0] += r0.x * q0.x - r0.y * q0.y;
      acc[v][1] += r0.x * q0.y + r0.y * q0.x;
      acc[v][2] += r0.x * r0.x - r0.y * r0.y;
      acc[v][3] += 2 * r0.x * r0.y;
      acc[v][4] += r0.x * r0.x + r0.y * r0.y;
    }
    const size_t off = (size_t)i * a.W + w0;
    if (CHK(2, off + VEC - 1, (long long)a.n * a.W)) {
      stv<R, VEC>(a.r + off, rv);
      stv<R, VEC>(a.p + off, rv);
      stv<R, VEC>(a.q + off, qv);
    }
  }
  double out[NQ];
  int w;
  double accd[VEC][NQ];
#pragma unroll
  for (int v = 0; v < VEC; ++v)
#pragma unroll
    for (int qq = 0; qq < NQ; ++qq) accd[v][qq] = (double)acc[v][qq];
  if (!block_then_grid_reduce<VEC, NQ>(accd, a.W, w_tile0, rb, a.nrb, a.partial, a.counters + tile, out, w))
    return;
  if (threadIdx.x < 32 * VEC) {
    WScal s = a.ws[w];
    const double2 mu = make_double2(out[0], out[1]);
    s.rho = make_double2(out[2], out[3]);
    s.r0n2 = out[4];
    s.rn2 = out[4];
    s.iters = 0;
    s.iters_total = 0;
    if (a.r00 != nullptr) a.r00[w] = out[4];
    s.brk = 0;
    s.beta = make_double2(0.0, 0.0);
    if (s.active && !(out[4] > 0.0)) s.active = 0;  // zero right-hand side: nothing to do
    if (s.active && (!cfinite(mu) || (mu.x == 0.0 && mu.y == 0.0))) { s.active = 0; s.brk = 1; }
    s.alpha = s.active ? cdiv(s.rho, mu) : make_double2(0.0, 0.0);
    a.ws[w] = s;
  }
}

// ------------------------------------------------------------------------------ update
// d += alpha p (d = alpha p on the first step); r -= alpha q; reduce rho' and ||r||^2.
// With final_acc, also U[i][c] = coefV[c] V[i][c] + sum_j 2 Re(w_j d_j).
// kAccU / kAccUEnd (the updates of a solve without refinement): no d at all -- the filter
// is linear in d, so each update adds the pole sum of its step to a real accumulator,
//   Uacc[i][c] (+)= sum_j 2 Re(w_j alpha_j p_j)     (working precision, scaled units),
// n x k reals instead of d's n x k x m complex entries read and written every update.
// Uacc is laid out tile by tile ([tile][row][columns of the tile]) so that each launch
// streams it; the last update (kAccUEnd) writes U = coefV V + Uacc / gscale * dsc in FP64.
template <typename R, int V, bool FIRST, int FM>
__device__ __forceinline__ void cocg_update_body(const CocgArgs<R> &a, const int rb, const int tile) {
  constexpr bool ACCU_END = FM == kAccUEnd;
  constexpr bool ACCU = FM == kAccU || ACCU_END;
  constexpr bool FINAL = FM != kFinalNone && !ACCU;
  constexpr int VEC = V;
  using C = cx_t<R>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int w_tile0 = tile * 32 * VEC;
  const int w0 = w_tile0 + lane * VEC;
  C al[VEC];
  double2 wt[VEC];  // weights stay FP64: the pole sum is formed in FP64
  bool act[VEC];
  bool any_act = false;
#pragma unroll
  for (int v = 0; v < VEC; ++v) {
    const WScal &s = a.ws[w0 + v];
    act[v] = s.active != 0;
    any_act |= act[v];
    al[v] = to_c<R>(s.alpha);
    wt[v] = a.wt[(w0 + v) & (a.mp - 1)];
  }
  constexpr int NQ = 3;
  R acc[VEC][NQ];  // per-thread partial sums in the working precision
#pragma unroll
  for (int v = 0; v < VEC; ++v)
#pragma unroll
    for (int qq = 0; qq < NQ; ++qq) acc[v][qq] = R(0);
  const int64_t i0 = (int64_t)rb * a.rows_per_block;
  const int64_t i1 = (i0 + a.rows_per_block < a.n ? i0 + a.rows_per_block : a.n);
  const int lanes_per_col = a.mp >= VEC ? a.mp / VEC : 1;
  const bool warp_act = __any_sync(0xffffffffu, any_act);
  const int cpt = 32 * VEC / a.mp;  // columns of a tile (kAccU accumulator layout)
#pragma unroll 1
  for (int64_t i = i0 + warp; i < i1; i += kWarps) {
    const size_t off = (size_t)i * a.W + w0;
    Vec<R, VEC> dv;
    R step[VEC];  // kAccU: 2 Re(w_j alpha_j p_j) of this lane's entries
#pragma unroll
    for (int v = 0; v < VEC; ++v) step[v] = R(0);
    // kAccU: this lane's accumulator entries (one per column it leads), loaded up front so
    // that the load overlaps the loads of p, q and r
    R uold[VEC];
    R *const uacc = reinterpret_cast<R *>(a.uacc) + ((size_t)tile * a.n + i) * cpt - (size_t)tile * cpt;
    if constexpr (ACCU) {
#pragma unroll
      for (int v = 0; v < VEC; ++v) {
        uold[v] = R(0);
        const int c = (w0 + v) / a.mp;
        const bool lead = a.mp >= VEC ? (v == 0 && (lane % lanes_per_col) == 0) : true;
        if (!FIRST && (warp_act || ACCU_END) && lead && c < a.k) uold[v] = uacc[c];
      }
    } else {
      if (FIRST) {
#pragma unroll
        for (int v = 0; v < VEC; ++v) dv.z[v] = cmake<C>(0, 0);
      } else if (any_act || FINAL) {
        if (CHK(3, off + VEC - 1, (long long)a.n * a.W)) dv = ldv<R, VEC>(a.d + off);
      }
    }
    if (any_act) {
      Vec<R, VEC> pv, qv, rv;
      if (CHK(4, off + VEC - 1, (long long)a.n * a.W)) {
        pv = ldv<R, VEC>(a.p + off);
        qv = ldv<R, VEC>(a.q + off);
        rv = ldv<R, VEC>(a.r + off);
      }
#pragma unroll
      for (int v = 0; v < VEC; ++v) {
        if (act[v]) {
          if constexpr (ACCU) {
            const C ap = cmul(al[v], pv.z[v]);
            step[v] = R(2) * ((R)wt[v].x * ap.x - (R)wt[v].y * ap.y);
          } else {
            dv.z[v] = cfma(al[v], pv.z[v], dv.z[v]);
          }
          rv.z[v] = cfms(al[v], qv.z[v], rv.z[v]);
        }
        const C rr = rv.z[v];
        acc[v][0] += rr.x * rr.x - rr.y * rr.y;
        acc[v][1] += 2 * rr.x * rr.y;
        acc[v][2] += rr.x * rr.x + rr.y * rr.y;
      }
      if (CHK(5, off + VEC - 1, (long long)a.n * a.W)) stv<R, VEC>(a.r + off, rv);
    }
    if constexpr (ACCU) {
      if (FIRST || ACCU_END || warp_act) {
        // pole sum of the step into the accumulator; the last update forms U in FP64
        auto put = [&](int c, R acc_new) {
          if (ACCU_END) {
            double corr = (double)acc_new;
            if (a.gscale != nullptr) corr /= a.gscale[c];
            if (a.dsc != nullptr) corr *= a.dsc[i];
            a.U[(size_t)i * a.ldu + c] = a.coefV[c] * a.V[(size_t)i * a.ldv + c] + corr;
          } else {
            uacc[c] = acc_new;
          }
        };
        if (a.mp >= VEC) {
          R sum = R(0);
#pragma unroll
          for (int v = 0; v < VEC; ++v) sum += step[v];
          for (int o = lanes_per_col >> 1; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
          const int c = w0 / a.mp;
          if ((lane % lanes_per_col) == 0 && c < a.k) put(c, uold[0] + sum);
        } else {
#pragma unroll
          for (int v = 0; v < VEC; ++v) {
            const int c = (w0 + v) / a.mp;
            if (c < a.k) put(c, uold[v] + step[v]);
          }
        }
      }
      continue;
    }
    if ((FIRST || any_act) && CHK(6, off + VEC - 1, (long long)a.n * a.W)) stv<R, VEC>(a.d + off, dv);
    if (FM == kFinalStoreD || FM == kFinalAddD) {
      // refinement: accumulate this step's correction into the FP64 D
#pragma unroll
      for (int v = 0; v < VEC; ++v) {
        double2 acc2 = FM == kFinalAddD ? a.D64[off + v] : make_double2(0.0, 0.0);
        acc2.x += (double)dv.z[v].x;
        acc2.y += (double)dv.z[v].y;
        a.D64[off + v] = acc2;
      }
    } else if (FINAL) {
      // U = coefV V + sum over this column's poles of 2 Re(w_j y_j), y_j = d_j (+ D_j)
      double part[VEC];
#pragma unroll
      for (int v = 0; v < VEC; ++v) {
        double yr = (double)dv.z[v].x, yi = (double)dv.z[v].y;
        if (FM == kFinalUFromD) {
          const double2 dd = a.D64[off + v];
          yr += dd.x;
          yi += dd.y;
        }
        part[v] = 2.0 * (wt[v].x * yr - wt[v].y * yi);
      }
      // preconditioned solves work on z = D^1/2 y: y = dsc_i z
      const double ds = a.dsc != nullptr ? a.dsc[i] : 1.0;
      if (a.mp >= VEC) {
        double s = 0.0;
#pragma unroll
        for (int v = 0; v < VEC; ++v) s += part[v];
        for (int o = lanes_per_col >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const int c = w0 / a.mp;
        if ((lane % lanes_per_col) == 0 && c < a.k) {
          if (a.gscale != nullptr) s /= a.gscale[c];
          if (a.dsc != nullptr) s *= ds;
          if (CHK(7, (long long)i * a.ldu + c, (long long)a.n * a.ldu) && CHK(8, c, a.k))
            a.U[(size_t)i * a.ldu + c] = a.coefV[c] * a.V[(size_t)i * a.ldv + c] + s;
        }
      } else {
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
          const int c = (w0 + v) / a.mp;
          if (c < a.k) {
            double s = a.gscale ? part[v] / a.gscale[c] : part[v];
            if (a.dsc != nullptr) s *= ds;
            a.U[(size_t)i * a.ldu + c] = a.coefV[c] * a.V[(size_t)i * a.ldv + c] + s;
          }
        }
      }
    }
  }
  double out[NQ];
  int w;
  double accd[VEC][NQ];
#pragma unroll
  for (int v = 0; v < VEC; ++v)
#pragma unroll
    for (int qq = 0; qq < NQ; ++qq) accd[v][qq] = (double)acc[v][qq];
  if (!block_then_grid_reduce<VEC, NQ>(accd, a.W, w_tile0, rb, a.nrb, a.partial, a.counters + tile, out, w))
    return;
  if (threadIdx.x < 32 * VEC) {
    WScal s = a.ws[w];
    if (s.active) {
      s.iters += 1;
      s.iters_total += 1;
      s.rn2 = out[2];
      const double2 rho_new = make_double2(out[0], out[1]);
      if (out[2] <= a.tol2 * s.r0n2) {
        s.active = 0;
      } else if (!cfinite(rho_new) || (s.rho.x == 0.0 && s.rho.y == 0.0)) {
        s.active = 0;
        s.brk = 1;
      } else {
        s.beta = cdiv(rho_new, s.rho);
        s.rho = rho_new;
      }
      if (a.it_cap > 0 && s.iters >= a.it_cap) s.active = 0;
      if (!s.active) s.beta = make_double2(0.0, 0.0);
      a.ws[w] = s;
    }
  }
}

// ------------------------------------------------------------------------------ spmm
// One CSR entry of a row chunk as the SpMM reads it from shared memory: a 16-byte record
// (FP32: column, a, b) or 24 bytes (FP64: a, b as a 16-byte pair, then the column).
template <typename R> struct SRec;
template <> struct alignas(16) SRec<float> { int c; float a, b, pad; };
template <> struct alignas(16) SRec<double> { double2 ab; int c, pad0, pad1, pad2; };
template <typename R> __device__ __forceinline__ void srec_put(SRec<R> *r, int lane, int c, R av, R bv);
template <> __device__ __forceinline__ void srec_put<float>(SRec<float> *r, int lane, int c, float av, float bv) {
  *reinterpret_cast<float4 *>(r + lane) = make_float4(__int_as_float(c), av, bv, 0.f);
}
template <> __device__ __forceinline__ void srec_put<double>(SRec<double> *r, int lane, int c, double av, double bv) {
  r[lane].ab = make_double2(av, bv);
  r[lane].c = c;
}
template <typename R> __device__ __forceinline__ void srec_get(const SRec<R> *r, int t, int &c, R &av, R &bv);
template <> __device__ __forceinline__ void srec_get<float>(const SRec<float> *r, int t, int &c, float &av, float &bv) {
  const float4 v = *reinterpret_cast<const float4 *>(r + t);
  c = __float_as_int(v.x);
  av = v.y;
  bv = v.z;
}
template <> __device__ __forceinline__ void srec_get<double>(const SRec<double> *r, int t, int &c, double &av, double &bv) {
  const double2 ab = r[t].ab;
  c = r[t].c;
  av = ab.x;
  bv = ab.y;
}

// Block and grid reduction of the mu partials of one SpMM launch, then alpha = rho / mu per
// (pole, column) in the last block of the tile (breakdown: mu = 0 or not finite).
template <typename R, int VEC>
__device__ __forceinline__ void spmm_tail(const CocgArgs<R> &a, const R (&acc)[VEC][2], const int w_tile0,
                                          const int rb, const int tile, const int nblocks) {
  constexpr int NQ = 2;
  double out[NQ];
  int w;
  double accd[VEC][NQ];
#pragma unroll
  for (int v = 0; v < VEC; ++v)
#pragma unroll
    for (int qq = 0; qq < NQ; ++qq) accd[v][qq] = (double)acc[v][qq];
  if (!block_then_grid_reduce<VEC, NQ>(accd, a.W, w_tile0, rb, nblocks, a.partial, a.counters + tile, out, w))
    return;
  if (threadIdx.x < 32 * VEC) {
    WScal s = a.ws[w];
    if (s.active) {
      const double2 mu = make_double2(out[0], out[1]);
      if (!cfinite(mu) || (mu.x == 0.0 && mu.y == 0.0)) {
        s.active = 0;
        s.brk = 1;
        s.alpha = make_double2(0.0, 0.0);
      } else {
        s.alpha = cdiv(s.rho, mu);
      }
      a.ws[w] = s;
    }
  }
}

// s = (A - sigma B) r; p = r + beta p; q = s + beta q; reduce mu = p^T q -> alpha = rho/mu.
template <typename R, int V, bool FRESH>
__device__ __forceinline__ void cocg_spmm_body(const CocgArgs<R> &a, const int rb, const int tile) {
  constexpr int VEC = V;
  using C = cx_t<R>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int w_tile0 = tile * 32 * VEC;
  const int w0 = w_tile0 + lane * VEC;
  constexpr bool kSrec = sizeof(R) == 8 ? SLRF_SPMM_SREC64 != 0 : SLRF_SPMM_SREC32 != 0;
  __shared__ SRec<R> srec_all[kSrec ? kWarps * 32 : 1];
  SRec<R> *const srec = srec_all + (kSrec ? warp * 32 : 0);
  // (beta and the poles are read again for each row's epilogue: not held across the gathers)
  bool any_act = false;
#pragma unroll
  for (int v = 0; v < VEC; ++v) any_act |= a.ws[w0 + v].active != 0;
  // warp-uniform: skip the tile's SpMM when no column in it is still iterating
  const bool warp_act = __any_sync(0xffffffffu, any_act);
  constexpr int NQ = 2;
  R acc[VEC][NQ];  // per-thread partial sums in the working precision
#pragma unroll
  for (int v = 0; v < VEC; ++v)
#pragma unroll
    for (int qq = 0; qq < NQ; ++qq) acc[v][qq] = R(0);
  const int64_t i0 = (int64_t)rb * a.rows_per_block;
  const int64_t i1 = (i0 + a.rows_per_block < a.n ? i0 + a.rows_per_block : a.n);
  if (warp_act) {
    // s = (A - sigma B) r for one row (sa = A r, sb = B r), lanes over this warp's columns
    const char *const rlane = reinterpret_cast<const char *>(a.r + w0);
    const unsigned wbytes = (unsigned)a.W * (unsigned)sizeof(C);
    auto gather_row = [&](int64_t i, C (&sa)[VEC], C (&sb)[VEC]) {
#pragma unroll
      for (int v = 0; v < VEC; ++v) { sa[v] = cmake<C>(0, 0); sb[v] = cmake<C>(0, 0); }
      const int64_t rs = a.rowptr[i], re = a.rowptr[i + 1];
      for (int64_t e0 = rs; e0 < re; e0 += 32) {
        const int cnt = (int)(re - e0 < 32 ? re - e0 : 32);
        int cl = 0;
        R avl = 0, bvl = 0;
        if (lane < cnt) { cl = a.col[e0 + lane]; avl = a.valA[e0 + lane]; bvl = a.valB[e0 + lane]; }
        if constexpr (kSrec) {
          // the warp's chunk of (column, a, b) goes to shared memory once; every entry is
          // then one broadcast shared load instead of three (FP64: five) register shuffles,
          // which share the load/store pipe with the gathers
          __syncwarp();
          srec_put<R>(srec, lane, cl, avl, bvl);
          __syncwarp();
        }
#pragma unroll kGatherUnroll
        for (int t = 0; t < cnt; ++t) {
          int c;
          R av, bv;
          if constexpr (kSrec) {
            srec_get<R>(srec, t, c, av, bv);
          } else {
            c = __shfl_sync(0xffffffffu, cl, t);
            av = __shfl_sync(0xffffffffu, avl, t);
            bv = __shfl_sync(0xffffffffu, bvl, t);
          }
          // byte offset c * W * sizeof(C) as one 32 x 32 -> 64-bit multiply-add (c >= 0)
          const Vec<R, VEC> x = ldv<R, VEC>(reinterpret_cast<const C *>(rlane + (unsigned long long)(unsigned)c * wbytes));
#pragma unroll
          for (int v = 0; v < VEC; ++v) {
            sa[v].x = fma(av, x.z[v].x, sa[v].x);
            sa[v].y = fma(av, x.z[v].y, sa[v].y);
            sb[v].x = fma(bv, x.z[v].x, sb[v].x);
            sb[v].y = fma(bv, x.z[v].y, sb[v].y);
          }
        }
      }
    };
    // p = r + beta p, q = s + beta q for the row, and its mu partial
    auto finish_row = [&](int64_t i, const C (&sa)[VEC], const C (&sb)[VEC], const Vec<R, VEC> &rv, Vec<R, VEC> pv, Vec<R, VEC> qv) {
      const size_t off = (size_t)i * a.W + w0;
#pragma unroll
      for (int v = 0; v < VEC; ++v) {
        const C be = to_c<R>(a.ws[w0 + v].beta);
        const C sg = a.sig[(w0 + v) & (a.mp - 1)];
        const C s = cfms(sg, sb[v], sa[v]);  // A r - sigma B r
        // a fresh start (refinement step) has p = r and q = (A - sigma B) r
        const C pn = FRESH ? rv.z[v] : cfma(be, pv.z[v], rv.z[v]);
        const C qn = FRESH ? s : cfma(be, qv.z[v], s);
        pv.z[v] = pn;
        qv.z[v] = qn;
        acc[v][0] += pn.x * qn.x - pn.y * qn.y;
        acc[v][1] += pn.x * qn.y + pn.y * qn.x;
      }
      stv_cs<R, VEC>(a.p + off, pv);
      stv_cs<R, VEC>(a.q + off, qv);
    };
    auto load_own = [&](int64_t i, Vec<R, VEC> &rv, Vec<R, VEC> &pv, Vec<R, VEC> &qv) {
      const size_t off = (size_t)i * a.W + w0;
      rv = ldv<R, VEC>(a.r + off);
      if (!FRESH) {
        pv = ldv_cs<R, VEC>(a.p + off);
        qv = ldv_cs<R, VEC>(a.q + off);
      }
    };
    for (int64_t i = i0 + warp; i < i1; i += kWarps) {
      C sa[VEC], sb[VEC];
      Vec<R, VEC> rv, pv, qv;
      gather_row(i, sa, sb);
      load_own(i, rv, pv, qv);
      finish_row(i, sa, sb, rv, pv, qv);
    }
  }
  spmm_tail<R, VEC>(a, acc, w_tile0, rb, tile, a.nrb);
}

// Record walk of the grouped-row SpMM for one warp (grouped-row format, see CocgArgs):
// groups gfirst, gfirst + gstride, ... below ngroups.  Per group it accumulates, for this
// lane's VEC pairs of the gathered row (x row c at xlane + c * xbytes),
//   sa[j] += a_j(c) x_c,   sb[j] += b_j(c) x_c      (j < G, the group's rows)
// over the group's records and then calls epi(g, sa, sb); sa and sb start at zero for every
// group.  The records go chunk by chunk (grp_chunk<R>() records) through the warp's two shared-
// memory buffers: lane 0 stages the next chunk but one with a 1-D bulk copy, so the records
// arrive through the TMA engine while the lanes gather and multiply; all lanes read a record
// with broadcast loads.  FP32: packed FP32 FMAs on (a, a) x (x0, x1).  Waits are bounded
// (2 s, then *err and a drain of the outstanding copies); inconsistent offsets set *err = 2
// (and, with SLRF_GRP_COLCHECK, a record column out of range *err = 3, gathering row 0; by
// default the columns are checked once when the records are built).
template <typename R, int V, int G, bool BD, typename Epi>
__device__ __forceinline__ void grp_walk(const int64_t ngroups, const int64_t *__restrict__ gptr,
                                         const unsigned char *__restrict__ grec, int *err, const int64_t nx,
                                         const int64_t gfirst, const int64_t gstride, const char *xlane,
                                         const unsigned xbytes, unsigned char *sbuf, uint64_t *bar, Epi &&epi) {
  constexpr int VEC = V;
  constexpr int RS = grec_bytes<R, G, BD>();
  constexpr int CH = grp_chunk<R, BD>();
  static_assert(!BD || (G == 3 && CH % 3 == 0), "B-diagonal records: 3-row groups, whole triples per chunk");
  using C = cx_t<R>;
  const int lane = threadIdx.x & 31;
  const int64_t gb1 = ngroups;
  if (lane == 0) {
    mbar_init(bar, 1);
    mbar_init(bar + 1, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  auto nchunks = [&](int64_t g) -> int {
    const int64_t c = gptr[g + 1] - gptr[g];
    return c <= 0 ? 1 : (int)((c + CH - 1) / CH);
  };
  const int64_t nrec = gptr[ngroups];  // records in all (bounds of every copy)
  auto first = [&](int64_t g, int c, int &cnt) -> int64_t {
    const int64_t e0 = gptr[g] + (int64_t)c * CH, e1 = gptr[g + 1];
    cnt = (int)(e1 - e0 < CH ? e1 - e0 : CH);
    if (cnt < 0 || e0 < 0 || e0 + cnt > nrec) {
      if (cnt != 0) atomicCAS(err, 0, 2);  // inconsistent offsets: copy nothing
      cnt = 0;
    }
    return e0;
  };
  auto issue = [&](int b, int64_t g, int c) {
    if (lane == 0) {
      int cnt;
      const int64_t e0 = first(g, c, cnt);
      // the lanes' shared-memory reads of this buffer (ordered by the __syncwarp before
      // the call) precede the asynchronous proxy's writes
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      if (cnt > 0) {
        mbar_expect_tx(bar + b, (uint32_t)(cnt * RS));
        bulk_g2s(sbuf + (size_t)b * CH * RS, grec + (size_t)e0 * RS, (uint32_t)(cnt * RS), bar + b);
      } else {
        mbar_arrive(bar + b);
      }
    }
  };
  int64_t cg = gfirst, ng = cg;  // current item (group, chunk), next item
  int cc = 0, nc = 0;
  auto advance = [&](int64_t &g, int &c) {
    if (c + 1 < nchunks(g)) ++c;
    else { g += gstride; c = 0; }
  };
  issue(0, cg, cc);
  advance(ng, nc);
  if (ng < gb1) issue(1, ng, nc);
  uint32_t ph0 = 0, ph1 = 0;
  int b = 0;
  bool failed = false;
  C sa[G][VEC], sb[G][VEC];
#pragma unroll
  for (int j = 0; j < G; ++j)
#pragma unroll
    for (int v = 0; v < VEC; ++v) { sa[j][v] = cmake<C>(0, 0); sb[j][v] = cmake<C>(0, 0); }
  while (cg < gb1) {
    if (!mbar_wait(bar + b, b ? ph1 : ph0, err, 1)) { failed = true; break; }
    if (b) ph1 ^= 1u; else ph0 ^= 1u;
    int cnt;
    first(cg, cc, cnt);
    const unsigned char *rb_ = sbuf + (size_t)b * CH * RS;
    if constexpr (BD) {
      // whole node triples: record t + d holds column 3J + d, whose B value belongs to row d
      // (a malformed tail shorter than a triple is skipped, never read past the chunk)
#pragma unroll kGrpUnrollBD
      for (int t = 0; t + 2 < cnt; t += 3) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const unsigned char *rp = rb_ + (t + d) * RS;
          const int c = *reinterpret_cast<const int *>(rp + grec_col<R, G, true>());
          const Vec<R, VEC> x = ldv<R, VEC>(reinterpret_cast<const C *>(xlane + (unsigned long long)(unsigned)c * xbytes));
          if constexpr (sizeof(R) == 4) {
            const float4 r4 = *reinterpret_cast<const float4 *>(rp);  // a0, a1, a2, b
            const float2 a0 = make_float2(r4.x, r4.x), a1 = make_float2(r4.y, r4.y), a2 = make_float2(r4.z, r4.z);
            const float2 bv = make_float2(r4.w, r4.w);
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
              sa[0][v] = ffma2(a0, x.z[v], sa[0][v]);
              sa[1][v] = ffma2(a1, x.z[v], sa[1][v]);
              sa[2][v] = ffma2(a2, x.z[v], sa[2][v]);
              sb[d][v] = ffma2(bv, x.z[v], sb[d][v]);
            }
          } else {
            const double2 r01 = reinterpret_cast<const double2 *>(rp)[0];  // a0, a1
            const double2 r23 = reinterpret_cast<const double2 *>(rp)[1];  // a2, b
            const double av[3] = {r01.x, r01.y, r23.x};
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
#pragma unroll
              for (int j = 0; j < 3; ++j) {
                sa[j][v].x = fma(av[j], x.z[v].x, sa[j][v].x);
                sa[j][v].y = fma(av[j], x.z[v].y, sa[j][v].y);
              }
              sb[d][v].x = fma(r23.y, x.z[v].x, sb[d][v].x);
              sb[d][v].y = fma(r23.y, x.z[v].y, sb[d][v].y);
            }
          }
        }
      }
    } else {
#pragma unroll kGrpUnroll
    for (int t = 0; t < cnt; ++t) {
      const unsigned char *rp = rb_ + t * RS;
      int c = *reinterpret_cast<const int *>(rp + grec_col<R, G>());
      if constexpr (SLRF_GRP_COLCHECK != 0) {
        if ((unsigned)c >= (unsigned)nx) {  // a corrupt record: flag it, gather row 0
          atomicCAS(err, 0, 3);
          (void)CHK(21, c, nx);
          c = 0;
        }
      }
      const Vec<R, VEC> x = ldv<R, VEC>(reinterpret_cast<const C *>(xlane + (unsigned long long)(unsigned)c * xbytes));
      // the record's 2 G values in 16-byte broadcast loads
      constexpr int NV = (grec_col<R, G>() + 15) / 16;
      float4 rv4[NV];
#pragma unroll
      for (int j = 0; j < NV; ++j) rv4[j] = reinterpret_cast<const float4 *>(rp)[j];
      const float *rvf = reinterpret_cast<const float *>(rv4);
      if constexpr (sizeof(R) == 4) {
#pragma unroll
        for (int j = 0; j < G; ++j) {
          const float2 av = SLRF_GRP_SPLAT ? make_float2(rvf[2 * j], rvf[2 * j + 1]) : make_float2(rvf[j], rvf[j]);
          const float2 bv = SLRF_GRP_SPLAT ? make_float2(rvf[2 * (G + j)], rvf[2 * (G + j) + 1])
                                           : make_float2(rvf[G + j], rvf[G + j]);
#pragma unroll
          for (int v = 0; v < VEC; ++v) {
            sa[j][v] = ffma2(av, x.z[v], sa[j][v]);
            sb[j][v] = ffma2(bv, x.z[v], sb[j][v]);
          }
        }
      } else {
        const double *rvd = reinterpret_cast<const double *>(rv4);
#pragma unroll
        for (int j = 0; j < G; ++j) {
          const double av = rvd[j];
          const double bv = rvd[G + j];
#pragma unroll
          for (int v = 0; v < VEC; ++v) {
            sa[j][v].x = fma(av, x.z[v].x, sa[j][v].x);
            sa[j][v].y = fma(av, x.z[v].y, sa[j][v].y);
            sb[j][v].x = fma(bv, x.z[v].x, sb[j][v].x);
            sb[j][v].y = fma(bv, x.z[v].y, sb[j][v].y);
          }
        }
      }
    }
    }
    if (cc + 1 >= nchunks(cg)) {
      epi(cg, sa, sb);  // the group's last chunk
#pragma unroll
      for (int j = 0; j < G; ++j)
#pragma unroll
        for (int v = 0; v < VEC; ++v) { sa[j][v] = cmake<C>(0, 0); sb[j][v] = cmake<C>(0, 0); }
    }
    __syncwarp();
    // stage the item after next into the buffer just read
    int64_t g2 = ng;
    int c2 = nc;
    if (g2 < gb1) {
      advance(g2, c2);
      if (g2 < gb1) issue(b, g2, c2);
    }
    cg = ng;
    cc = nc;
    ng = g2;
    nc = c2;
    b ^= 1;
  }
  if (failed) {
    // wait (bounded) for the copies this warp may still have in flight, then leave
    if (lane == 0) {
      mbar_wait(bar + b, b ? ph1 : ph0, err, 1);
      if (ng < gb1) mbar_wait(bar + (b ^ 1), b ? ph0 : ph1, err, 1);
    }
    __syncwarp();
  }
}

// s = (A - sigma B) r for groups of G consecutive rows that share one union column list
// (grouped-row format): every gathered row of r feeds all G rows, so a row costs union/G
// gathers instead of its own count (a 3-dof elasticity node: 27 instead of 81).  Then, per
// row, p = r + beta p, q = s + beta q and the mu partials.
template <typename R, int V, int G, bool BD, bool FRESH>
__device__ __forceinline__ void cocg_spmm_grp_body(const CocgArgs<R> &a, const int rb, const int tile) {
  constexpr int VEC = V;
  constexpr int RS = grec_bytes<R, G, BD>();
  using C = cx_t<R>;
  extern __shared__ __align__(128) unsigned char grp_smem[];
  __shared__ __align__(8) uint64_t s_bar[kWarps][2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int w_tile0 = tile * 32 * VEC;
  const int w0 = w_tile0 + lane * VEC;
  // (beta and the poles are read again in each group's epilogue: not held across the walk)
  bool any_act = false;
#pragma unroll
  for (int v = 0; v < VEC; ++v) any_act |= a.ws[w0 + v].active != 0;
  const bool warp_act = __any_sync(0xffffffffu, any_act);
  R acc[VEC][2];
#pragma unroll
  for (int v = 0; v < VEC; ++v) acc[v][0] = acc[v][1] = R(0);
  // Interleaved assignment: block rb takes the stripes rb, rb + nrb, rb + 2 nrb, ... of
  // kWarps consecutive groups (one per warp).  The blocks in flight then sweep the matrix
  // together through a window of about nrb stripes, so a gathered row of r is reused by all
  // the groups that need it while it is still in L2, also when one column tile of r is
  // larger than L2 (nrb is one resident wave of this kernel).
  const int64_t gstride = (int64_t)a.nrb * kWarps;
  const int64_t gfirst = (int64_t)rb * kWarps + warp;
  if (warp_act && gfirst < a.ngroups) {
    auto epi = [&](int64_t g, const C (&sa)[G][VEC], const C (&sb)[G][VEC]) {
      C sg[VEC], be[VEC];
#pragma unroll
      for (int v = 0; v < VEC; ++v) {
        be[v] = to_c<R>(a.ws[w0 + v].beta);
        sg[v] = a.sig[(w0 + v) & (a.mp - 1)];
      }
#pragma unroll
      for (int j = 0; j < G; ++j) {
        const int64_t i = g * G + j;
        if (i < a.n) {
          const size_t off = (size_t)i * a.W + w0;
          if (!CHK(20, off + VEC - 1, (long long)a.n * a.W)) continue;
          const Vec<R, VEC> rv = ldv<R, VEC>(a.r + off);
          Vec<R, VEC> pv, qv;
          if (!FRESH) {
            pv = ldv_cs<R, VEC>(a.p + off);
            qv = ldv_cs<R, VEC>(a.q + off);
          }
#pragma unroll
          for (int v = 0; v < VEC; ++v) {
            const C sv = cfms(sg[v], sb[j][v], sa[j][v]);  // A r - sigma B r
            const C pn = FRESH ? rv.z[v] : cfma(be[v], pv.z[v], rv.z[v]);
            const C qn = FRESH ? sv : cfma(be[v], qv.z[v], sv);
            pv.z[v] = pn;
            qv.z[v] = qn;
            acc[v][0] += pn.x * qn.x - pn.y * qn.y;
            acc[v][1] += pn.x * qn.y + pn.y * qn.x;
          }
          stv_cs<R, VEC>(a.p + off, pv);
          stv_cs<R, VEC>(a.q + off, qv);
        }
      }
    };
    grp_walk<R, VEC, G, BD>(a.ngroups, a.gptr, a.grec, a.err, a.n, gfirst, gstride,
                            reinterpret_cast<const char *>(a.r + w0), (unsigned)a.W * (unsigned)sizeof(C),
                            grp_smem + (size_t)warp * 2 * grp_chunk<R, BD>() * RS, s_bar[warp], epi);
  }
  spmm_tail<R, VEC>(a, acc, w_tile0, rb, tile, a.nrb);
}

// ------------------------------------------------------------------------------ residual
// Refinement step s >= 2 of the FP32 path: the FP64 residual of the accumulated correction
//   R = r0 - (A - sigma B) D,   r0 = c_w gscale_c g,   D in FP64,
// written as the new FP32 right-hand side r (p and q follow in the fresh SpMM); new
// scalars rho = R^T R, ||R||^2 per w.  Every column with a nonzero residual (and no
// earlier breakdown) is refined; its FP32 solve stops at tol ||R|| or It_max.
template <typename R, int V>
__device__ __forceinline__ void cocg_residual_body(const CocgArgs<R> &a, const int rb, const int tile) {
  constexpr int VEC = V;
  using C = cx_t<R>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int w_tile0 = tile * 32 * VEC;
  const int w0 = w_tile0 + lane * VEC;
  double2 sg[VEC], cf[VEC];
  int cidx[VEC];
  bool ok[VEC];
#pragma unroll
  for (int v = 0; v < VEC; ++v) {
    const int w = w0 + v;
    sg[v] = a.sig64[w & (a.mp - 1)];
    cidx[v] = w / a.mp;
    ok[v] = cidx[v] < a.k;
    double2 c = a.cfac[w];
    if (a.gscale != nullptr && ok[v]) {
      const double gs = a.gscale[cidx[v]];
      c.x *= gs;
      c.y *= gs;
    }
    cf[v] = c;
  }
  constexpr int NQ = 3;
  double acc[VEC][NQ];
#pragma unroll
  for (int v = 0; v < VEC; ++v)
#pragma unroll
    for (int qq = 0; qq < NQ; ++qq) acc[v][qq] = 0.0;
  const int64_t i0 = (int64_t)rb * a.rows_per_block;
  const int64_t i1 = (i0 + a.rows_per_block < a.n ? i0 + a.rows_per_block : a.n);
  for (int64_t i = i0 + warp; i < i1; i += kWarps) {
    double2 sa[VEC], sb[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) { sa[v] = make_double2(0, 0); sb[v] = make_double2(0, 0); }
    const int64_t rs = a.rowptr[i], re = a.rowptr[i + 1];
    for (int64_t e0 = rs; e0 < re; e0 += 32) {
      const int cnt = (int)(re - e0 < 32 ? re - e0 : 32);
      int cl = 0;
      double avl = 0, bvl = 0;
      if (lane < cnt) { cl = a.col[e0 + lane]; avl = a.valA64[e0 + lane]; bvl = a.valB64[e0 + lane]; }
      for (int t = 0; t < cnt; ++t) {
        const int c = __shfl_sync(0xffffffffu, cl, t);
        const double av = __shfl_sync(0xffffffffu, avl, t);
        const double bv = __shfl_sync(0xffffffffu, bvl, t);
        const double2 *xr = a.D64 + (size_t)c * a.W + w0;
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
          const double2 x = xr[v];
          sa[v].x = fma(av, x.x, sa[v].x);
          sa[v].y = fma(av, x.y, sa[v].y);
          sb[v].x = fma(bv, x.x, sb[v].x);
          sb[v].y = fma(bv, x.y, sb[v].y);
        }
      }
    }
    const size_t off = (size_t)i * a.W + w0;
    Vec<R, VEC> rv;
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
      const double g = ok[v] ? a.g[(size_t)i * a.ldg + cidx[v]] : 0.0;
      // r0 - (A D - sigma B D)
      const double mdx = sa[v].x - (sg[v].x * sb[v].x - sg[v].y * sb[v].y);
      const double mdy = sa[v].y - (sg[v].x * sb[v].y + sg[v].y * sb[v].x);
      C r;
      r.x = (R)(cf[v].x * g - mdx);
      r.y = (R)(cf[v].y * g - mdy);
      rv.z[v] = r;
      const double rx = (double)r.x, ry = (double)r.y;
      acc[v][0] += rx * rx - ry * ry;
      acc[v][1] += 2.0 * rx * ry;
      acc[v][2] += rx * rx + ry * ry;
    }
    stv<R, VEC>(a.r + off, rv);
  }
  double out[NQ];
  int w;
  if (!block_then_grid_reduce<VEC, NQ>(acc, a.W, w_tile0, rb, a.nrb, a.partial, a.counters + tile, out, w))
    return;
  if (threadIdx.x < 32 * VEC) {
    WScal s = a.ws[w];
    const bool valid = (w / a.mp) < a.k && (w & (a.mp - 1)) < a.m;
    s.rho = make_double2(out[0], out[1]);
    s.r0n2 = out[2];
    s.rn2 = out[2];
    s.iters = 0;
    s.beta = make_double2(0.0, 0.0);
    s.alpha = make_double2(0.0, 0.0);
    s.active = (valid && s.brk == 0 && out[2] > 0.0) ? 1 : 0;
    a.ws[w] = s;
  }
}

// ------------------------------------------------------------------------------ kernels
// Single problem: blockIdx.x = row block, blockIdx.y = tile.
template <typename R, int V>
__global__ void __launch_bounds__(kThreads, (cocg_minb<R, V>())) cocg_init_kernel(const CocgArgs<R> a) {
  cocg_init_body<R, V>(a, blockIdx.x, blockIdx.y);
}
template <typename R, int V, bool FIRST, int FM>
__global__ void __launch_bounds__(kThreads, (cocg_minb<R, V>())) cocg_update_kernel(const CocgArgs<R> a, int tile0) {
  cocg_update_body<R, V, FIRST, FM>(a, blockIdx.x, tile0 + blockIdx.y);
}
// Two groups of tiles in one launch: the SpMM of tiles [s0, s0 + ns) and the update of tiles
// [u0, u0 + nu).  Tiles are independent systems (own scalars, partial slots and counters),
// so the two run side by side: the SpMM is bound by the FP64 pipe (or by the gather path
// in FP32), the update by HBM.  Blocks alternate between the two kinds so that both are
// resident from the start; within each kind the row block varies fastest.
// resident blocks per SM of the grouped SpMM (more registers: G rows of accumulators)
template <typename R, int V, int G> __host__ __device__ constexpr int cocg_grp_minb() {
  return G == 1 ? cocg_minb<R, V>() : SLRF_GRP_MINB;
}
template <typename R, int V, bool FIRST, int FM>
__global__ void __launch_bounds__(kThreads, (cocg_minb<R, V>())) cocg_dual_kernel(const CocgArgs<R> a, int s0, int ns,
                                                                              int u0, int nu) {
  const int NS = a.nrb * ns, NU = a.nrb * nu;
  const int both = 2 * (NS < NU ? NS : NU);
  const int b = blockIdx.x;
  bool spmm;
  int item;
  if (b < both) {
    spmm = (b & 1) == 0;
    item = b >> 1;
  } else {
    spmm = NS > NU;
    item = (b - both) + (NS < NU ? NS : NU);
  }
  if (spmm) cocg_spmm_body<R, V, false>(a, item % a.nrb, s0 + item / a.nrb);
  else cocg_update_body<R, V, FIRST, FM>(a, item % a.nrb, u0 + item / a.nrb);
}
template <typename R, int V, bool FRESH>
__global__ void __launch_bounds__(kThreads, (cocg_minb<R, V>())) cocg_spmm_kernel(const CocgArgs<R> a) {
  cocg_spmm_body<R, V, FRESH>(a, blockIdx.x, blockIdx.y);
}
template <typename R, int V, int G, bool BD, bool FRESH>
__global__ void __launch_bounds__(kThreads, (cocg_grp_minb<R, V, G>())) cocg_spmm_grp_kernel(const CocgArgs<R> a) {
  cocg_spmm_grp_body<R, V, G, BD, FRESH>(a, blockIdx.x, blockIdx.y);
}
template <typename R, int V>
__global__ void __launch_bounds__(kThreads, 2) cocg_residual_kernel(const CocgArgs<R> a) {
  cocg_residual_body<R, V>(a, blockIdx.x, blockIdx.y);
}

// Many problems in one persistent launch: work item t of the list belongs to problem p
// with prefix[p] <= t < prefix[p+1]; inside a problem the row block varies fastest and
// the tile slowest (as in the single-problem grid).  Blocks stride over the items.
__device__ __forceinline__ int batch_problem(const int *prefix, int P, int item) {
  int lo = 0, hi = P;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (prefix[mid] <= item) lo = mid;
    else hi = mid;
  }
  return lo;
}
#define SLRF_BATCH_LOOP(BODY)                                               \
  const int total = prefix[P];                                              \
  for (int item = blockIdx.x; item < total; item += gridDim.x) {            \
    const int pb = batch_problem(prefix, P, item);                          \
    const CocgArgs<R> &a = args[pb];                                        \
    const int local = item - prefix[pb];                                    \
    BODY;                                                                   \
    __syncthreads();                                                        \
  }
// (the batched path runs plain CSR only: lane width cocg_vec_csr<R>(), checked by the host)
template <typename R>
__global__ void __launch_bounds__(kThreads, (cocg_minb<R, cocg_vec_csr<R>()>())) cocg_init_batched(const CocgArgs<R> *args, const int *prefix, int P) {
  SLRF_BATCH_LOOP((cocg_init_body<R, cocg_vec_csr<R>()>(a, local % a.nrb, local / a.nrb)))
}
template <typename R, bool FIRST, int FM>
__global__ void __launch_bounds__(kThreads, (cocg_minb<R, cocg_vec_csr<R>()>())) cocg_update_batched(const CocgArgs<R> *args, const int *prefix, int P) {
  SLRF_BATCH_LOOP((cocg_update_body<R, cocg_vec_csr<R>(), FIRST, FM>(a, local % a.nrb, local / a.nrb)))
}
template <typename R, bool FRESH>
__global__ void __launch_bounds__(kThreads, (cocg_minb<R, cocg_vec_csr<R>()>())) cocg_spmm_batched(const CocgArgs<R> *args, const int *prefix, int P) {
  SLRF_BATCH_LOOP((cocg_spmm_body<R, cocg_vec_csr<R>(), FRESH>(a, local % a.nrb, local / a.nrb)))
}
template <typename R>
__global__ void __launch_bounds__(kThreads, 2) cocg_residual_batched(const CocgArgs<R> *args, const int *prefix, int P) {
  SLRF_BATCH_LOOP((cocg_residual_body<R, cocg_vec_csr<R>()>(a, local % a.nrb, local / a.nrb)))
}
#undef SLRF_BATCH_LOOP

// ------------------------------------------------------------------------------ grouped-row format
// One thread per group of G consecutive rows: a G-way merge of the rows' sorted column
// lists.  Count pass: distinct columns; fill pass: one record per distinct column with the
// G rows' A and B values (zero where a row lacks the column) and the column index.
__global__ void grp_count_kernel(int64_t n, int G, const int64_t *__restrict__ rowptr,
                                 const int32_t *__restrict__ col, int *__restrict__ cnt) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i0 = g * G;
  if (i0 >= n) return;
  int64_t pos[4], end[4];
  const int rows = (int)(n - i0 < G ? n - i0 : G);
  for (int j = 0; j < rows; ++j) { pos[j] = rowptr[i0 + j]; end[j] = rowptr[i0 + j + 1]; }
  int c = 0;
  for (;;) {
    int32_t m = INT32_MAX;
    bool any = false;
    for (int j = 0; j < rows; ++j)
      if (pos[j] < end[j]) { any = true; m = min(m, col[pos[j]]); }
    if (!any) break;
    ++c;
    for (int j = 0; j < rows; ++j)
      if (pos[j] < end[j] && col[pos[j]] == m) ++pos[j];
  }
  cnt[g] = c;
}

template <typename R, int G>
__global__ void grp_fill_kernel(int64_t n, const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                                const double *__restrict__ valA, const double *__restrict__ valB,
                                const int64_t *__restrict__ gptr, unsigned char *__restrict__ rec) {
  constexpr int RS = grec_bytes<R, G>();
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i0 = g * G;
  if (i0 >= n) return;
  int64_t pos[G], end[G];
  const int rows = (int)(n - i0 < G ? n - i0 : G);
  for (int j = 0; j < G; ++j) {
    pos[j] = j < rows ? rowptr[i0 + j] : 0;
    end[j] = j < rows ? rowptr[i0 + j + 1] : 0;
  }
  int64_t e = gptr[g];
  for (;;) {
    int32_t m = INT32_MAX;
    bool any = false;
    for (int j = 0; j < G; ++j)
      if (pos[j] < end[j]) { any = true; m = min(m, col[pos[j]]); }
    if (!any) break;
    unsigned char *rp = rec + (size_t)e * RS;
    for (int t = 0; t < RS / 4; ++t) reinterpret_cast<int *>(rp)[t] = 0;  // padding too
    for (int j = 0; j < G; ++j) {
      double av = 0.0, bv = 0.0;
      if (pos[j] < end[j] && col[pos[j]] == m) {
        av = valA[pos[j]];
        bv = valB[pos[j]];
        ++pos[j];
      }
      if constexpr (sizeof(R) == 4 && SLRF_GRP_SPLAT) {
        reinterpret_cast<float2 *>(rp)[j] = make_float2((float)av, (float)av);
        reinterpret_cast<float2 *>(rp)[G + j] = make_float2((float)bv, (float)bv);
      } else if constexpr (sizeof(R) == 4) {
        reinterpret_cast<float *>(rp)[j] = (float)av;
        reinterpret_cast<float *>(rp)[G + j] = (float)bv;
      } else {
        reinterpret_cast<double *>(rp)[j] = av;
        reinterpret_cast<double *>(rp)[G + j] = bv;
      }
    }
    *reinterpret_cast<int *>(rp + grec_col<R, G>()) = m;
    ++e;
  }
}

// Records of the grouped format: every column in [0, n), offsets non-decreasing from 0.
// *flag = 1 otherwise.
template <typename R, int G, bool BD>
__global__ void grp_check_kernel(int64_t n, int64_t ngroups, const int64_t *__restrict__ gptr,
                                 const unsigned char *__restrict__ rec, int *flag) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t nrec = gptr[ngroups];
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += stride)
    if (gptr[g] < 0 || gptr[g + 1] < gptr[g] || (BD && (gptr[g + 1] - gptr[g]) % 3 != 0)) atomicExch(flag, 1);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nrec; e += stride) {
    const int c = *reinterpret_cast<const int *>(rec + (size_t)e * grec_bytes<R, G, BD>() + grec_col<R, G, BD>());
    if (c < 0 || (int64_t)c >= n) atomicExch(flag, 1);
  }
}
template <typename R>
void grp_check(int64_t n, int G, int64_t ngroups, const int64_t *gptr, const unsigned char *rec, int *flag,
               int blocks, cudaStream_t st, bool bd) {
  switch (G) {
    case 2: grp_check_kernel<R, 2, false><<<blocks, 256, 0, st>>>(n, ngroups, gptr, rec, flag); break;
    case 3:
      if (bd) grp_check_kernel<R, 3, true><<<blocks, 256, 0, st>>>(n, ngroups, gptr, rec, flag);
      else grp_check_kernel<R, 3, false><<<blocks, 256, 0, st>>>(n, ngroups, gptr, rec, flag);
      break;
    case 4: grp_check_kernel<R, 4, false><<<blocks, 256, 0, st>>>(n, ngroups, gptr, rec, flag); break;
    default: break;
  }
}
template void grp_check<float>(int64_t, int, int64_t, const int64_t *, const unsigned char *, int *, int, cudaStream_t,
                               bool);
template void grp_check<double>(int64_t, int, int64_t, const int64_t *, const unsigned char *, int *, int,
                                cudaStream_t, bool);

// B-diagonal records: every group of 3 rows (rows 3g .. 3g + 2, node g) has its records in
// aligned column triples (position t holds column 3J + t mod 3, positions t, t + 1, t + 2 of a
// triple the same J), and every B value off the row c mod 3 is zero.  One thread per group.
template <typename R>
__global__ void grp_bd_detect_kernel(int64_t n, int64_t ngroups, const int64_t *__restrict__ gptr,
                                     const unsigned char *__restrict__ rec, int *flag) {
  constexpr int RS = grec_bytes<R, 3>();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += stride) {
    const int64_t e0 = gptr[g], e1 = gptr[g + 1];
    bool ok = (e1 - e0) % 3 == 0 && 3 * g + 2 < n;
    for (int64_t e = e0; ok && e < e1; ++e) {
      const unsigned char *rp = rec + (size_t)e * RS;
      const int c = *reinterpret_cast<const int *>(rp + grec_col<R, 3>());
      const int t = (int)((e - e0) % 3);
      if (c % 3 != t) ok = false;
      if (t > 0 && c != *reinterpret_cast<const int *>(rp - RS + grec_col<R, 3>()) + 1) ok = false;
      for (int j = 0; j < 3; ++j) {
        const double b = sizeof(R) == 8 ? reinterpret_cast<const double *>(rp)[3 + j]
                                        : (double)reinterpret_cast<const float *>(rp)[SLRF_GRP_SPLAT ? 2 * (3 + j) : 3 + j];
        if (j != t && b != 0.0) ok = false;
      }
    }
    if (!ok) atomicExch(flag, 1);
  }
}
template <typename R>
__global__ void grp_bd_convert_kernel(int64_t nrec, const unsigned char *__restrict__ rec, unsigned char *bdrec) {
  constexpr int RS = grec_bytes<R, 3>(), RB = grec_bytes<R, 3, true>();
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nrec) return;
  const unsigned char *rp = rec + (size_t)e * RS;
  unsigned char *bp = bdrec + (size_t)e * RB;
  const int c = *reinterpret_cast<const int *>(rp + grec_col<R, 3>());
  const int d = c % 3;
  for (int t = 0; t < RB / 4; ++t) reinterpret_cast<int *>(bp)[t] = 0;
  if constexpr (sizeof(R) == 8) {
    const double *v = reinterpret_cast<const double *>(rp);
    double *o = reinterpret_cast<double *>(bp);
    o[0] = v[0]; o[1] = v[1]; o[2] = v[2]; o[3] = v[3 + d];
  } else {
    const float *v = reinterpret_cast<const float *>(rp);
    float *o = reinterpret_cast<float *>(bp);
    const int s = SLRF_GRP_SPLAT ? 2 : 1;
    o[0] = v[0]; o[1] = v[s]; o[2] = v[2 * s]; o[3] = v[s * (3 + d)];
  }
  *reinterpret_cast<int *>(bp + grec_col<R, 3, true>()) = c;
}
template <typename R>
void grp_bd_detect(int64_t n, int64_t ngroups, const int64_t *gptr, const unsigned char *rec, int *flag, int blocks,
                   cudaStream_t st) {
  grp_bd_detect_kernel<R><<<blocks, 256, 0, st>>>(n, ngroups, gptr, rec, flag);
}
template <typename R>
void grp_bd_convert(int64_t nrec, const unsigned char *rec, unsigned char *bdrec, cudaStream_t st) {
  if (nrec > 0) grp_bd_convert_kernel<R><<<(unsigned)((nrec + 255) / 256), 256, 0, st>>>(nrec, rec, bdrec);
}
template void grp_bd_detect<float>(int64_t, int64_t, const int64_t *, const unsigned char *, int *, int, cudaStream_t);
template void grp_bd_detect<double>(int64_t, int64_t, const int64_t *, const unsigned char *, int *, int, cudaStream_t);
template void grp_bd_convert<float>(int64_t, const unsigned char *, unsigned char *, cudaStream_t);
template void grp_bd_convert<double>(int64_t, const unsigned char *, unsigned char *, cudaStream_t);

void grp_count(int64_t n, int G, const int64_t *rowptr, const int32_t *col, int *cnt, cudaStream_t st) {
  const int64_t ng = (n + G - 1) / G;
  grp_count_kernel<<<(unsigned)((ng + 255) / 256), 256, 0, st>>>(n, G, rowptr, col, cnt);
}
template <typename R>
void grp_fill(int64_t n, int G, const int64_t *rowptr, const int32_t *col, const double *valA, const double *valB,
              const int64_t *gptr, unsigned char *rec, cudaStream_t st) {
  const int64_t ng = (n + G - 1) / G;
  const unsigned blocks = (unsigned)((ng + 255) / 256);
  switch (G) {
    case 2: grp_fill_kernel<R, 2><<<blocks, 256, 0, st>>>(n, rowptr, col, valA, valB, gptr, rec); break;
    case 3: grp_fill_kernel<R, 3><<<blocks, 256, 0, st>>>(n, rowptr, col, valA, valB, gptr, rec); break;
    case 4: grp_fill_kernel<R, 4><<<blocks, 256, 0, st>>>(n, rowptr, col, valA, valB, gptr, rec); break;
    default: grp_fill_kernel<R, 1><<<blocks, 256, 0, st>>>(n, rowptr, col, valA, valB, gptr, rec); break;
  }
}
template void grp_fill<float>(int64_t, int, const int64_t *, const int32_t *, const double *, const double *,
                              const int64_t *, unsigned char *, cudaStream_t);
template void grp_fill<double>(int64_t, int, const int64_t *, const int32_t *, const double *, const double *,
                               const int64_t *, unsigned char *, cudaStream_t);

// ------------------------------------------------------------------------------ prepare
__global__ void cocg_prepare_kernel(int W, int k, int m, int mp, const double2 *sig, const double2 *wt,
                                    const double *theta, double2 *cfac, double *coefV, WScal *ws) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  const int j = w & (mp - 1), c = w / mp;
  const bool valid = (c < k) && (j < m);
  WScal s;
  s.alpha = s.beta = s.rho = make_double2(0.0, 0.0);
  s.r0n2 = s.rn2 = 0.0;
  s.active = valid ? 1 : 0;
  s.iters = 0;
  s.brk = 0;
  s.iters_total = 0;
  ws[w] = s;
  double2 cf = make_double2(1.0, 0.0);
  if (theta != nullptr && valid) {
    // warm start: r0 = (A - theta B) v / (sigma - theta)
    cf = cdiv(make_double2(1.0, 0.0), make_double2(sig[j].x - theta[c], sig[j].y));
  }
  cfac[w] = cf;
  if (j == 0 && c < k) {
    double phi = 0.0;
    if (theta != nullptr) {
      for (int jj = 0; jj < m; ++jj) {
        // Phi(theta) = sum_j 2 Re(w_j / (theta - sigma_j))
        const double2 z = cdiv(wt[jj], make_double2(theta[c] - sig[jj].x, -sig[jj].y));
        phi += 2.0 * z.x;
      }
    }
    coefV[c] = phi;
  }
}

// gscale[c] = 1 / max_i |g[i][c]| (1 for a zero column).  Positive doubles order like
// their bit patterns, so the column maximum is an integer atomicMax.
__global__ void col_absmax_kernel(int64_t n, int k, const double *g, int ld, unsigned long long *mx) {
  const int c = blockIdx.y * blockDim.x + threadIdx.x;
  if (c >= k) return;
  double m = 0.0;
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) m = fmax(m, fabs(g[i * ld + c]));
  atomicMax(mx + c, (unsigned long long)__double_as_longlong(m));
}
__global__ void col_scale_kernel(int k, const unsigned long long *mx, double *gscale) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= k) return;
  const double m = __longlong_as_double((long long)mx[c]);
  gscale[c] = (m > 0.0 && isfinite(m)) ? 1.0 / m : 1.0;
}
void col_scale(int64_t n, int k, const double *g, int ld, unsigned long long *tmp, double *gscale, cudaStream_t st) {
  cudaMemsetAsync(tmp, 0, k * sizeof(unsigned long long), st);
  dim3 grid((unsigned)(n < 512 ? n : 512), (k + 127) / 128);
  col_absmax_kernel<<<grid, 128, 0, st>>>(n, k, g, ld, tmp);
  col_scale_kernel<<<(k + 127) / 128, 128, 0, st>>>(k, tmp, gscale);
}

void cocg_prepare(int W, int k, int m, int mp, const double2 *sig, const double2 *wt, const double *theta,
                  double2 *cfac, double *coefV, WScal *ws, cudaStream_t st) {
  cocg_prepare_kernel<<<(W + 255) / 256, 256, 0, st>>>(W, k, m, mp, sig, wt, theta, cfac, coefV, ws);
}

template <typename R> static dim3 grid_of(const CocgArgs<R> &a) {
  return dim3((unsigned)a.nrb, (unsigned)(a.W / (32 * a.vec)));
}
// Calls f(std::integral_constant<int, V>) with the lane width a.vec as a constant.
template <typename R, typename F> static void with_vec(const CocgArgs<R> &a, F &&f) {
  if constexpr (sizeof(R) == 8) {
    f(std::integral_constant<int, 1>{});
  } else {
    if (a.vec == 4) f(std::integral_constant<int, 4>{});
    else f(std::integral_constant<int, 2>{});
  }
}
// Arguments a launch cannot use launch nothing: code 4 in *a.err (status SLRF_EINVAL).
template <typename R> static bool refuse(const CocgArgs<R> &a, cudaStream_t st) {
  // low byte only (a memset is allowed under stream capture); the flag starts at zero
  if (a.err != nullptr) cudaMemsetAsync(a.err, 4, 1, st);
  return false;
}
template <typename R> static bool args_guard(const CocgArgs<R> &a, cudaStream_t st) {
  return cocg_layout_ok(a) ? true : refuse(a, st);
}
template <typename R> static bool mode_guard(const CocgArgs<R> &a, int fm, cudaStream_t st) {
  return (cocg_layout_ok(a) && cocg_mode_ok(a, fm)) ? true : refuse(a, st);
}

template <typename R> void cocg_init(const CocgArgs<R> &a, cudaStream_t st) {
  if (!args_guard(a, st)) return;
  with_vec(a, [&](auto vc) {
    constexpr int V = decltype(vc)::value;
    cocg_init_kernel<R, V><<<grid_of(a), kThreads, 0, st>>>(a);
  });
}
template <typename R, int V>
static void update_launch(const CocgArgs<R> &a, bool first, int fm, dim3 g, int tile0, cudaStream_t st) {
#define UPD(F, M) cocg_update_kernel<R, V, F, M><<<g, kThreads, 0, st>>>(a, tile0)
  if (first) {
    switch (fm) {
      case kFinalNone: UPD(true, kFinalNone); break;
      case kFinalU: UPD(true, kFinalU); break;
      case kFinalStoreD: UPD(true, kFinalStoreD); break;
      case kFinalAddD: UPD(true, kFinalAddD); break;
      case kAccU: UPD(true, kAccU); break;
      case kAccUEnd: UPD(true, kAccUEnd); break;
      default: UPD(true, kFinalUFromD); break;
    }
  } else {
    switch (fm) {
      case kFinalNone: UPD(false, kFinalNone); break;
      case kFinalU: UPD(false, kFinalU); break;
      case kFinalStoreD: UPD(false, kFinalStoreD); break;
      case kFinalAddD: UPD(false, kFinalAddD); break;
      case kAccU: UPD(false, kAccU); break;
      case kAccUEnd: UPD(false, kAccUEnd); break;
      default: UPD(false, kFinalUFromD); break;
    }
  }
#undef UPD
}
template <typename R> void cocg_update(const CocgArgs<R> &a, bool first, int fm, cudaStream_t st, int tile0,
                                      int ntiles) {
  if (!mode_guard(a, fm, st)) return;
  dim3 g = grid_of(a);
  if (ntiles > 0) g.y = (unsigned)ntiles;
  with_vec(a, [&](auto vc) { update_launch<R, decltype(vc)::value>(a, first, fm, g, tile0, st); });
}
template <typename R, int V>
static void dual_launch(const CocgArgs<R> &a, int s0, int ns, int u0, int nu, bool first, int fm, cudaStream_t st) {
  const unsigned blocks = (unsigned)a.nrb * (unsigned)(ns + nu);
#define DUAL(F, M) cocg_dual_kernel<R, V, F, M><<<blocks, kThreads, 0, st>>>(a, s0, ns, u0, nu)
  if (first) {
    if (fm == kAccU) DUAL(true, kAccU);
    else DUAL(true, kFinalNone);  // a group's first update is never its last (It_max >= 2)
  } else {
    switch (fm) {
      case kFinalNone: DUAL(false, kFinalNone); break;
      case kFinalU: DUAL(false, kFinalU); break;
      case kFinalStoreD: DUAL(false, kFinalStoreD); break;
      case kFinalAddD: DUAL(false, kFinalAddD); break;
      case kAccU: DUAL(false, kAccU); break;
      case kAccUEnd: DUAL(false, kAccUEnd); break;
      default: DUAL(false, kFinalUFromD); break;
    }
  }
#undef DUAL
}
template <typename R> void cocg_dual(const CocgArgs<R> &a, int s0, int ns, int u0, int nu, bool first, int fm,
                                    cudaStream_t st) {
  if (!mode_guard(a, fm, st)) return;
  with_vec(a, [&](auto vc) { dual_launch<R, decltype(vc)::value>(a, s0, ns, u0, nu, first, fm, st); });
}
template <typename R, int V, int G> static void spmm_grp_launch(const CocgArgs<R> &a, cudaStream_t st, bool fresh) {
  if constexpr (G == 3) {
    if (a.bdiag) {
      constexpr int sm = grp_smem_bytes<R, 3, true>();
      if (fresh) cocg_spmm_grp_kernel<R, V, 3, true, true><<<grid_of(a), kThreads, sm, st>>>(a);
      else cocg_spmm_grp_kernel<R, V, 3, true, false><<<grid_of(a), kThreads, sm, st>>>(a);
      return;
    }
  }
  if (fresh) cocg_spmm_grp_kernel<R, V, G, false, true><<<grid_of(a), kThreads, grp_smem_bytes<R, G>(), st>>>(a);
  else cocg_spmm_grp_kernel<R, V, G, false, false><<<grid_of(a), kThreads, grp_smem_bytes<R, G>(), st>>>(a);
}
template <typename R, int V> static void spmm_launch(const CocgArgs<R> &a, cudaStream_t st, bool fresh) {
  switch (a.G) {
    case 2: spmm_grp_launch<R, V, 2>(a, st, fresh); return;
    case 3: spmm_grp_launch<R, V, 3>(a, st, fresh); return;
    case 4: spmm_grp_launch<R, V, 4>(a, st, fresh); return;
    default: break;
  }
  if (fresh) cocg_spmm_kernel<R, V, true><<<grid_of(a), kThreads, 0, st>>>(a);
  else cocg_spmm_kernel<R, V, false><<<grid_of(a), kThreads, 0, st>>>(a);
}
template <typename R> void cocg_spmm(const CocgArgs<R> &a, cudaStream_t st, bool fresh) {
  if (!args_guard(a, st)) return;
  with_vec(a, [&](auto vc) { spmm_launch<R, decltype(vc)::value>(a, st, fresh); });
}

// Dynamic shared memory above the default 48 KB for every grouped kernel instance
// (called once per process, before any launch or stream capture).
// ------------------------------------------------------------------------------ real SpMM
// Real products through the FP32 grouped records: each lane takes VEC pairs of adjacent real
// columns of x32, so the packed FMA (a, a) x (x_c, x_c+1) of the complex SpMM serves two real
// columns at once.  Grid (row blocks, column tiles of 64 VEC real columns); interleaved
// stripes as in the COCG SpMM.
constexpr int kReal32Vec = 4;  // pairs of real columns per lane
int grp_real32_ld(int k) {
  const int t = 64 * kReal32Vec;
  return (k + t - 1) / t * t;
}
__global__ void to_f32_scaled_kernel(int64_t n, int k, const double *__restrict__ X, int ldx,
                                     const double *__restrict__ s, float *__restrict__ Y, int ldy) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * ldy) return;
  const int64_t i = t / ldy;
  const int c = (int)(t - i * ldy);
  Y[t] = c < k ? (float)(s != nullptr ? X[i * ldx + c] * s[i] : X[i * ldx + c]) : 0.f;
}
struct GrpReal32 {
  int64_t n, ngroups;
  const int64_t *gptr;
  const unsigned char *grec;
  int *err;
  int nrb;
  const float *x;
  int ldx;
  int k;
  double *YA, *YB;
  int ldy;
  const double *yscale;
};
template <int G, bool BD>
__global__ void __launch_bounds__(kThreads, (cocg_grp_minb<float, kReal32Vec, G>())) spmm_grp_real32_kernel(const GrpReal32 a) {
  constexpr int VEC = kReal32Vec;
  constexpr int RS = grec_bytes<float, G, BD>();
  extern __shared__ __align__(128) unsigned char grp_smem[];
  __shared__ __align__(8) uint64_t s_bar[kWarps][2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c0 = (int)blockIdx.y * 64 * VEC + lane * 2 * VEC;  // the lane's pointer (see ldv): tile + 2 VEC lane
  // pair v of the lane (two real columns) sits at pair index 64 (v / 2) + 2 lane + v % 2 of the tile
  const int ct = (int)blockIdx.y * 64 * VEC;
  const int64_t gstride = (int64_t)a.nrb * kWarps;
  const int64_t gfirst = (int64_t)blockIdx.x * kWarps + warp;
  if (gfirst >= a.ngroups) return;  // warp-uniform; the kernel has no block-wide barrier
  auto epi = [&](int64_t g, const float2 (&sa)[G][VEC], const float2 (&sb)[G][VEC]) {
#pragma unroll
    for (int j = 0; j < G; ++j) {
      const int64_t i = g * G + j;
      if (i >= a.n) continue;
      const double ys = a.yscale != nullptr ? a.yscale[i] : 1.0;
#pragma unroll
      for (int v = 0; v < VEC; ++v)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int c = ct + 2 * (64 * (v / 2) + 2 * lane + (v % 2)) + e;
          if (c < a.k) {
            if (a.YA) a.YA[(size_t)i * a.ldy + c] = ys * (double)(e ? sa[j][v].y : sa[j][v].x);
            if (a.YB) a.YB[(size_t)i * a.ldy + c] = ys * (double)(e ? sb[j][v].y : sb[j][v].x);
          }
        }
    }
  };
  grp_walk<float, VEC, G, BD>(a.ngroups, a.gptr, a.grec, a.err, a.n, gfirst, gstride,
                              reinterpret_cast<const char *>(a.x + c0), (unsigned)a.ldx * 4u,
                              grp_smem + (size_t)warp * 2 * grp_chunk<float, BD>() * RS, s_bar[warp], epi);
}
void spmm_grp_real32(int64_t n, int G, int64_t ngroups, const int64_t *gptr, const unsigned char *grec, int *err,
                     int nrb, const double *X, int ldx, int k, const double *xscale, float *x32, double *YA,
                     double *YB, int ldy, const double *yscale, cudaStream_t st, bool bd) {
  if (n <= 0 || k <= 0 || nrb <= 0) return;
  const int ld32 = grp_real32_ld(k);
  const int64_t tot = n * ld32;
  to_f32_scaled_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, k, X, ldx, xscale, x32, ld32);
  GrpReal32 a{n, ngroups, gptr, grec, err, nrb, x32, ld32, k, YA, YB, ldy, yscale};
  const dim3 grid((unsigned)nrb, (unsigned)(ld32 / (64 * kReal32Vec)));
  switch (G) {
    case 2: spmm_grp_real32_kernel<2, false><<<grid, kThreads, grp_smem_bytes<float, 2>(), st>>>(a); break;
    case 3:
      if (bd) spmm_grp_real32_kernel<3, true><<<grid, kThreads, grp_smem_bytes<float, 3, true>(), st>>>(a);
      else spmm_grp_real32_kernel<3, false><<<grid, kThreads, grp_smem_bytes<float, 3>(), st>>>(a);
      break;
    case 4: spmm_grp_real32_kernel<4, false><<<grid, kThreads, grp_smem_bytes<float, 4>(), st>>>(a); break;
    default: break;
  }
}

// FP64 real products through FP64 B-diagonal records (3-row groups): a lane takes one
// double2 -- two adjacent real columns -- of the padded FP64 copy x64, so a warp covers 64
// columns per tile and the FMAs are those of the complex FP64 SpMM (A and B products per
// gathered row: 3 + 1).  Output row i is multiplied by yscale[i] (null: 1).
struct GrpReal64 {
  int64_t n, ngroups;
  const int64_t *gptr;
  const unsigned char *grec;
  int *err;
  int nrb;
  const double *x;
  int ldx;
  int k;
  double *YA, *YB;
  int ldy;
  const double *yscale;
};
int grp_real64_ld(int k) { return (k + 63) / 64 * 64; }
__global__ void to_f64_scaled_kernel(int64_t n, int k, const double *__restrict__ X, int ldx,
                                     const double *__restrict__ s, double *__restrict__ Y, int ldy) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * ldy) return;
  const int64_t i = t / ldy;
  const int c = (int)(t - i * ldy);
  Y[t] = c < k ? (s != nullptr ? X[i * ldx + c] * s[i] : X[i * ldx + c]) : 0.0;
}
__global__ void __launch_bounds__(kThreads, (cocg_grp_minb<double, 1, 3>())) spmm_grp_real64_kernel(const GrpReal64 a) {
  constexpr int RS = grec_bytes<double, 3, true>();
  extern __shared__ __align__(128) unsigned char grp_smem[];
  __shared__ __align__(8) uint64_t s_bar[kWarps][2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c0 = (int)blockIdx.y * 64 + 2 * lane;  // this lane's two real columns
  const int64_t gstride = (int64_t)a.nrb * kWarps;
  const int64_t gfirst = (int64_t)blockIdx.x * kWarps + warp;
  if (gfirst >= a.ngroups) return;  // warp-uniform; the kernel has no block-wide barrier
  auto epi = [&](int64_t g, const double2 (&sa)[3][1], const double2 (&sb)[3][1]) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int64_t i = g * 3 + j;
      if (i >= a.n) continue;
      const double ys = a.yscale != nullptr ? a.yscale[i] : 1.0;
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int c = c0 + e;
        if (c < a.k) {
          if (a.YA) a.YA[(size_t)i * a.ldy + c] = ys * (e ? sa[j][0].y : sa[j][0].x);
          if (a.YB) a.YB[(size_t)i * a.ldy + c] = ys * (e ? sb[j][0].y : sb[j][0].x);
        }
      }
    }
  };
  grp_walk<double, 1, 3, true>(a.ngroups, a.gptr, a.grec, a.err, a.n, gfirst, gstride,
                               reinterpret_cast<const char *>(a.x + c0), (unsigned)a.ldx * 8u,
                               grp_smem + (size_t)warp * 2 * grp_chunk<double, true>() * RS, s_bar[warp], epi);
}
void spmm_grp_real64(int64_t n, int64_t ngroups, const int64_t *gptr, const unsigned char *grec, int *err, int nrb,
                     const double *X, int ldx, int k, const double *xscale, double *x64, double *YA, double *YB,
                     int ldy, const double *yscale, cudaStream_t st) {
  if (n <= 0 || k <= 0 || nrb <= 0) return;
  const int ld64 = grp_real64_ld(k);
  const int64_t tot = n * ld64;
  to_f64_scaled_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, k, X, ldx, xscale, x64, ld64);
  GrpReal64 a{n, ngroups, gptr, grec, err, nrb, x64, ld64, k, YA, YB, ldy, yscale};
  const dim3 grid((unsigned)nrb, (unsigned)(ld64 / 64));
  spmm_grp_real64_kernel<<<grid, kThreads, grp_smem_bytes<double, 3, true>(), st>>>(a);
}

template <typename R, int V, int G> static void grp_attrs_v() {
  const int sm = grp_smem_bytes<R, G>();
  cudaFuncSetAttribute(cocg_spmm_grp_kernel<R, V, G, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  cudaFuncSetAttribute(cocg_spmm_grp_kernel<R, V, G, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if constexpr (G == 3) {
    const int sbd = grp_smem_bytes<R, 3, true>();
    cudaFuncSetAttribute(cocg_spmm_grp_kernel<R, V, 3, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sbd);
    cudaFuncSetAttribute(cocg_spmm_grp_kernel<R, V, 3, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sbd);
  }
}
template <typename R, int G> static void grp_attrs() {
  if constexpr (sizeof(R) == 8) {
    grp_attrs_v<R, 1, G>();
  } else {
    grp_attrs_v<R, 2, G>();
    grp_attrs_v<R, 4, G>();
    cudaFuncSetAttribute(spmm_grp_real32_kernel<G, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         grp_smem_bytes<float, G>());
    if constexpr (G == 3)
      cudaFuncSetAttribute(spmm_grp_real32_kernel<3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           grp_smem_bytes<float, 3, true>());
  }
}
void cocg_kernel_attrs() {
  static bool done = false;
  if (done) return;
  cudaFuncSetAttribute(spmm_grp_real64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       grp_smem_bytes<double, 3, true>());
  grp_attrs<float, 2>();
  grp_attrs<float, 3>();
  grp_attrs<float, 4>();
  grp_attrs<double, 2>();
  grp_attrs<double, 3>();
  grp_attrs<double, 4>();
  cudaGetLastError();
  done = true;
}
template <typename R, int G, bool BD> static int grp_occ() {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, cocg_spmm_grp_kernel<R, cocg_vec_grp<R>(), G, BD, false>,
                                                    kThreads, grp_smem_bytes<R, G, BD>()) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return b;
}
int grp_blocks_per_sm(int G, bool fp32, bool bd) {
  switch (G) {
    case 2: return fp32 ? grp_occ<float, 2, false>() : grp_occ<double, 2, false>();
    case 3:
      if (bd) return fp32 ? grp_occ<float, 3, true>() : grp_occ<double, 3, true>();
      return fp32 ? grp_occ<float, 3, false>() : grp_occ<double, 3, false>();
    case 4: return fp32 ? grp_occ<float, 4, false>() : grp_occ<double, 4, false>();
    default: return 0;
  }
}
template <typename R> void cocg_residual(const CocgArgs<R> &a, cudaStream_t st) {
  if (!args_guard(a, st)) return;
  with_vec(a, [&](auto vc) {
    constexpr int V = decltype(vc)::value;
    cocg_residual_kernel<R, V><<<grid_of(a), kThreads, 0, st>>>(a);
  });
}

template void cocg_init<double>(const CocgArgs<double> &, cudaStream_t);
template void cocg_init<float>(const CocgArgs<float> &, cudaStream_t);
template void cocg_update<double>(const CocgArgs<double> &, bool, int, cudaStream_t, int, int);
template void cocg_update<float>(const CocgArgs<float> &, bool, int, cudaStream_t, int, int);
template void cocg_dual<double>(const CocgArgs<double> &, int, int, int, int, bool, int, cudaStream_t);
template void cocg_dual<float>(const CocgArgs<float> &, int, int, int, int, bool, int, cudaStream_t);
template void cocg_spmm<double>(const CocgArgs<double> &, cudaStream_t, bool);
template void cocg_spmm<float>(const CocgArgs<float> &, cudaStream_t, bool);
template void cocg_residual<float>(const CocgArgs<float> &, cudaStream_t);

// ------------------------------------------------------------------------------ batched launchers
static int batch_grid(int total) {
  const int cap = device_sm_count() * 4;
  return total < cap ? total : cap;
}

template <typename R> void cocg_init_batched_launch(const CocgArgs<R> *args, const int *prefix, int P, int total,
                                                    cudaStream_t st) {
  cocg_init_batched<R><<<batch_grid(total), kThreads, 0, st>>>(args, prefix, P);
}
template <typename R> void cocg_update_batched_launch(const CocgArgs<R> *args, const int *prefix, int P, int total,
                                                      bool first, int fm, cudaStream_t st) {
  const int g = batch_grid(total);
#define UPD(F, M) cocg_update_batched<R, F, M><<<g, kThreads, 0, st>>>(args, prefix, P)
  if (first) {
    switch (fm) {
      case kFinalNone: UPD(true, kFinalNone); break;
      case kFinalU: UPD(true, kFinalU); break;
      case kFinalStoreD: UPD(true, kFinalStoreD); break;
      case kFinalAddD: UPD(true, kFinalAddD); break;
      case kAccU: UPD(true, kAccU); break;
      case kAccUEnd: UPD(true, kAccUEnd); break;
      default: UPD(true, kFinalUFromD); break;
    }
  } else {
    switch (fm) {
      case kFinalNone: UPD(false, kFinalNone); break;
      case kFinalU: UPD(false, kFinalU); break;
      case kFinalStoreD: UPD(false, kFinalStoreD); break;
      case kFinalAddD: UPD(false, kFinalAddD); break;
      case kAccU: UPD(false, kAccU); break;
      case kAccUEnd: UPD(false, kAccUEnd); break;
      default: UPD(false, kFinalUFromD); break;
    }
  }
#undef UPD
}
template <typename R> void cocg_spmm_batched_launch(const CocgArgs<R> *args, const int *prefix, int P, int total,
                                                    bool fresh, cudaStream_t st) {
  if (fresh) cocg_spmm_batched<R, true><<<batch_grid(total), kThreads, 0, st>>>(args, prefix, P);
  else cocg_spmm_batched<R, false><<<batch_grid(total), kThreads, 0, st>>>(args, prefix, P);
}
template <typename R> void cocg_residual_batched_launch(const CocgArgs<R> *args, const int *prefix, int P, int total,
                                                        cudaStream_t st) {
  cocg_residual_batched<R><<<batch_grid(total), kThreads, 0, st>>>(args, prefix, P);
}
#define INST(R)                                                                                            \
  template void cocg_init_batched_launch<R>(const CocgArgs<R> *, const int *, int, int, cudaStream_t);    \
  template void cocg_update_batched_launch<R>(const CocgArgs<R> *, const int *, int, int, bool, int,      \
                                              cudaStream_t);                                              \
  template void cocg_spmm_batched_launch<R>(const CocgArgs<R> *, const int *, int, int, bool, cudaStream_t);
INST(double)
INST(float)
#undef INST
template void cocg_residual_batched_launch<float>(const CocgArgs<float> *, const int *, int, int, cudaStream_t);

}  // namespace slrf
