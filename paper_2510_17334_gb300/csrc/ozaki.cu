// Ozaki-split FP64 products on tcgen05 (see ozaki.cuh for the arithmetic).
//
// Digit layout.  An operand with R rows (padded to 32) and K products (padded to 32) is
// stored per slice s as k-blocks of 32 products; a k-block holds two k-steps of 16, and a
// k-step holds R/8 groups of 8 rows, each group two 8 x 8 core matrices (K-major, 16 B per
// row).  A 128-row tile of one (slice, k-step) is thus 4 KB contiguous and a 32-row tile
// 1 KB: the MMA kernel fetches them with plain bulk copies and reads them through
// no-swizzle shared-memory descriptors (core matrix stride 128 B along K, 256 B along rows).
//
// MMA kernel.  A work unit is a 128 x 32 output tile over a range of k-blocks; CTAs are
// persistent (one per SM) and walk the units b, b + gridDim.x, ...:
//   warp 4 lane 0   bulk-copies 7 A and 7 B slices per k-block into a 3-stage ring;
//   warp 5          allocates TMEM; lane 0 issues 2 x 28 MMAs (M128 N32 K16) per k-block
//                   into six accumulators (levels 0..4 and the merged 5..6) of one of two
//                   TMEM buffers, which alternate between 128-product chunks;
//   warps 0-3       drain a finished buffer (tcgen05.ld, one TMEM lane quarter each) into
//                   64-bit integer sums of the exact levels and an FP32 sum of the merged
//                   level, while the next chunk runs on the other buffer.
// Every wait is bounded by a 2 s deadline on the global timer; on expiry the CTA records a
// code in *err, finishes its outstanding copies and MMAs, frees TMEM and returns.
#include "ozaki.cuh"

#include <algorithm>

namespace slrf {
namespace {

constexpr int kS = 7;          // digit slices
constexpr int kAcc = 6;        // accumulators per TMEM buffer
constexpr int kTM = 128, kTN = 32;
constexpr int kChunkKB = 4;    // k-blocks (of 32) per exact chunk: 128 products
constexpr int kStages = 3;
constexpr int kATile = 4096;   // 128 rows x 16 products x 2 B
constexpr int kBTile = 1024;   // 32 rows x 16 products x 2 B
constexpr int kStageA = kS * 2 * kATile;
constexpr int kStageB = kS * 2 * kBTile;
constexpr int kStage = kStageA + kStageB;
constexpr int kBarOff = kStages * kStage;
constexpr int kMmaSmem = kBarOff + 128;
constexpr uint32_t kTmemCols = 512;  // 2 buffers x 6 accumulators x 32 columns = 384 used
constexpr int kESent = (int)0x80808080;  // exponent of an all-zero row
constexpr int kENonFinite = 4096;        // exponent marking a row with Inf/NaN
constexpr int kMaxChunksPerCta = 64;     // keeps the 64-bit sums below 2^62
constexpr size_t kDigitSlack = 8192;     // a last 128-row tile may read past the array end

__host__ __device__ inline size_t off16(int s, int KB, int kb, int j, int R8, int g8, int h, int row) {
  return ((((size_t)(s * KB + kb) * 2 + j) * R8 + g8) * 2 + h) * 8 + row;
}

__host__ __device__ inline int64_t pad32(int64_t x) { return (x + 31) / 32 * 32; }

size_t digit_bytes(int64_t rows, int64_t K) { return (size_t)kS * pad32(rows) * pad32(K) * 2 + kDigitSlack; }

// ------------------------------------------------------------------------- PTX wrappers
// (shared-memory address, global timer, mbarrier and bulk-copy wrappers: common.cuh)
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t cols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(slot)), "r"(cols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t cols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols) : "memory");
}
// D (TMEM, FP32) (+)= A (smem, bf16, K-major) B (smem, bf16, K-major)^T
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}
// 32 consecutive FP32 columns of this thread's TMEM lane; waits for the load.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r[q]);
}

// Shared-memory descriptor, no swizzle, K-major: core matrices 128 B apart along K (LBO)
// and 256 B apart along rows (SBO); descriptor version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(256 >> 4) << 32) |
         (1ull << 46);
}
// Instruction descriptor of kind::f16: FP32 accumulator, bf16 A and B, both K-major.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTN >> 3) << 17) |
                            ((uint32_t)(kTM >> 4) << 24);

// ------------------------------------------------------------------------- splitting
__device__ __forceinline__ int exp_of(double x) {  // E with |x| < 2^E (0 / subnormal: sentinel)
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  if (ex == 0x7FF) return kENonFinite;
  return ex == 0 ? kESent : ex - 1022;
}

// Digits of 8 values sharing the exponent E, packed per slice as 8 bf16 (element q in
// halfword q).
__device__ __forceinline__ void digits8(const double (&x)[8], int E, uint4 (&out)[kS]) {
  uint32_t w[kS][4];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x[q]);
    const int ex = (int)((b >> 52) & 0x7FF);
    long long v = 0;
    if (ex != 0 && ex != 0x7FF && E != kESent && E != kENonFinite) {
      const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
      const int sh = (ex - 1023) - E + 4;  // |x| 2^(56-E) = m 2^sh, sh <= 3
      if (sh >= 0) v = (long long)(m << sh);
      else if (sh > -60) v = (long long)((m + (1ull << (-sh - 1))) >> (-sh));
    }
    int d[kS];
#pragma unroll
    for (int s = kS - 1; s >= 1; --s) {
      int t = (int)(v & 255);
      v >>= 8;
      if (t >= 128) { t -= 256; v += 1; }
      d[s] = t;
    }
    d[0] = (int)v;
    const bool neg = (b >> 63) != 0;
#pragma unroll
    for (int s = 0; s < kS; ++s) {
      const float f = (float)(neg ? -d[s] : d[s]) * __int_as_float((127 - 8 * s) << 23);  // d 2^(-8s)
      const uint32_t h = __float_as_uint(f) >> 16;  // exact: |d| has at most 8 significant bits
      if (q & 1) w[s][q >> 1] |= h << 16;
      else w[s][q >> 1] = h;
    }
  }
#pragma unroll
  for (int s = 0; s < kS; ++s) out[s] = make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
}

// E[c] = max over rows of the exponent of X[r][c] (E pre-set to kESent bytes 0x80).  Block
// 32 columns x 8 row lanes; a shared-memory max per block, then one atomicMax per column
// (integer max: the result does not depend on the order).
__global__ void __launch_bounds__(256) oz_colexp_kernel(int64_t n, const double *__restrict__ X, int ldx, int k,
                                                        int *E, const int *run_if) {
  if (run_if != nullptr && *run_if == 0) return;
  __shared__ int red[8][33];
  const int c = blockIdx.x * 32 + threadIdx.x;
  int m = kESent;
  if (c < k)
    for (int64_t r = (int64_t)blockIdx.y * 8 + threadIdx.y; r < n; r += (int64_t)gridDim.y * 8)
      m = max(m, exp_of(X[r * ldx + c]));
  red[threadIdx.y][threadIdx.x] = m;
  __syncthreads();
  if (threadIdx.y == 0 && c < k) {
#pragma unroll
    for (int y = 1; y < 8; ++y) m = max(m, red[y][threadIdx.x]);
    if (m != kESent) atomicMax(E + c, m);
  }
}

void colexp(int64_t n, const double *X, int ldx, int k, int *E, const int *run_if, cudaStream_t st) {
  const int gy = (int)std::min<int64_t>(std::max<int64_t>((n + 255) / 256, 1), 1024);
  oz_colexp_kernel<<<dim3((k + 31) / 32, gy), dim3(32, 8), 0, st>>>(n, X, ldx, k, E, run_if);
}

// Column operand: operand row i = column i of X, products over the rows of X.  One thread
// per (i, group of 8 products).
__global__ void __launch_bounds__(256) oz_split_cols_kernel(int64_t n, const double *__restrict__ X, int ldx, int k,
                                                            int Rp, int KB, uint4 *__restrict__ dig,
                                                            const int *__restrict__ E, const int *run_if) {
  if (run_if != nullptr && *run_if == 0) return;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int i = (int)(t % Rp);
  const int64_t g = t / Rp;
  if (g >= (int64_t)KB * 4) return;
  const int e = i < k ? E[i] : kESent;
  double x[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int64_t r = g * 8 + q;
    x[q] = (i < k && r < n) ? X[r * ldx + i] : 0.0;
  }
  uint4 d[kS];
  digits8(x, e, d);
  const int gi = (int)g;
#pragma unroll
  for (int s = 0; s < kS; ++s) dig[off16(s, KB, gi >> 2, (gi >> 1) & 1, Rp / 8, i >> 3, gi & 1, i & 7)] = d[s];
}

// Row operand: operand row r = row r of X (k1 <= 512 products).  One block per 8 rows:
// a warp per row finds the exponent and the digits, staged in shared memory so that the
// block writes whole 128 B core matrices.
__global__ void __launch_bounds__(256) oz_split_rows_kernel(int64_t n, const double *__restrict__ X, int ldx,
                                                            int k1, int KB, int R8, uint4 *__restrict__ dig,
                                                            int *__restrict__ E) {
  extern __shared__ uint4 stg[];  // [kS][G][8]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int G = KB * 4;
  const int64_t r = (int64_t)blockIdx.x * 8 + warp;
  int e = kESent;
  if (r < n)
    for (int c = lane; c < k1; c += 32) e = max(e, exp_of(X[r * ldx + c]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
  if (lane == 0 && r < n) E[r] = e;
  for (int g = lane; g < G; g += 32) {
    double x[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int c = g * 8 + q;
      x[q] = (r < n && c < k1) ? X[r * ldx + c] : 0.0;
    }
    uint4 d[kS];
    digits8(x, e, d);
#pragma unroll
    for (int s = 0; s < kS; ++s) stg[(s * G + g) * 8 + warp] = d[s];
  }
  __syncthreads();
  const int total = kS * G * 8;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int row = t & 7, sg = t >> 3, g = sg % G, s = sg / G;
    dig[off16(s, KB, g >> 2, (g >> 1) & 1, R8, blockIdx.x, g & 1, row)] = stg[t];
  }
}

// ------------------------------------------------------------------------- MMA kernel
struct OzMma {
  const uint16_t *dA, *dB;
  int RA8, RB8, KB;  // rows/8 of the two layouts, k-blocks of both
  int kb_per_split;
  int m_tiles, n_tiles;
  int sym;
  int tiles, units;  // output tiles; work units = tiles x row splits
  int mode;          // 0: FP64 partial tiles to part; 1: Z = alpha 2^(EA+EB-16) D + beta Z
  double *part;
  int MR, NC;        // partial tile array: [split][MR][NC]
  const int *EA, *EB;
  double *Z;
  int ldz;
  int64_t rows;
  int cols;
  double alpha, beta;
  int *err;
  const int *run_if;
};

__device__ __forceinline__ void tile_of(const OzMma &p, int idx, int &t, int &u) {
  if (!p.sym) { t = idx / p.n_tiles; u = idx % p.n_tiles; return; }
  for (t = 0; t < p.m_tiles; ++t) {
    const int u0 = (kTM * t) / kTN;  // first 32-column tile touching the upper triangle
    const int cnt = p.n_tiles - u0;
    if (idx < cnt) { u = u0 + idx; return; }
    idx -= cnt;
  }
  t = 0; u = 0;
}

// Work unit q: tile (q mod tiles) over the k-blocks of row split (q / tiles).  Consecutive
// units share their row split (Gram) or their 128-row tile of A (product), so the CTAs in
// flight re-read the same digit tiles from L2.
__device__ __forceinline__ void unit_of(const OzMma &p, int q, int &t, int &u, int &split, int &kb0, int &nkb) {
  split = q / p.tiles;
  tile_of(p, q % p.tiles, t, u);
  kb0 = split * p.kb_per_split;
  nkb = min(p.KB, kb0 + p.kb_per_split) - kb0;  // >= 1 by construction
}

// Persistent: CTA b takes the units b, b + gridDim.x, ...; the three roles walk the same
// sequence, so the copy ring, the MMA stream and the TMEM double buffer run on across
// unit boundaries (k-block counter g, chunk counter c).
__global__ void __launch_bounds__(192, 1) oz_mma_kernel(const OzMma p) {
  if (p.run_if != nullptr && *p.run_if == 0) return;
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kBarOff);
  uint64_t *full = bars, *empty = bars + 3, *tfull = bars + 6, *tempty = bars + 8, *done = bars + 10;
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 11);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < kStages; ++i) { mbar_init(full + i, 1); mbar_init(empty + i, 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(tfull + b, 1); mbar_init(tempty + b, 128); }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 5) tmem_alloc(tslot, kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 4) {
    if (lane == 0) {
      int g = 0;
      bool ok = true;
      for (int q = blockIdx.x; q < p.units && ok; q += gridDim.x) {
        int t, u, split, kb0, nkb;
        unit_of(p, q, t, u, split, kb0, nkb);
        for (int i = 0; i < nkb; ++i, ++g) {
          const int s_ = g % kStages;
          if (g >= kStages && !mbar_wait(empty + s_, ((g / kStages) - 1) & 1, p.err, 1)) { ok = false; break; }
          unsigned char *sa = smem + s_ * kStage, *sb = sa + kStageA;
          mbar_expect_tx(full + s_, kStage);
          const int kb = kb0 + i;
#pragma unroll 1
          for (int sl = 0; sl < kS; ++sl)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
              bulk_g2s(sa + (sl * 2 + j) * kATile, p.dA + off16(sl, p.KB, kb, j, p.RA8, 16 * t, 0, 0) * 8, kATile,
                       full + s_);
              bulk_g2s(sb + (sl * 2 + j) * kBTile, p.dB + off16(sl, p.KB, kb, j, p.RB8, 4 * u, 0, 0) * 8, kBTile,
                       full + s_);
            }
        }
      }
      // every armed stage has landed before the CTA may exit (a no-op in normal runs)
      for (int i = max(0, g - kStages); i < g; ++i) mbar_wait(full + i % kStages, (i / kStages) & 1, p.err, 6);
    }
  } else if (warp == 5) {
    if (lane == 0) {
      const uint32_t sbase = su32(smem);
      int g = 0, c = 0, buf = 0;
      bool ok = true;
      for (int q = blockIdx.x; q < p.units && ok; q += gridDim.x) {
        int t, u, split, kb0, nkb;
        unit_of(p, q, t, u, split, kb0, nkb);
        for (int i = 0; i < nkb; ++i, ++g) {
          const bool first = (i % kChunkKB) == 0;
          if (first) {
            buf = c & 1;
            if (c >= 2 && !mbar_wait(tempty + buf, ((c >> 1) - 1) & 1, p.err, 2)) { ok = false; break; }
          }
          const int s_ = g % kStages;
          if (!mbar_wait(full + s_, (g / kStages) & 1, p.err, 3)) { ok = false; break; }
          tc_fence_after();
          const uint32_t a0 = sbase + s_ * kStage, b0 = a0 + kStageA;
          const uint32_t dbuf = tmem + (uint32_t)(buf * kAcc * kTN);
#pragma unroll
          for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int sl = 0; sl < kS; ++sl)
#pragma unroll
              for (int tl = 0; tl + sl < kS; ++tl) {
                const int lvl = sl + tl < 5 ? sl + tl : 5;
                const uint32_t acc = (first && j == 0 && sl == 0 && tl <= 5) ? 0u : 1u;
                mma_bf16(dbuf + (uint32_t)(lvl * kTN), sdesc(a0 + (sl * 2 + j) * kATile),
                         sdesc(b0 + (tl * 2 + j) * kBTile), kIdesc, acc);
              }
          mma_commit(empty + s_);
          if ((i % kChunkKB) == kChunkKB - 1 || i == nkb - 1) {
            mma_commit(tfull + buf);
            ++c;
          }
        }
      }
      mma_commit(done);
      mbar_wait(done, 0, p.err, 4);
    }
    __syncwarp();
  } else {
    // epilogue: warp w owns TMEM lanes 32w..32w+31 = output rows 128t + 32w + lane
    int c = 0;
    bool ok = true;
    for (int q = blockIdx.x; q < p.units && ok; q += gridDim.x) {
      int t, u, split, kb0, nkb;
      unit_of(p, q, t, u, split, kb0, nkb);
      long long I[32];
      float f5[32];
#pragma unroll
      for (int qq = 0; qq < 32; ++qq) { I[qq] = 0; f5[qq] = 0.f; }
      const int nch = (nkb + kChunkKB - 1) / kChunkKB;
      for (int k = 0; k < nch; ++k, ++c) {
        const int buf = c & 1;
        if (!mbar_wait(tfull + buf, (c >> 1) & 1, p.err, 5)) { ok = false; break; }
        tc_fence_after();
        const uint32_t tb = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(buf * kAcc * kTN);
        float v[32];
#pragma unroll
        for (int lvl = 0; lvl < 5; ++lvl) {
          tmem_ld32(tb + (uint32_t)(lvl * kTN), v);
          const float sc = __int_as_float((127 + 8 * lvl) << 23);  // 2^(8 lvl)
#pragma unroll
          for (int qq = 0; qq < 32; ++qq)
            I[qq] += (long long)__float2int_rn(v[qq] * sc) * (1ll << (8 * (4 - lvl)));
        }
        tmem_ld32(tb + (uint32_t)(5 * kTN), v);
#pragma unroll
        for (int qq = 0; qq < 32; ++qq) f5[qq] += v[qq];
        tc_fence_before();
        mbar_arrive(tempty + buf);
      }
      if (!ok) break;
      // Sum of the levels in FP64 (the merged levels keep their FP32 sum's bits: rounding
      // them into the 64-bit units would cost 2^-49 of a single product); powers of two are
      // applied to the exponent bits.  GB300 runs FP64 at 2 operations per clock per SM, so
      // the finish of 128 x 32 outputs per unit is kept to three FP64 operations each.
      const int64_t row = (int64_t)kTM * t + 32 * warp + lane;
      if (p.mode == 0) {
        double *dst = p.part + ((int64_t)split * p.MR + row) * p.NC + kTN * u;
#pragma unroll
        for (int qq = 0; qq < 32; ++qq) dst[qq] = fma((double)I[qq], 0x1p-32, (double)f5[qq]);
      } else if (row < p.rows) {
        const int ea = max(p.EA[row], -1100);
        // uniform flags, decided once (FP64 compares run on the FP64 pipe)
        const int amode = p.alpha == 1.0 ? 0 : (p.alpha == -1.0 ? 1 : 2);
        const int bmode = p.beta == 0.0 ? 0 : (p.beta == 1.0 ? 1 : 2);
#pragma unroll
        for (int qq = 0; qq < 32; ++qq) {
          const int col = kTN * u + qq;
          if (col >= p.cols) continue;
          const int eb = max(p.EB[col], -1100);
          double z = fma((double)f5[qq], 4294967296.0, (double)I[qq]);  // in units of 2^-32
          const int e = ea + eb - 48;  // value = z 2^(EA + EB - 16 - 32)
          long long zb = __double_as_longlong(z);
          if (ea == kENonFinite || eb == kENonFinite) {
            zb = 0x7ff8000000000000ll;
          } else if ((zb & 0x7FFFFFFFFFFFFFFFll) != 0) {
            const int ez = (int)((zb >> 52) & 0x7FF);  // biased exponent of z (>= 1023)
            if (ez + e >= 1 && ez + e <= 2046) zb += (long long)e << 52;
            else zb = __double_as_longlong(scalbn(z, e));
          }
          if (amode == 1) zb ^= (long long)0x8000000000000000ull;  // alpha = -1: flip the sign bit
          z = __longlong_as_double(zb);
          if (amode == 2) z *= p.alpha;
          double *zp = p.Z + row * p.ldz + col;
          if (bmode == 1) z += *zp;
          else if (bmode == 2) z = fma(p.beta, *zp, z);
          *zp = z;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 5) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

// C = 2^(EA+EB-16) sum_split part; sym mirrors the lower triangle.
__global__ void oz_gram_finalize_kernel(int k1, int k2, int nsplit, int MR, int NC, const double *__restrict__ part,
                                        const int *__restrict__ EA, const int *__restrict__ EB, int sym, double *C,
                                        int ldc, const int *run_if) {
  if (run_if != nullptr && *run_if == 0) return;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)k1 * k2) return;
  const int i = (int)(t / k2), j = (int)(t % k2);
  int si = i, sj = j;
  if (sym && i > j) { si = j; sj = i; }
  double s = 0.0;
  for (int z = 0; z < nsplit; ++z) s += part[((int64_t)z * MR + si) * NC + sj];
  const int ea = max(EA[si], -1100), eb = max(EB[sj], -1100);
  C[(size_t)i * ldc + j] = (ea == kENonFinite || eb == kENonFinite) ? __longlong_as_double(0x7ff8000000000000ll)
                                                                     : scalbn(s, ea + eb - 16);
}

int num_sms() { return device_sm_count(); }

void set_smem_attrs() {
  static bool done = false;
  if (done) return;
  cudaFuncSetAttribute(oz_mma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kMmaSmem);
  cudaFuncSetAttribute(oz_split_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kS * 64 * 8 * 16);
  done = true;
}

struct GramPlan {
  int m_tiles, n_tiles, tiles, KB, kb_per_split, nsplit, MR, NC;
};

GramPlan gram_plan(int64_t n, int k1, int k2, bool sym) {
  GramPlan g;
  g.m_tiles = (k1 + kTM - 1) / kTM;
  g.n_tiles = (k2 + kTN - 1) / kTN;
  if (sym) {
    g.tiles = 0;
    for (int t = 0; t < g.m_tiles; ++t) g.tiles += g.n_tiles - (kTM * t) / kTN;
  } else {
    g.tiles = g.m_tiles * g.n_tiles;
  }
  g.KB = (int)(pad32(n) / 32);
  const int chunks = std::max(1, (g.KB + kChunkKB - 1) / kChunkKB);
  int ns = std::max(1, num_sms() / g.tiles);
  ns = std::max(ns, (chunks + kMaxChunksPerCta - 1) / kMaxChunksPerCta);
  ns = std::min(ns, chunks);
  g.kb_per_split = ((chunks + ns - 1) / ns) * kChunkKB;
  g.nsplit = (g.KB + g.kb_per_split - 1) / g.kb_per_split;
  g.MR = g.m_tiles * kTM;
  g.NC = g.n_tiles * kTN;
  return g;
}

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

// Workspace layout of oz_gram: exponents, digits of X (and of Y unless Y is X), partial tiles.
struct GramLayout {
  size_t eb_off, da_off, db_off, part_off, bytes;
};
GramLayout gram_layout(int64_t n, int k1, int k2, bool same, const GramPlan &g) {
  GramLayout l;
  l.eb_off = (size_t)pad32(k1);  // in ints
  l.da_off = up256((size_t)(pad32(k1) + pad32(k2)) * sizeof(int));
  l.db_off = l.da_off + up256(digit_bytes(k1, n));
  l.part_off = same ? l.db_off : l.db_off + up256(digit_bytes(k2, n));
  l.bytes = l.part_off + (size_t)g.nsplit * g.MR * g.NC * sizeof(double);
  return l;
}
// Workspace layout of oz_gemm: row exponents of X, column exponents of S, digits of both.
struct GemmLayout {
  size_t eb_off, da_off, db_off, bytes;
};
GemmLayout gemm_layout(int64_t n, int k1, int k2) {
  GemmLayout l;
  l.eb_off = (size_t)pad32(n);
  l.da_off = up256((size_t)(pad32(n) + pad32(k2)) * sizeof(int));
  l.db_off = l.da_off + up256(digit_bytes(n, k1));
  l.bytes = l.db_off + up256(digit_bytes(k2, k1));
  return l;
}

}  // namespace

size_t oz_work_bytes(int64_t n, int k1, int k2) {
  // any k1' <= k1, k2' <= k2, symmetric or not: at most max(SMs, chunks / 64) splits of
  // partial tiles no larger than the k1 x k2 tile grid
  const int kmax = std::max(k1, k2);
  const int64_t chunks = std::max<int64_t>(1, (pad32(n) / 32 + kChunkKB - 1) / kChunkKB);
  const size_t splits = (size_t)std::max<int64_t>(num_sms(), (chunks + kMaxChunksPerCta - 1) / kMaxChunksPerCta);
  const size_t part = splits * (size_t)((kmax + kTM - 1) / kTM * kTM) * (size_t)pad32(kmax) * sizeof(double);
  const size_t gram = up256((size_t)2 * pad32(kmax) * sizeof(int)) + 2 * up256(digit_bytes(kmax, n)) + part;
  return std::max(gram, gemm_layout(n, kmax, kmax).bytes) + 256;
}

void oz_gram(int64_t n, const double *X, int ldx, int k1, const double *Y, int ldy, int k2, double *C, int ldc,
             bool sym, void *work, size_t work_bytes, int *err, cudaStream_t st, const int *run_if) {
  if (k1 <= 0 || k2 <= 0) return;
  if (n <= 0) {  // an empty product is zero
    for (int i = 0; i < k1; ++i) cudaMemsetAsync(C + (size_t)i * ldc, 0, sizeof(double) * k2, st);
    return;
  }
  set_smem_attrs();
  const bool same = X == Y && ldx == ldy && k1 == k2;  // one digit array serves both operands
  const GramPlan g = gram_plan(n, k1, k2, sym);
  const GramLayout lay = gram_layout(n, k1, k2, same, g);
  if (lay.bytes > work_bytes) {  // never in a correctly sized context: refuse instead of overrunning
    cudaMemsetAsync(err, 0x7f, sizeof(int), st);
    return;
  }
  unsigned char *w = static_cast<unsigned char *>(work);
  int *EA = reinterpret_cast<int *>(w);
  int *EB = same ? EA : EA + lay.eb_off;
  uint4 *dA = reinterpret_cast<uint4 *>(w + lay.da_off);
  uint4 *dB = same ? dA : reinterpret_cast<uint4 *>(w + lay.db_off);
  double *part = reinterpret_cast<double *>(w + lay.part_off);
  const int RA = (int)pad32(k1), RB = (int)pad32(k2);
  // exponents
  cudaMemsetAsync(EA, 0x80, sizeof(int) * RA, st);
  colexp(n, X, ldx, k1, EA, run_if, st);
  if (!same) {
    cudaMemsetAsync(EB, 0x80, sizeof(int) * RB, st);
    colexp(n, Y, ldy, k2, EB, run_if, st);
  }
  // digits (the tail past the last k-block row groups stays as it is: only padded rows read it)
  {
    const int64_t tot = (int64_t)RA * g.KB * 4;
    oz_split_cols_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, X, ldx, k1, RA, g.KB, dA, EA, run_if);
  }
  if (!same) {
    const int64_t tot = (int64_t)RB * g.KB * 4;
    oz_split_cols_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, Y, ldy, k2, RB, g.KB, dB, EB, run_if);
  }
  OzMma p{};
  p.dA = reinterpret_cast<const uint16_t *>(dA);
  p.dB = reinterpret_cast<const uint16_t *>(dB);
  p.RA8 = RA / 8; p.RB8 = RB / 8; p.KB = g.KB;
  p.kb_per_split = g.kb_per_split;
  p.m_tiles = g.m_tiles; p.n_tiles = g.n_tiles;
  p.sym = sym ? 1 : 0;
  p.mode = 0;
  p.part = part; p.MR = g.MR; p.NC = g.NC;
  p.err = err;
  p.run_if = run_if;
  p.tiles = g.tiles;
  p.units = g.tiles * g.nsplit;
  oz_mma_kernel<<<std::min(p.units, num_sms()), 192, kMmaSmem, st>>>(p);
  const int64_t tot = (int64_t)k1 * k2;
  oz_gram_finalize_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(k1, k2, g.nsplit, g.MR, g.NC, part, EA, EB,
                                                                        sym ? 1 : 0, C, ldc, run_if);
}

void oz_gemm(int64_t n, const double *X, int ldx, int k1, const double *S, int lds, int k2, double *Z, int ldz,
             double alpha, double beta, void *work, size_t work_bytes, int *err, cudaStream_t st) {
  if (n <= 0 || k2 <= 0) return;
  set_smem_attrs();
  const GemmLayout lay = gemm_layout(n, k1, k2);
  if (lay.bytes > work_bytes || k1 > 512) {
    cudaMemsetAsync(err, 0x7f, sizeof(int), st);
    return;
  }
  unsigned char *w = static_cast<unsigned char *>(work);
  const int64_t RA = pad32(n);
  const int RB = (int)pad32(k2);
  const int KB = (int)(pad32(k1) / 32);
  int *EA = reinterpret_cast<int *>(w);
  int *EB = EA + lay.eb_off;
  uint4 *dA = reinterpret_cast<uint4 *>(w + lay.da_off);
  uint4 *dB = reinterpret_cast<uint4 *>(w + lay.db_off);
  // A: rows of X; B: columns of S (products over the k1 rows of S)
  oz_split_rows_kernel<<<(unsigned)(RA / 8), 256, (size_t)kS * KB * 4 * 8 * sizeof(uint4), st>>>(
      n, X, ldx, k1, KB, (int)(RA / 8), dA, EA);
  cudaMemsetAsync(EB, 0x80, sizeof(int) * RB, st);
  colexp(k1, S, lds, k2, EB, nullptr, st);
  {
    const int64_t tot = (int64_t)RB * KB * 4;
    oz_split_cols_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(k1, S, lds, k2, RB, KB, dB, EB, nullptr);
  }
  OzMma p{};
  p.dA = reinterpret_cast<const uint16_t *>(dA);
  p.dB = reinterpret_cast<const uint16_t *>(dB);
  p.RA8 = (int)(RA / 8); p.RB8 = RB / 8; p.KB = KB;
  p.kb_per_split = KB;
  p.m_tiles = (int)((n + kTM - 1) / kTM);
  p.n_tiles = (k2 + kTN - 1) / kTN;
  p.sym = 0;
  p.mode = 1;
  p.EA = EA; p.EB = EB;
  p.Z = Z; p.ldz = ldz; p.rows = n; p.cols = k2;
  p.alpha = alpha; p.beta = beta;
  p.err = err;
  p.tiles = p.m_tiles * p.n_tiles;
  p.units = p.tiles;
  oz_mma_kernel<<<std::min(p.units, num_sms()), 192, kMmaSmem, st>>>(p);
}

}  // namespace slrf
