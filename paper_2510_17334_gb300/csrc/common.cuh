// Device helpers shared by the SLRF kernels: complex arithmetic on double2/float2,
// warp reductions, the last-block reduction handshake and a bounded grid barrier.
#pragma once

#include <cuda_runtime.h>
#include <atomic>
#include <stdint.h>
#include <stdio.h>

namespace slrf {

// ---------------------------------------------------------------- real/complex traits
template <typename R> struct Cx;
template <> struct Cx<double> { using T = double2; };
template <> struct Cx<float> { using T = float2; };
template <typename R> using cx_t = typename Cx<R>::T;

template <typename C> __host__ __device__ inline C cmake(double re, double im) {
  C z; z.x = re; z.y = im; return z;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
// a * b (complex, unconjugated)
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  C z; z.x = a.x * b.x - a.y * b.y; z.y = a.x * b.y + a.y * b.x; return z;
}
// acc + a * b
template <typename C> __device__ __forceinline__ C cfma(C a, C b, C acc) {
  acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
  return acc;
}
// acc - a * b
template <typename C> __device__ __forceinline__ C cfms(C a, C b, C acc) {
  acc.x = fma(-a.x, b.x, fma(a.y, b.y, acc.x));
  acc.y = fma(-a.x, b.y, fma(-a.y, b.x, acc.y));
  return acc;
}
__host__ __device__ inline double2 cdiv(double2 a, double2 b) {
  // Smith's algorithm
  double2 z;
  if (fabs(b.x) >= fabs(b.y)) {
    double r = b.y / b.x, d = b.x + b.y * r;
    z.x = (a.x + a.y * r) / d; z.y = (a.y - a.x * r) / d;
  } else {
    double r = b.x / b.y, d = b.y + b.x * r;
    z.x = (a.x * r + a.y) / d; z.y = (a.y * r - a.x) / d;
  }
  return z;
}
__host__ __device__ inline bool cfinite(double2 a) { return isfinite(a.x) && isfinite(a.y); }

// Packed FP32 FMA (two lanes of fma.rn.f32x2, sm_100 and later): c + a * b elementwise,
// each half rounded exactly like fmaf.
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;"
      : "=l"(d)
      : "l"(*reinterpret_cast<unsigned long long *>(&a)), "l"(*reinterpret_cast<unsigned long long *>(&b)),
        "l"(*reinterpret_cast<unsigned long long *>(&c)));
  return *reinterpret_cast<float2 *>(&d);
}

// ---------------------------------------------------------------- debug bounds checks
// SLRF_CHECKS=1 (a debug build): every checked global access verifies its index against
// the extent the kernel was given; the first violation is printed with its site, the
// access is skipped.  Off by default (CHK is then the constant true).
#ifndef SLRF_CHECKS
#define SLRF_CHECKS 0
#endif
#if SLRF_CHECKS
__device__ __noinline__ inline bool slrf_chk_fail(int site, long long idx, long long bound) {
  printf("SLRF_CHECK site %d idx %lld bound %lld block (%d,%d) thread %d\n", site, idx, bound, (int)blockIdx.x,
         (int)blockIdx.y, (int)threadIdx.x);
  return false;
}
#define CHK(site, idx, bound)                                                    \
  ((((long long)(idx)) >= 0 && ((long long)(idx)) < ((long long)(bound))) || \
   slrf_chk_fail((site), (long long)(idx), (long long)(bound)))
#else
#define CHK(site, idx, bound) true
#endif

// ---------------------------------------------------------------- reductions
template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Last-block handshake: every block calls this after writing its partials; exactly one
// block (the last to arrive) gets true, and then sees all partials written before.
// The caller resets *counter to 0 when the last block is done.
__device__ __forceinline__ bool last_block_arrive(unsigned *counter, unsigned total) {
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) am_last = (atomicAdd(counter, 1u) == total - 1u);
  __syncthreads();
  if (am_last) __threadfence();
  return am_last;
}

// ---------------------------------------------------------------- bounded grid barrier
// For cooperative launches only (all blocks co-resident).  *count lives in global memory
// and starts at 0; it only grows: barrier number e (1, 2, ...) is complete once it holds
// e * nblocks, so an arrival is one fire-and-forget add after the block's stores are
// fenced, and a waiter polls one word (no reset, no second counter on the critical path).
// A block that waits longer than the spin limit sets *err = 1 and returns false; a block
// that sees *err set returns false too; callers leave the kernel when it returns false.
struct GridBarrier {
  unsigned *count;
  int *err;
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ inline bool grid_sync(const GridBarrier &gb, unsigned nblocks, unsigned &epoch) {
  __shared__ int ok;
  __syncthreads();
  ++epoch;
  if (threadIdx.x == 0) {
    ok = 1;
    __threadfence();
    atomicAdd(gb.count, 1u);
    const unsigned target = epoch * nblocks;
    long long spins = 0;
    while ((int)(ld_acquire_gpu(gb.count) - target) < 0) {
      if ((++spins & 63) == 0) {
        if (*(volatile int *)gb.err) { ok = 0; break; }
        if (spins > (1ll << 22)) { atomicExch(gb.err, 1); ok = 0; break; }  // a few seconds of polls
        __nanosleep(32);
      }
    }
  }
  __syncthreads();
  return ok != 0;
}


// ---------------------------------------------------------------- mbarrier and bulk copies
// Shared-memory address, global timer, mbarrier and 1-D bulk-copy (TMA engine) wrappers.
// Every wait is bounded: mbar_wait gives up after 2 s on the global timer and records a
// code in *err.
__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase of parity `parity` to complete; false (and *err = code) after 2 s.
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity, int *err, int code) {
  if (mbar_try(b, parity)) return true;
  const uint64_t t0 = gtimer();
  while (!mbar_try(b, parity)) {
    if (gtimer() - t0 > 2000000000ull) {
      atomicCAS(err, 0, code);
      return false;
    }
  }
  return true;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   su32(dst)),
               "l"(src), "r"(bytes), "r"(su32(bar))
               : "memory");
}

// ---------------------------------------------------------------- host: grid sizing
// Multiprocessors of the current device, queried once per device and cached (grids of the
// grid-stride kernels and the split counts of the tall-skinny products are sized from it).
inline int device_sm_count() {
  constexpr int kMaxDev = 64;
  static std::atomic<int> cache[kMaxDev];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) dev = 0;
  int v = dev < kMaxDev ? cache[dev].load(std::memory_order_relaxed) : 0;
  if (v > 0) return v;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
    cudaGetLastError();  // clear the failed query
    v = 1;
  }
  if (dev < kMaxDev) cache[dev].store(v, std::memory_order_relaxed);
  return v;
}

}  // namespace slrf
