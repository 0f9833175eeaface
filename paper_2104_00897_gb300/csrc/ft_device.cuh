// Device helpers: mbarrier and TMA (inline PTX for sm_103a), bounded waits, and the
// upward-rounded binary32 arithmetic used for the round-off thresholds.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace ftk {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Make initialised barriers visible to the async (TMA) proxy.
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for the barrier phase with a wall-clock limit. Returns false on timeout (the caller
// records FT_STATUS_TIMEOUT and abandons the tile). No trap, no unbounded spin.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  for (uint32_t it = 0;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 63u) == 63u && global_timer_ns() - t0 > limit_ns) return false;
  }
}

// 2-D tiled TMA load into shared memory, completing `bytes` on the barrier. x is the
// innermost (contiguous) coordinate, in elements.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int32_t x,
                                            int32_t y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], "
      "[%2];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_addr(bar)), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void tma_prefetch_desc(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// ---------------------------------------------------------------------------------------
// Upward-rounded binary32 arithmetic. Every operation rounds toward +infinity, so sums and
// products of non-negative values computed this way are upper bounds of the exact values.
// ---------------------------------------------------------------------------------------
// Upper bound of |x| as a binary32 value, built from the high word of x with integer
// operations only (no FP64-pipe instruction: on GB300 that pipe is the bottleneck, and a
// binary64 -> binary32 conversion issues to it). The high word holds the sign, the 11-bit
// exponent e and the top 20 significand bits; re-biasing e to 8 bits and adding one unit
// in the 20th significand bit bounds the dropped low bits from above. |x| < 2^-126 maps
// to 2^-126, |x| >= 2^128 to +inf (the caller's overflow path).
__device__ __forceinline__ double abs_int(double x) {
  return __hiloint2double(__double2hiint(x) & 0x7fffffff, __double2loint(x));
}
__device__ __forceinline__ float abs_up(double x) {
  const uint32_t hi = static_cast<uint32_t>(__double2hiint(x)) & 0x7fffffffu;
  const uint32_t e = hi >> 20;
  uint32_t b = ((hi - (896u << 20)) << 3) + 8u;
  b = (e < 897u) ? 0x00800000u : b;
  b = (e > 1150u) ? 0x7f800000u : b;
  return __uint_as_float(b);
}
__device__ __forceinline__ float add_up(float a, float b) { return __fadd_ru(a, b); }
__device__ __forceinline__ float fma_up(float a, float b, float c) { return __fmaf_ru(a, b, c); }
__device__ __forceinline__ float mul_up(float a, float b) { return __fmul_ru(a, b); }

// gamma_n = n u / (1 - n u), u = 2^-53, rounded up in binary32.
__device__ __forceinline__ float gamma_up(int64_t n) {
  const float nf = __ll2float_ru(n);
  const float nu = __fmul_ru(nf, 0x1p-53f);  // 2^-53 is exact in binary32
  const float den = __fsub_rd(1.0f, nu);
  return __fdiv_ru(nu, den);
}

__device__ __forceinline__ double flip_bit_f64(double x, int bit) {
  return __longlong_as_double(__double_as_longlong(x) ^ (1ll << bit));
}

}  // namespace ftk
