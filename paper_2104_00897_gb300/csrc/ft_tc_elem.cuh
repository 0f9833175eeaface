// Element kinds of the tensor-core path (BF16, FP8 E4M3): storage, loads of eight
// consecutive K-contiguous elements, and the pieces in which B e enters the checksum
// operand. Shared by the encode pre-pass, the product kernel's epilogue and the resolve pass.
#pragma once

#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_fp8.h>

namespace ftk {
namespace {

__device__ __forceinline__ float bf16_to_f32(uint16_t b) { return __uint_as_float(static_cast<uint32_t>(b) << 16); }

__device__ __forceinline__ float e4m3_to_f32(uint8_t b) {
  return __half2float(__half(__nv_cvt_fp8_to_halfraw(static_cast<__nv_fp8_storage_t>(b), __NV_E4M3)));
}

// Input element kinds of the tensor-core path.
//   kBytes     storage bytes per element
//   kPieces    checksum columns holding the pieces of B e (rows 0 .. kPieces-1 of a block)
//   kPieceSum  bound of sum_p |piece_p| / |B e| (for the threshold's prediction part)
// BF16: B e as hi + mid + lo bfloat16 (exact for a binary32 value), scale 1.
// E4M3: B e as 8 e4m3 pieces with fixed scales 2^(9 - 4p): each piece is the nearest e4m3
//   of what the previous ones leave (subnormals flushed and carried). |B e| <= 248 * 448 fits
//   the first piece; each piece that is not flushed takes the top 4 bits of what is left, and
//   the scales step by 2^4, so the pieces hold the binary32 sum B e (at most 24 significant
//   bits, a multiple of 2^-9) exactly.
template <int KIND> struct Elem;
template <> struct Elem<0> {
  static constexpr int kBytes = 2, kPieces = 3;
  static constexpr float kPieceSum = 1.0078125f;
  // Eight consecutive elements of one K-contiguous line from k (a multiple of 8), zero
  // at and beyond K; one 16-byte load (aligned: ld is a multiple of 8 elements, bases
  // 16-byte aligned).
  using Raw = uint4;
  static __device__ __forceinline__ Raw zero() { return make_uint4(0u, 0u, 0u, 0u); }
  static __device__ __forceinline__ Raw load_raw(const void* line, int64_t k, int32_t K) {
    const uint16_t* l = static_cast<const uint16_t*>(line);
    if (k + 8 <= K) return *reinterpret_cast<const uint4*>(l + k);
    uint32_t t[4] = {0u, 0u, 0u, 0u};
    for (int q = 0; q < 8; ++q)
      if (k + q < K) t[q >> 1] |= (uint32_t)l[k + q] << (16 * (q & 1));
    return make_uint4(t[0], t[1], t[2], t[3]);
  }
  static __device__ __forceinline__ void load8(const void* line, int64_t k, int32_t K, float (&x)[8]) {
    unpack(load_raw(line, k, K), x);
  }
  static __device__ __forceinline__ void unpack(const Raw w, float (&x)[8]) {
    const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      x[2 * h] = __uint_as_float(ws[h] << 16);
      x[2 * h + 1] = __uint_as_float(ws[h] & 0xffff0000u);
    }
  }
  static __device__ __forceinline__ float at(const void* line, int64_t k) {
    return bf16_to_f32(static_cast<const uint16_t*>(line)[k]);
  }
};
template <> struct Elem<1> {
  static constexpr int kBytes = 1, kPieces = 8;
  static constexpr float kPieceSum = 1.25f;
  // as above with one 8-byte load (ld a multiple of 16 elements)
  using Raw = uint2;
  static __device__ __forceinline__ Raw zero() { return make_uint2(0u, 0u); }
  static __device__ __forceinline__ Raw load_raw(const void* line, int64_t k, int32_t K) {
    const uint8_t* l = static_cast<const uint8_t*>(line);
    if (k + 8 <= K) return *reinterpret_cast<const uint2*>(l + k);
    uint32_t t[2] = {0u, 0u};
    for (int q = 0; q < 8; ++q)
      if (k + q < K) t[q >> 2] |= (uint32_t)l[k + q] << (8 * (q & 3));
    return make_uint2(t[0], t[1]);
  }
  static __device__ __forceinline__ void load8(const void* line, int64_t k, int32_t K, float (&x)[8]) {
    unpack(load_raw(line, k, K), x);
  }
  // two codes per conversion instruction (the lower-addressed code in the low byte)
  static __device__ __forceinline__ void unpack(const Raw w, float (&x)[8]) {
    const uint32_t ws[2] = {w.x, w.y};
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const __half2_raw r =
            __nv_cvt_fp8x2_to_halfraw2(static_cast<__nv_fp8x2_storage_t>(ws[h] >> (16 * q)), __NV_E4M3);
        const float2 f = __half22float2(__half2(r));
        x[4 * h + 2 * q] = f.x;
        x[4 * h + 2 * q + 1] = f.y;
      }
  }
  static __device__ __forceinline__ float at(const void* line, int64_t k) {
    return e4m3_to_f32(static_cast<const uint8_t*>(line)[k]);
  }
};

}  // namespace
}  // namespace ftk
