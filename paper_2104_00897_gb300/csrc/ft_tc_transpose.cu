// K-major copies of MN-major operands for the tensor-core path, and the format conversions of
// bfloat16 outputs. The tcgen05 product kernel and the checksum encode read every operand
// K-contiguous (rows of K elements, 128-byte swizzled TMA boxes); an operand stored the other
// way (op(A) with its rows contiguous, or op(B) with its columns contiguous) is transposed
// once into library workspace: each thread loads a block of 8 x 8 16-bit or 16 x 16 8-bit
// elements with 16-byte loads, transposes it in registers by byte permutes and stores it
// with 16-byte stores.
#include <cstdint>
#include <type_traits>

#include <cuda_bf16.h>

#include "ft_tc.h"

namespace ftk {

namespace {

// In-register transpose of an n x n block of EB-byte elements, n = 16 / EB (8 x 8 of 16-bit,
// 16 x 16 of 8-bit), held as n rows of four 32-bit words: elements of neighbouring rows are
// interleaved by byte permutes, then ever larger groups of words are exchanged between rows
// s apart (s = 2, 4, 8): the recursive block transpose. Row i ends holding column i.
template <int EB>
__device__ __forceinline__ void transpose_block(uint32_t (&w)[16 / EB][4]) {
  constexpr int n = 16 / EB;
  if (EB == 2) {
#pragma unroll
    for (int p = 0; p < n / 2; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint32_t a = w[2 * p][q], b = w[2 * p + 1][q];
        w[2 * p][q] = __byte_perm(a, b, 0x5410);
        w[2 * p + 1][q] = __byte_perm(a, b, 0x7632);
      }
  } else {
#pragma unroll
    for (int p = 0; p < n / 2; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint32_t a = w[2 * p][q], b = w[2 * p + 1][q];
        w[2 * p][q] = __byte_perm(a, b, 0x6240);
        w[2 * p + 1][q] = __byte_perm(a, b, 0x7351);
      }
#pragma unroll
    for (int base = 0; base < n; base += 4)
#pragma unroll
      for (int r = base; r < base + 2; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint32_t a = w[r][q], b = w[r + 2][q];
          w[r][q] = __byte_perm(a, b, 0x5410);
          w[r + 2][q] = __byte_perm(a, b, 0x7632);
        }
  }
  // word groups of g between rows s apart
#pragma unroll
  for (int s = (EB == 2 ? 2 : 4), g = 1; s < n; s *= 2, g *= 2)
#pragma unroll
    for (int base = 0; base < n; base += 2 * s)
#pragma unroll
      for (int r = base; r < base + s; ++r)
#pragma unroll
        for (int w0 = 0; w0 < 4; w0 += 2 * g)
#pragma unroll
          for (int q = 0; q < g; ++q) {
            const uint32_t t = w[r][w0 + g + q];
            w[r][w0 + g + q] = w[r + s][w0 + q];
            w[r + s][w0 + q] = t;
          }
}

// dst[r * pitch + k] = src[r + k * ld] for r < R, k < K; EB bytes per element (1 or 2).
// Each thread moves one n x n block (n = 16 / EB): n 16-byte loads along r (rows k of the
// source), a transpose in registers, n 16-byte stores along k. Lane l of a warp takes block
// row (l & 7) of 8 and block column (l >> 3) of 4: a source row is read in 128-byte runs, a
// destination row written in 64-byte runs; the CTA's 8 warps take consecutive groups of 4
// block columns. Blocks at the edges, or without 16-byte alignment, move element by element.
constexpr int kKmWarps = 8;
template <int EB>
__global__ void __launch_bounds__(kKmWarps * 32) kmajor_copy_kernel(const uint8_t* __restrict__ src, int64_t R,
                                                                   int64_t K, int64_t ld, uint8_t* __restrict__ dst,
                                                                   int64_t pitch, int vec) {
  constexpr int n = 16 / EB;
  using T = typename std::conditional<EB == 2, uint16_t, uint8_t>::type;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t rb = static_cast<int64_t>(blockIdx.x) * 8 + (lane & 7);
  const int64_t kb = (static_cast<int64_t>(blockIdx.y) * kKmWarps + warp) * 4 + (lane >> 3);
  const int64_t r0 = rb * n, k0 = kb * n;
  if (r0 >= R || k0 >= K) return;
  if (vec && r0 + n <= R && k0 + n <= K) {
    uint32_t w[n][4];
#pragma unroll
    for (int q = 0; q < n; ++q) {
      const uint4 v = *reinterpret_cast<const uint4*>(src + (r0 + (k0 + q) * ld) * EB);
      w[q][0] = v.x; w[q][1] = v.y; w[q][2] = v.z; w[q][3] = v.w;
    }
    transpose_block<EB>(w);
#pragma unroll
    for (int q = 0; q < n; ++q)
      *reinterpret_cast<uint4*>(dst + ((r0 + q) * pitch + k0) * EB) = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
  } else {
    const T* s = reinterpret_cast<const T*>(src);
    T* d = reinterpret_cast<T*>(dst);
    for (int q = 0; q < n && k0 + q < K; ++q)
      for (int x = 0; x < n && r0 + x < R; ++x) d[(r0 + x) * pitch + k0 + q] = s[r0 + x + (k0 + q) * ld];
  }
}

// Format conversions of an R x Cc column-major matrix (element (r, c) at r + c * ld), eight
// rows per work item with 16-byte bfloat16 / 32-byte FP32 accesses when vec (bases and
// leading dimensions allow it), element by element otherwise.
// kToBf16: dst (bfloat16) = nearest bfloat16 of src (FP32); else dst (FP32) = src (bfloat16).
template <bool kToBf16>
__global__ void __launch_bounds__(256) convert_kernel(const void* __restrict__ src, int64_t sld, void* __restrict__ dst,
                                                      int64_t dld, int64_t R, int64_t Cc, int vec) {
  const int64_t nch = (R + 7) / 8, items = nch * Cc;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < items; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / nch, r0 = (e - c * nch) * 8;
    if (kToBf16) {
      const float* s = static_cast<const float*>(src) + r0 + c * sld;
      uint16_t* d = static_cast<uint16_t*>(dst) + r0 + c * dld;
      if (vec && r0 + 8 <= R) {
        const float4 a = reinterpret_cast<const float4*>(s)[0], b = reinterpret_cast<const float4*>(s)[1];
        const float f[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
          w[q] = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(f[2 * q])) |
                 ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(f[2 * q + 1])) << 16);
        *reinterpret_cast<uint4*>(d) = make_uint4(w[0], w[1], w[2], w[3]);
      } else {
        for (int64_t r = r0; r < R && r < r0 + 8; ++r) d[r - r0] = __bfloat16_as_ushort(__float2bfloat16_rn(s[r - r0]));
      }
    } else {
      const uint16_t* s = static_cast<const uint16_t*>(src) + r0 + c * sld;
      float* d = static_cast<float*>(dst) + r0 + c * dld;
      if (vec && r0 + 8 <= R) {
        const uint4 w = *reinterpret_cast<const uint4*>(s);
        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
        float f[8];
#pragma unroll
        for (int q = 0; q < 4; ++q) { f[2 * q] = __uint_as_float(ws[q] << 16); f[2 * q + 1] = __uint_as_float(ws[q] & 0xffff0000u); }
        reinterpret_cast<float4*>(d)[0] = make_float4(f[0], f[1], f[2], f[3]);
        reinterpret_cast<float4*>(d)[1] = make_float4(f[4], f[5], f[6], f[7]);
      } else {
        for (int64_t r = r0; r < R && r < r0 + 8; ++r) d[r - r0] = __uint_as_float((uint32_t)s[r - r0] << 16);
      }
    }
  }
}

// C = beta C over an R x Cc column-major bfloat16 matrix (beta == 0 writes zeros: C is not read).
__global__ void scale_bf16_kernel(uint16_t* C, int64_t ldc, int64_t R, int64_t Cc, float beta) {
  const int64_t total = R * Cc;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % R, j = e / R;
    uint16_t* c = C + i + j * ldc;
    const float v = beta == 0.0f ? 0.0f : beta * __uint_as_float((uint32_t)*c << 16);
    *c = __bfloat16_as_ushort(__float2bfloat16_rn(v));
  }
}

static unsigned grid_for(int64_t items) {
  const int64_t b = (items + 255) / 256;
  return (unsigned)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

}  // namespace

cudaError_t launch_f32_to_bf16(const float* src, int64_t sld, uint16_t* dst, int64_t dld, int64_t R, int64_t Cc,
                               cudaStream_t st) {
  if (R == 0 || Cc == 0) return cudaSuccess;
  const int vec = ((reinterpret_cast<uintptr_t>(src) & 15u) == 0 && (sld & 3) == 0 &&
                   (reinterpret_cast<uintptr_t>(dst) & 15u) == 0 && (dld & 7) == 0) ? 1 : 0;
  convert_kernel<true><<<grid_for((R + 7) / 8 * Cc), 256, 0, st>>>(src, sld, dst, dld, R, Cc, vec);
  return cudaGetLastError();
}

cudaError_t launch_bf16_to_f32(const uint16_t* src, int64_t sld, float* dst, int64_t dld, int64_t R, int64_t Cc,
                               cudaStream_t st) {
  if (R == 0 || Cc == 0) return cudaSuccess;
  const int vec = ((reinterpret_cast<uintptr_t>(src) & 15u) == 0 && (sld & 7) == 0 &&
                   (reinterpret_cast<uintptr_t>(dst) & 15u) == 0 && (dld & 3) == 0) ? 1 : 0;
  convert_kernel<false><<<grid_for((R + 7) / 8 * Cc), 256, 0, st>>>(src, sld, dst, dld, R, Cc, vec);
  return cudaGetLastError();
}

cudaError_t launch_scale_bf16(uint16_t* C, int64_t ldc, int64_t R, int64_t Cc, float beta, cudaStream_t st) {
  if (R == 0 || Cc == 0) return cudaSuccess;
  scale_bf16_kernel<<<grid_for(R * Cc), 256, 0, st>>>(C, ldc, R, Cc, beta);
  return cudaGetLastError();
}

int64_t tc_kmajor_pitch(int64_t K, int elem_bytes) {
  const int64_t v = 16 / elem_bytes;
  return (K + v - 1) / v * v;
}

cudaError_t launch_kmajor_copy(const void* src, int64_t R, int64_t K, int64_t ld, int elem_bytes, void* dst,
                               int64_t pitch, cudaStream_t st) {
  if (R == 0 || K == 0) return cudaSuccess;
  const int vec = ((reinterpret_cast<uintptr_t>(src) & 15u) == 0 && ((ld * elem_bytes) & 15) == 0 &&
                   (reinterpret_cast<uintptr_t>(dst) & 15u) == 0 && ((pitch * elem_bytes) & 15) == 0)
                      ? 1
                      : 0;
  const int64_t n = 16 / elem_bytes;  // block edge (elements)
  const int64_t nrb = (R + n - 1) / n, nkb = (K + n - 1) / n;
  const dim3 grid(static_cast<unsigned>((nrb + 7) / 8), static_cast<unsigned>((nkb + 4 * kKmWarps - 1) / (4 * kKmWarps)));
  if (grid.y > 65535u) return cudaErrorInvalidConfiguration;
  if (elem_bytes == 2)
    kmajor_copy_kernel<2><<<grid, kKmWarps * 32, 0, st>>>(static_cast<const uint8_t*>(src), R, K, ld,
                                                          static_cast<uint8_t*>(dst), pitch, vec);
  else
    kmajor_copy_kernel<1><<<grid, kKmWarps * 32, 0, st>>>(static_cast<const uint8_t*>(src), R, K, ld,
                                                          static_cast<uint8_t*>(dst), pitch, vec);
  return cudaGetLastError();
}

}  // namespace ftk
