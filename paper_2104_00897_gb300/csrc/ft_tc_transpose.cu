// K-major copies of MN-major operands for the tensor-core path. The tcgen05 product kernel
// and the checksum encode read every operand K-contiguous (rows of K elements, 128-byte
// swizzled TMA boxes); an operand stored the other way (op(A) with its rows contiguous, or
// op(B) with its columns contiguous) is transposed once into library workspace through
// shared memory, with 16-byte loads and stores on both sides where alignment allows.
#include <cstdint>
#include <type_traits>

#include "ft_tc.h"

namespace ftk {

namespace {

constexpr int kTT = 64;  // tile edge (elements) of the transpose

// dst[r * pitch + k] = src[r + k * ld] for r < R, k < K; EB bytes per element (1 or 2).
// Tile (r0, k0) of 64 x 64: loaded with rows r contiguous, stored with k contiguous.
template <int EB>
__global__ void __launch_bounds__(256) kmajor_copy_kernel(const uint8_t* __restrict__ src, int64_t R, int64_t K,
                                                          int64_t ld, uint8_t* __restrict__ dst, int64_t pitch,
                                                          int vec) {
  using T = typename std::conditional<EB == 2, uint16_t, uint8_t>::type;
  __shared__ T tile[kTT][kTT + 16 / EB];  // tile[k][r], padded against bank conflicts
  const T* s = reinterpret_cast<const T*>(src);
  T* d = reinterpret_cast<T*>(dst);
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * kTT, k0 = static_cast<int64_t>(blockIdx.y) * kTT;
  constexpr int V = 16 / EB;  // elements per 16-byte vector
  const bool full = vec && r0 + kTT <= R && k0 + kTT <= K;
  if (full) {
    for (int q = threadIdx.x; q < kTT * (kTT / V); q += 256) {
      const int kk = q / (kTT / V), rv = (q % (kTT / V)) * V;
      const uint4 w = *reinterpret_cast<const uint4*>(s + (r0 + rv) + (k0 + kk) * ld);
      const T* e = reinterpret_cast<const T*>(&w);
#pragma unroll
      for (int x = 0; x < V; ++x) tile[kk][rv + x] = e[x];
    }
  } else {
    for (int q = threadIdx.x; q < kTT * kTT; q += 256) {
      const int kk = q / kTT, rr = q % kTT;
      const int64_t r = r0 + rr, k = k0 + kk;
      tile[kk][rr] = (r < R && k < K) ? s[r + k * ld] : T(0);
    }
  }
  __syncthreads();
  if (full) {
    for (int q = threadIdx.x; q < kTT * (kTT / V); q += 256) {
      const int rr = q / (kTT / V), kv = (q % (kTT / V)) * V;
      uint4 w;
      T* e = reinterpret_cast<T*>(&w);
#pragma unroll
      for (int x = 0; x < V; ++x) e[x] = tile[kv + x][rr];
      *reinterpret_cast<uint4*>(d + (r0 + rr) * pitch + k0 + kv) = w;
    }
  } else {
    for (int q = threadIdx.x; q < kTT * kTT; q += 256) {
      const int rr = q / kTT, kk = q % kTT;
      const int64_t r = r0 + rr, k = k0 + kk;
      if (r < R && k < K) d[r * pitch + k] = tile[kk][rr];
    }
  }
}

}  // namespace

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
  const dim3 grid(static_cast<unsigned>((R + kTT - 1) / kTT), static_cast<unsigned>((K + kTT - 1) / kTT));
  if (grid.y > 65535u) return cudaErrorInvalidConfiguration;
  if (elem_bytes == 2)
    kmajor_copy_kernel<2><<<grid, 256, 0, st>>>(static_cast<const uint8_t*>(src), R, K, ld,
                                                static_cast<uint8_t*>(dst), pitch, vec);
  else
    kmajor_copy_kernel<1><<<grid, 256, 0, st>>>(static_cast<const uint8_t*>(src), R, K, ld,
                                                static_cast<uint8_t*>(dst), pitch, vec);
  return cudaGetLastError();
}

}  // namespace ftk
