// Encode pre-pass of the reduced-precision (tcgen05) ABFT GEMM, and the layout of its
// workspace. FT-BLAS (Zhai et al., ICS '21) Section II.A: the checksum row e^T A of A^c and
// the checksum column B e of B^r, per verification tile, plus the magnitude sums the
// thresholds need; Section V.B reads each operand element once for all of them.
#include <cstring>

#include "ft_device.cuh"
#include "ft_internal.h"
#include "ft_tc.h"
#include "ft_tc_elem.cuh"

namespace ftk {

namespace {

constexpr int BM = kTcBM;             // 128 rows of A per block (the tile's rows)

// ---------------------------------------------------------------------------------------
// Encode pre-pass (bandwidth-bound): one read of A and one read of B. Kernel-frame A is
// M x K and B is K x N, both K-contiguous, so each is a set of K-contiguous lines: the
// rows of A, the columns of B. A CTA takes a block of L lines (the 128 rows of a tile of
// A, the 248 columns of a tile of B) and 256 (BF16) or 512 (E4M3) consecutive k. Lane l of
// warp w loads 16 bytes of k per line (8 BF16 or 16 E4M3 elements) of lines w, w + 8, ...;
// the eight warps' partial sums meet in shared memory. From A it forms only what every
// tile's row check needs, sum_k |A(i,k)| per row; e^T A per row block, which only the
// lazy column side of a mismatching tile uses, is formed after the GEMM for those tiles'
// row blocks alone (tc_colsum_kernel).
// Sums over a block are plain binary32 sums: their rounding, at most gamma_L(2^-24) times
// the sum of magnitudes in any order, is a term of the thresholds. Sums of magnitudes round
// upward, so they bound the exact sums.
// ---------------------------------------------------------------------------------------
constexpr int ENC_WARPS = 8;
// Elements per lane and line (one 16-byte load: 8 BF16 or 16 E4M3 codes) and k per CTA.
template <int KIND>
struct EncVec {
  static constexpr int kV = KIND == 1 ? 16 : 8;
  static constexpr int kKC = 32 * kV;
};
constexpr int enc_kc(int kind) { return kind == 1 ? EncVec<1>::kKC : EncVec<0>::kKC; }

// Lane l holds la[u], a partial sum for line u of a group of 8 lines. Returns the upward
// sum over the 32 lanes of line (l >> 2): recursive halving, 9 shuffles.
__device__ __forceinline__ float reduce_scatter8_up(const float (&la)[8], int lane) {
  const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
  float v4[4], v2[2];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float keep = h16 ? la[4 + j] : la[j], send = h16 ? la[j] : la[4 + j];
    v4[j] = __fadd_ru(keep, __shfl_xor_sync(0xffffffffu, send, 16));
  }
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const float keep = h8 ? v4[2 + j] : v4[j], send = h8 ? v4[j] : v4[2 + j];
    v2[j] = __fadd_ru(keep, __shfl_xor_sync(0xffffffffu, send, 8));
  }
  float v = __fadd_ru(h4 ? v2[1] : v2[0], __shfl_xor_sync(0xffffffffu, h4 ? v2[0] : v2[1], 4));
  v = __fadd_ru(v, __shfl_xor_sync(0xffffffffu, v, 2));
  return __fadd_ru(v, __shfl_xor_sync(0xffffffffu, v, 1));
}

// s[q] += x[q] for q < N, two lanes of binary32 per instruction (add.rn.f32x2): each sum
// takes the same values in the same order as N scalar additions.
template <int N>
__device__ __forceinline__ void add_f32x2n(float (&s)[N], const float (&x)[N]) {
#pragma unroll
  for (int q = 0; q < N; q += 2) {
    unsigned long long a = (static_cast<unsigned long long>(__float_as_uint(s[q + 1])) << 32) | __float_as_uint(s[q]);
    const unsigned long long b =
        (static_cast<unsigned long long>(__float_as_uint(x[q + 1])) << 32) | __float_as_uint(x[q]);
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(a) : "l"(a), "l"(b));
    s[q] = __uint_as_float(static_cast<uint32_t>(a));
    s[q + 1] = __uint_as_float(static_cast<uint32_t>(a >> 32));
  }
}

struct EncArgs {
  const void* X; int64_t ld;
  int32_t nlines, K, L;
  int32_t nkc;             // k-chunks per line block
  float* rowAbsA;          // rows pass: [M] upward sum_k |A(i,k)|, by the block's last k-chunk
  unsigned* rowdone;       // rows pass: [nblocks] k-chunks finished (zeroed before the launch)
  float* sum;              // rows pass: [nblocks][pitch] e^T A per block
  float* abs_sum;          // rows pass: [nblocks][pitch] upward sum_{i in block} |A(i,k)|
  int64_t pitch;           // also the checksum operand's row pitch (elements)
  TcPending* pend;         // rows pass: its tile count is zeroed before the GEMM
  float* line_part;        // rows pass: [nkc][M] upward sum of |A(i,k)| over one k-chunk
  float* maxAbsBe;         // [nblocks of B]
  void* chk;               // columns pass: pieces of B e in rows J*8 + p (unused rows zero)
};

// Shared memory of one encode CTA, declared once per kernel (both roles use it): the
// float4 stores into the reduction arrays need their 16-byte alignment.
template <int KC>
struct __align__(16) EncSmem {
  float red_s[ENC_WARPS][KC];
  float red_a[ENC_WARPS][KC];
  int last_chunk;
};

// kV consecutive elements of one K-contiguous line from k (a multiple of kV), zero at and
// beyond K: one 16-byte load (ld a multiple of 16 bytes, base 16-byte aligned).
template <int KIND>
__device__ __forceinline__ uint4 load_line16(const uint8_t* line, int64_t k, int32_t K) {
  constexpr int V = EncVec<KIND>::kV, EB = Elem<KIND>::kBytes;
  if (k + V <= K) return *reinterpret_cast<const uint4*>(line + k * EB);
  uint32_t t[4] = {0u, 0u, 0u, 0u};
  for (int q = 0; q < V; ++q)
    if (k + q < K) {
      const uint32_t v = EB == 2 ? reinterpret_cast<const uint16_t*>(line)[k + q] : line[k + q];
      t[(q * EB) >> 2] |= v << (8 * ((q * EB) & 3));
    }
  return make_uint4(t[0], t[1], t[2], t[3]);
}
template <int KIND>
__device__ __forceinline__ void unpack16(const uint4 w, float (&x)[EncVec<KIND>::kV]) {
  if constexpr (KIND == 0) {
    float y[8];
    Elem<0>::unpack(w, y);
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = y[q];
  } else {
    float y[8];
    Elem<1>::unpack(make_uint2(w.x, w.y), y);
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = y[q];
    Elem<1>::unpack(make_uint2(w.z, w.w), y);
#pragma unroll
    for (int q = 0; q < 8; ++q) x[8 + q] = y[q];
  }
}

template <bool kRowsOfA, int KIND>
__device__ __forceinline__ void encode_block(const EncArgs& g, int blk, int kc, EncSmem<EncVec<KIND>::kKC>& sm) {
  constexpr int V = EncVec<KIND>::kV, KC = EncVec<KIND>::kKC;
  auto& red_s = sm.red_s;
  auto& red_a = sm.red_a;
  int& last_chunk = sm.last_chunk;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t line0 = (int64_t)blk * g.L;
  const int nI = (int)min((int64_t)g.L, (int64_t)g.nlines - line0);
  const int64_t k = (int64_t)kc * KC + lane * V;
  const uint8_t* X = static_cast<const uint8_t*>(g.X);
  constexpr int EB = Elem<KIND>::kBytes;
  float s[V], a[V];
#pragma unroll
  for (int q = 0; q < V; ++q) { s[q] = 0.f; a[q] = 0.f; }
  const int T = (nI + ENC_WARPS - 1) / ENC_WARPS;  // lines per warp, rounded up
  // 8 lines loaded per iteration: 128 bytes in flight per lane
  for (int t0 = 0; t0 < T; t0 += 8) {
    uint4 raw[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int l = warp + ENC_WARPS * (t0 + u);
      raw[u] = (l < nI && k < g.K) ? load_line16<KIND>(X + (line0 + l) * g.ld * EB, k, g.K) : make_uint4(0u, 0u, 0u, 0u);
    }
    float la[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      float x[V];
      unpack16<KIND>(raw[u], x);
      float lsum = 0.f;
#pragma unroll
      for (int q = 0; q < V; ++q) {
        if (kRowsOfA) {
          lsum = __fadd_ru(lsum, fabsf(x[q]));
        } else {
          a[q] = __fadd_ru(a[q], fabsf(x[q]));
        }
      }
      if (!kRowsOfA) add_f32x2n(s, x);
      la[u] = lsum;
    }
    if (kRowsOfA) {
      const float v = reduce_scatter8_up(la, lane);
      const int l = warp + ENC_WARPS * (t0 + (lane >> 2));
      if ((lane & 3) == 0 && l < nI) g.line_part[(int64_t)kc * g.nlines + line0 + l] = v;
    }
  }
  const int tk = threadIdx.x;
  if (kRowsOfA) {
    // (e^T A and sum_i |A(i,k)| per row block are formed only for the row blocks of tiles
    // that reach the resolve pass: tc_colsum_kernel)
    if (blk == 0 && kc == 0 && tk == 0) g.pend->count = 0u;
    // the line block's last k-chunk to finish sums the per-chunk partials of its rows
    // (in chunk order: the result does not depend on which chunk finished last)
    __threadfence();
    __syncthreads();
    if (tk == 0) last_chunk = atomicAdd(&g.rowdone[blk], 1u) == (unsigned)(g.nkc - 1);
    __syncthreads();
    if (last_chunk) {
      __threadfence();
      if (tk < nI) {
        float a2 = 0.f;
        for (int c2 = 0; c2 < g.nkc; ++c2) a2 = __fadd_ru(a2, __ldcg(&g.line_part[(int64_t)c2 * g.nlines + line0 + tk]));
        g.rowAbsA[line0 + tk] = a2;
      }
    }
  } else {
#pragma unroll
    for (int q = 0; q < V; q += 4) {
      *reinterpret_cast<float4*>(&red_s[warp][lane * V + q]) = make_float4(s[q], s[q + 1], s[q + 2], s[q + 3]);
      *reinterpret_cast<float4*>(&red_a[warp][lane * V + q]) = make_float4(a[q], a[q + 1], a[q + 2], a[q + 3]);
    }
    __syncthreads();
    float mx = 0.f;
#pragma unroll
    for (int t2 = tk; t2 < KC; t2 += ENC_WARPS * 32) {  // one or two k per thread
      const int64_t kk = (int64_t)kc * KC + t2;
      float S = 0.f, Aab = 0.f;
#pragma unroll
      for (int w = 0; w < ENC_WARPS; ++w) { S += red_s[w][t2]; Aab = __fadd_ru(Aab, red_a[w][t2]); }
      if (kk >= g.K) continue;
      mx = fmaxf(mx, Aab);
      if (KIND == 0) {
        // three bfloat16 pieces, each the nearest bfloat16 of what the previous ones leave:
        // together they hold the binary32 sum exactly (8 + 8 + 8 significand bits)
        const __nv_bfloat16 h = __float2bfloat16_rn(S);
        const float r1 = S - __bfloat162float(h);
        const __nv_bfloat16 m = __float2bfloat16_rn(r1);
        const __nv_bfloat16 lo = __float2bfloat16_rn(r1 - __bfloat162float(m));
        constexpr int kChk = tc_chk_rows(0);
        uint16_t* col = static_cast<uint16_t*>(g.chk) + (int64_t)blk * kChk * g.pitch + kk;
        col[0] = __bfloat16_as_ushort(h);
        col[g.pitch] = __bfloat16_as_ushort(m);
        col[2 * g.pitch] = __bfloat16_as_ushort(lo);
#pragma unroll
        for (int r = 3; r < kChk; ++r) col[r * g.pitch] = 0;
      } else {
        // eight e4m3 pieces with scales 2^(9 - 4p): piece p is the nearest e4m3 of
        // r / 2^(9 - 4p), r what the previous pieces leave; a subnormal piece is flushed to
        // zero and its value carried. |S| <= 248 * 448 < 256 * 2^9, and each remainder is at
        // most half an e4m3 unit of the piece before, so every r / 2^(9 - 4p) stays within
        // +-256, and r - piece is exact (the two are within a factor of two). The last
        // remainder is zero: the pieces take 4 bits each of S's at most 24.
        uint8_t* col = static_cast<uint8_t*>(g.chk) + (int64_t)blk * tc_chk_rows(1) * g.pitch + kk;
        float r = S, inv = 0x1p-9f, sc = 0x1p9f;
#pragma unroll
        for (int pc = 0; pc < Elem<1>::kPieces; ++pc, inv *= 16.f, sc *= 0.0625f) {
          __nv_fp8_storage_t q = __nv_cvt_float_to_fp8(r * inv, __NV_SATFINITE, __NV_E4M3);
          if ((q & 0x78u) == 0) q = 0;
          col[pc * g.pitch] = q;
          r -= e4m3_to_f32(q) * sc;
        }
      }
    }
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, w));
    if (lane == 0) atomicMax(reinterpret_cast<unsigned int*>(&g.maxAbsBe[blk]), __float_as_uint(mx));
  }
}

// One launch for both operands: blocks x < nMb encode row blocks of A, the rest column
// blocks of B, so the two reads overlap.
template <int KIND>
__global__ void __launch_bounds__(256, 3) encode_kernel(EncArgs ga, EncArgs gb, int nMb) {
  __shared__ EncSmem<EncVec<KIND>::kKC> sm;
  if ((int)blockIdx.x < nMb) encode_block<true, KIND>(ga, blockIdx.x, blockIdx.y, sm);
  else encode_block<false, KIND>(gb, blockIdx.x - nMb, blockIdx.y, sm);
}

// Eight codes per thread through the encode's own unpacking (codes 8-byte aligned).
__global__ void decode_e4m3_kernel(const uint8_t* codes, float* out, int64_t n) {
  const int64_t groups = (n + 7) / 8;
  for (int64_t g8 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g8 < groups; g8 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = 8 * g8;
    float x[8];
    Elem<1>::unpack(Elem<1>::load_raw(codes + k, 0, (int32_t)(n - k < 8 ? n - k : 8)), x);
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (k + q < n) out[k + q] = x[q];
  }
}

}  // namespace

cudaError_t launch_decode_e4m3(const uint8_t* codes, float* out, int64_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const int64_t blocks = ((n + 7) / 8 + 255) / 256;
  decode_e4m3_kernel<<<(unsigned)(blocks < 1024 ? blocks : 1024), 256, 0, st>>>(codes, out, n);
  return cudaGetLastError();
}

int64_t tc_kpitch(int32_t K) { return (K + 15) / 16 * 16; }

size_t tc_workspace_bytes(int32_t M, int32_t N, int32_t K, int kind) {
  const int64_t bn = tc_bn_prot(kind), chk = tc_chk_rows(kind);
  const int64_t nMb = (M + BM - 1) / BM, nNb = (N + bn - 1) / bn;
  const int64_t kpitch = tc_kpitch(K), nkc = (K + enc_kc(kind) - 1) / enc_kc(kind);
  const int64_t eb = kind == 0 ? 2 : 1;
  auto up = [](int64_t x) { return (x + 255) / 256 * 256; };
  return up(nNb * chk * kpitch * eb) + up(nMb * kpitch * 4) + up(nMb * kpitch * 4) + up(M * 4) +
         up(nNb * 4 + nMb * 4) + up(nkc * M * 4) + up((int64_t)sizeof(TcPending));
}

TcWorkspace tc_workspace_carve(void* base, int32_t M, int32_t N, int32_t K, int kind) {
  const int64_t bn = tc_bn_prot(kind), chk = tc_chk_rows(kind);
  const int64_t nMb = (M + BM - 1) / BM, nNb = (N + bn - 1) / bn;
  const int64_t kpitch = tc_kpitch(K), nkc = (K + enc_kc(kind) - 1) / enc_kc(kind);
  const int64_t eb = kind == 0 ? 2 : 1;
  auto up = [](int64_t x) { return (x + 255) / 256 * 256; };
  char* c = static_cast<char*>(base);
  TcWorkspace w;
  w.chk = c; c += up(nNb * chk * kpitch * eb);
  w.kpitch = kpitch;
  w.sA = reinterpret_cast<float*>(c); c += up(nMb * kpitch * 4);
  w.absSA = reinterpret_cast<float*>(c); c += up(nMb * kpitch * 4);
  w.rowAbsA = reinterpret_cast<float*>(c); c += up(M * 4);
  w.maxAbsBe = reinterpret_cast<float*>(c);
  w.rowdone = reinterpret_cast<unsigned*>(w.maxAbsBe + nNb);
  w.zero_bytes = (size_t)(nNb * 4 + nMb * 4);  // maxAbsBe and rowdone, cleared before the encode
  c += up(nNb * 4 + nMb * 4);
  w.rowPart = reinterpret_cast<float*>(c); c += up(nkc * M * 4);
  w.pend = reinterpret_cast<TcPending*>(c); c += up((int64_t)sizeof(TcPending));
  w.bytes = static_cast<size_t>(c - static_cast<char*>(base));
  return w;
}

template <int KIND>
static void launch_encode_kind(const TcParams& p, const TcWorkspace& w, cudaStream_t st) {
  constexpr int bn = tc_bn_prot(KIND);
  const int nMb = (p.M + BM - 1) / BM, nNb = (p.N + bn - 1) / bn, nkc = (p.K + EncVec<KIND>::kKC - 1) / EncVec<KIND>::kKC;
  EncArgs ga, gb;
  std::memset(&ga, 0, sizeof(ga));
  ga.X = p.A; ga.ld = p.lda; ga.nlines = p.M; ga.K = p.K; ga.L = BM; ga.nkc = nkc;
  ga.sum = w.sA; ga.abs_sum = w.absSA; ga.line_part = w.rowPart; ga.rowAbsA = w.rowAbsA; ga.rowdone = w.rowdone;
  ga.pitch = w.kpitch; ga.pend = w.pend;
  std::memset(&gb, 0, sizeof(gb));
  gb.X = p.B; gb.ld = p.ldb; gb.nlines = p.N; gb.K = p.K; gb.L = bn; gb.nkc = nkc;
  gb.maxAbsBe = w.maxAbsBe; gb.chk = w.chk; gb.pitch = w.kpitch;
  encode_kernel<KIND><<<dim3(nMb + nNb, nkc), ENC_WARPS * 32, 0, st>>>(ga, gb, nMb);
}

cudaError_t launch_tc_encode(const TcParams& p, const TcWorkspace& w, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(w.maxAbsBe, 0, w.zero_bytes, st);
  if (e != cudaSuccess) return e;
  if (p.kind == 0) launch_encode_kind<0>(p, w, st);
  else launch_encode_kind<1>(p, w, st);
  return cudaGetLastError();
}

}  // namespace ftk
