// Emulated FP64 ABFT-protected GEMM on the fifth-generation tensor cores (sm_103a).
//
// GB300's binary64 units retire about 1.26 TFLOP/s; its E4M3 tensor cores about 3000 times
// that. Here binary64 operands are split into small integer slices whose products the
// tensor cores form exactly, and the checksums of FT-BLAS (Zhai et al., ICS '21) become
// exact integer relations:
//   - scales: row i of op(A) is scaled by 2^-e_i (e_i the binary exponent of its largest
//     magnitude), column j of op(B) by 2^-f_j, so every scaled value lies in (-1, 1);
//   - slices: x = sum_p a_p 16^-(p+1), a_p = nearest integer of 16 r_p, r_{p+1} = 16 r_p -
//     a_p 16 (exact in binary64); |a_0| <= 16, |a_p| <= 8: E4M3 values;
//   - groups: G_g = sum_{p+q=g} A_p B_q for g < s, accumulated by tcgen05 kind::f8f6f4 in
//     binary32; every partial sum is an integer below 2^24 (K <= 2^18 / (s+2)), so exact;
//   - checksums (Section II.A): the last rows of each B stage hold the four base-16 digits
//     of B_q e over the tile's columns, so the MMA also forms sum_t 16^t A_p (B_q e)_t. The
//     row sums of every group are compared with it exactly: the threshold is zero;
//   - combination: S = sum_g G_g 16^(s-1-g), exact: two 64-bit Horner sums (one step per
//     group) over the first and second half of the groups in a per-CTA scratch, joined in
//     128 bits after the last group; v = S 2^(e_i + f_j - 4(s+1)) rounded once to binary64 and C = alpha v +
//     beta C_in, checked by its row sums against alpha sum_j v + beta sum_j C_in within the
//     rounding of both (C = beta C folded in and verified after the output, Section V.B);
//   - locate and correct (Sections V.A, VI.C): a flagged row is not stored; the resolve
//     pass recomputes it exactly from the slices and stores the recomputed values, so C is
//     the fault-free C bit for bit. Elements that differed are the located errors.
//
// Kernels: exponent and slice kernels (bandwidth-bound passes over A and B), the checksum
// digits of the B slices, the persistent product kernel (warp 0 TMA, warp 1 MMA issue,
// warps 2-5 epilogue, TMEM double-buffered per group), and the resolve pass.
#include <climits>
#include <cstring>

#include "ft_device.cuh"
#include "ft_emu.h"
#include "ft_internal.h"

namespace ftk {

namespace {

constexpr int EBM = kEmuBM;
constexpr int EBNM = 256;             // MMA N = TMEM columns per buffer = B stage rows
constexpr int EBKB = 128;             // k-tile: 128 E4M3 values = 128 bytes
constexpr int ESTAGES = 4;
constexpr int ENTHREADS = 192;
constexpr uint32_t ETMEM_COLS = 512;
constexpr int32_t kExpNone = INT32_MIN / 2;  // exponent of a zero line (atomicMax start value)

// ---------------------------------------------------------------------------------------
// Exact binary64 helpers
// ---------------------------------------------------------------------------------------
// 2^n as a binary64 value, n in [-1074, 1023].
__device__ __forceinline__ double pow2(int n) {
  if (n >= -1022) return __longlong_as_double(static_cast<long long>(n + 1023) << 52);
  return __longlong_as_double(1ll << (n + 1074));
}

// x 2^n rounded once to nearest (ties to even), as the standard scaling does: one
// multiplication by an exact power of two when 2^n is representable; else exact steps
// toward the range first.
__device__ double scale_pow2(double x, int n) {
  if (n > 1023) {
    x = __dmul_rn(x, pow2(1023));
    n -= 1023;
    if (n > 1023) n = 1023;
    return __dmul_rn(x, pow2(n));
  }
  while (n < -1074 && fabs(x) >= 0x1p-822) {  // exact: the result stays normal
    x = __dmul_rn(x, 0x1p-200);
    n += 200;
  }
  if (n < -1074) return __dmul_rn(x, 0.0);  // below half the smallest subnormal: a signed zero
  return __dmul_rn(x, pow2(n));
}

// Nearest binary64 value (ties to even) of a 128-bit integer. Values of more than 64 bits
// are shifted to 64 bits with the dropped bits' OR kept in the last bit (11 bits below
// the 53 kept ones, so the one rounding of the 64-bit conversion is the right one), then
// scaled back exactly.
__device__ double i128_to_f64(__int128 x) {
  const bool neg = x < 0;
  const unsigned __int128 u = neg ? (unsigned __int128)0 - (unsigned __int128)x : (unsigned __int128)x;
  const uint64_t hi = static_cast<uint64_t>(u >> 64), lo = static_cast<uint64_t>(u);
  double r;
  if (hi == 0) {
    r = __ull2double_rn(lo);
  } else {
    const int sh = 64 - __clzll(static_cast<long long>(hi));  // 1 .. 64
    uint64_t top, sticky;
    if (sh == 64) {
      top = hi;
      sticky = lo != 0;
    } else {
      top = (hi << (64 - sh)) | (lo >> sh);
      sticky = (lo & ((1ull << sh) - 1)) != 0;
    }
    r = __dmul_rn(__ull2double_rn(top | sticky), pow2(sh));
  }
  return neg ? -r : r;
}

// E4M3 code of an integer v, |v| <= 16 (at most four significant bits: exact).
__device__ __forceinline__ uint32_t e4m3_of_int(int v) {
  if (v == 0) return 0u;
  const uint32_t n = static_cast<uint32_t>(v < 0 ? -v : v);
  const int E = 31 - __clz(n);  // 0 .. 4
  const uint32_t mant = E <= 3 ? (n << (3 - E)) & 7u : (n >> (E - 3)) & 7u;
  return (v < 0 ? 0x80u : 0u) | (static_cast<uint32_t>(E + 7) << 3) | mant;
}
// Integer value of an E4M3 code that holds one (the slices and digits only hold integers).
__device__ __forceinline__ int int_of_e4m3(uint32_t b) {
  const int E = static_cast<int>((b >> 3) & 15u), m = static_cast<int>(b & 7u);
  if (E < 7) return 0;
  const int mag = ((8 + m) << (E - 7)) >> 3;
  return (b & 0x80u) ? -mag : mag;
}

// frexp exponent of a finite nonzero value from its bits (subnormals included).
__device__ __forceinline__ int frexp_exp_bits(unsigned long long b) {
  const int E = static_cast<int>((b >> 52) & 0x7ff);
  if (E != 0) return E - 1022;
  const unsigned long long m = b & ((1ull << 52) - 1);
  return (64 - __clzll(static_cast<long long>(m))) - 1074;
}

// The slices of x = a 2^-e (|x| < 1) in integer arithmetic. With N_p = rint(16^(p+1) x)
// (nearest, ties to even), the slices of the recurrence r_0 = 16 x, a_p = rint(r_p),
// r_{p+1} = 16 (r_p - a_p) are a_p = N_p - 16 N_{p-1}: r_p = 16^(p+1) x - 16 N_{p-1}, and
// moving by a multiple of 16 (an even integer) commutes with rounding to nearest even.
// a = M 2^E_a exactly (M < 2^53), so N_p is M shifted to the binary point 4 (p+1) places
// below x's and rounded there; no binary64 arithmetic is involved. s <= 15 keeps N_p below
// 2^60.
__device__ __forceinline__ void int_slices(unsigned long long b, int e, int s, int (&out)[kEmuSlicesMax]) {
  const int Ef = static_cast<int>((b >> 52) & 0x7ff);
  const unsigned long long mant = b & ((1ull << 52) - 1);
  const unsigned long long M = Ef ? (mant | (1ull << 52)) : mant;
  const int base = (Ef ? Ef : 1) - 1075 - e;  // x = M 2^base
  const bool neg = (b >> 63) != 0;
  long long prev = 0;
#pragma unroll
  for (int q = 0; q < kEmuSlicesMax; ++q) {
    if (q >= s) {  // unused slices are zero (the loop stays unrolled, the array in registers)
      out[q] = 0;
      continue;
    }
    const int sh = -(base + 4 * (q + 1));
    unsigned long long n;
    if (M == 0 || sh >= 64) {
      n = 0;
    } else if (sh <= 0) {
      n = M << (-sh);
    } else {
      const unsigned long long qq = M >> sh, rem = M & ((1ull << sh) - 1), half = 1ull << (sh - 1);
      n = qq + ((rem > half || (rem == half && (qq & 1ull))) ? 1ull : 0ull);
    }
    const long long N = neg ? -static_cast<long long>(n) : static_cast<long long>(n);
    out[q] = static_cast<int>(N - 16 * prev);
    prev = N;
  }
}

// ---------------------------------------------------------------------------------------
// Split: exponents, slices and checksum digits (bandwidth-bound passes)
// ---------------------------------------------------------------------------------------
constexpr int kExpChunk = 2048;  // k per CTA of the exponent pass

// Largest frexp exponent of each line r of src (atomicMax into e[r]), and non-finite flags
// of the lines and of their blocks of blk lines. KC: k is the contiguous index (lanes over
// k); otherwise lines are contiguous (lanes over lines).
template <bool KC>
__global__ void __launch_bounds__(256) emu_exp_kernel(EmuSource src, int64_t K, int32_t* e, uint8_t* bad,
                                                      uint8_t* blk_bad, int blk) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t k0 = static_cast<int64_t>(blockIdx.y) * kExpChunk;
  const int64_t k1 = min(K, k0 + kExpChunk);
  if (KC) {
    const int64_t r = static_cast<int64_t>(blockIdx.x) * 8 + warp;
    int m = kExpNone;
    bool nf = false;
    if (r < src.R)
      for (int64_t k = k0 + lane; k < k1; k += 32) {
        const unsigned long long x = reinterpret_cast<const unsigned long long*>(src.base)[r * src.rs + k * src.ks];
        if (((x >> 52) & 0x7ff) == 0x7ff) nf = true;
        else if ((x << 1) != 0) m = max(m, frexp_exp_bits(x));
      }
    m = __reduce_max_sync(0xffffffffu, m);
    nf = __any_sync(0xffffffffu, nf);
    if (lane == 0 && r < src.R) {
      if (m > kExpNone) atomicMax(&e[r], m);
      if (nf) { bad[r] = 1; blk_bad[r / blk] = 1; }
    }
  } else {
    __shared__ int sm[8][32];
    __shared__ int snf[8][32];
    const int64_t r = static_cast<int64_t>(blockIdx.x) * 32 + lane;
    int m = kExpNone, nf = 0;
    if (r < src.R)
      for (int64_t k = k0 + warp; k < k1; k += 8) {
        const unsigned long long x = reinterpret_cast<const unsigned long long*>(src.base)[r * src.rs + k * src.ks];
        if (((x >> 52) & 0x7ff) == 0x7ff) nf = 1;
        else if ((x << 1) != 0) m = max(m, frexp_exp_bits(x));
      }
    sm[warp][lane] = m;
    snf[warp][lane] = nf;
    __syncthreads();
    if (warp == 0 && r < src.R) {
      for (int w = 1; w < 8; ++w) { m = max(m, sm[w][lane]); nf |= snf[w][lane]; }
      if (m > kExpNone) atomicMax(&e[r], m);
      if (nf) { bad[r] = 1; blk_bad[r / blk] = 1; }
    }
  }
}

constexpr int kSliceRows = 32, kSliceK = 128;

// Slices of lines [r0, r0 + 32) x [k0, k0 + 128) of src into out[p][r][k] (E4M3 bytes,
// rows of kpitch bytes), p < s. Lines at and beyond R, lines holding a non-finite value and
// k at and beyond K give zero slices.
template <bool KC>
__global__ void __launch_bounds__(256) emu_slice_kernel(EmuSource src, int64_t K, int64_t R_pad, int64_t kpitch,
                                                        int s, const int32_t* e, const uint8_t* bad, uint8_t* out) {
  __shared__ unsigned long long tile[kSliceRows][kSliceK + 1];
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * kSliceRows, k0 = static_cast<int64_t>(blockIdx.y) * kSliceK;
  for (int idx = threadIdx.x; idx < kSliceRows * kSliceK; idx += 256) {
    const int rr = KC ? idx / kSliceK : idx % kSliceRows;
    const int kk = KC ? idx % kSliceK : idx / kSliceRows;
    const int64_t r = r0 + rr, k = k0 + kk;
    unsigned long long x = 0ull;
    if (r < src.R && k < K) x = reinterpret_cast<const unsigned long long*>(src.base)[r * src.rs + k * src.ks];
    tile[rr][kk] = x;
  }
  __syncthreads();
  const int64_t slice_bytes = R_pad * kpitch;
  for (int item = threadIdx.x; item < kSliceRows * (kSliceK / 4); item += 256) {
    const int rr = item / (kSliceK / 4), kq = item % (kSliceK / 4);
    const int64_t r = r0 + rr, k = k0 + 4 * kq;
    if (r >= R_pad || k >= kpitch) continue;
    const bool live = r < src.R && !bad[r];
    const int ex = (live && e[r] > kExpNone) ? e[r] : 0;
    uint32_t w[kEmuSlicesMax];
#pragma unroll
    for (int p = 0; p < kEmuSlicesMax; ++p) w[p] = 0u;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int a[kEmuSlicesMax];
      int_slices((live && k + q < K) ? tile[rr][4 * kq + q] : 0ull, ex, s, a);
#pragma unroll
      for (int p = 0; p < kEmuSlicesMax; ++p) w[p] |= e4m3_of_int(a[p]) << (8 * q);
    }
#pragma unroll
    for (int p = 0; p < kEmuSlicesMax; ++p)
      if (p < s) *reinterpret_cast<uint32_t*>(out + p * slice_bytes + r * kpitch + k) = w[p];
  }
}

// Checksum digits (protected launches): for each slice q, column block nb and k, v = sum
// over the block's bn columns of b_q(k, j), written as four base-16 digits d_t in [-8, 8]
// (nearest-integer division by 16) into rows nb * 8 + t of chk's slice q; rows 4..7 zero.
__global__ void __launch_bounds__(256) emu_digit_kernel(const uint8_t* bslices, int64_t n_pad, int64_t kpitch,
                                                        int bn, int nNb, uint8_t* chk) {
  const int64_t k = (static_cast<int64_t>(blockIdx.x) * 256 + threadIdx.x) * 4;
  const int nb = blockIdx.y, q = blockIdx.z;
  if (k >= kpitch) return;
  const uint8_t* src = bslices + static_cast<int64_t>(q) * n_pad * kpitch + static_cast<int64_t>(nb) * bn * kpitch + k;
  int v[4] = {0, 0, 0, 0};
  for (int jj = 0; jj < bn; ++jj) {
    const uint32_t wd = *reinterpret_cast<const uint32_t*>(src + jj * kpitch);
#pragma unroll
    for (int t = 0; t < 4; ++t) v[t] += int_of_e4m3((wd >> (8 * t)) & 0xffu);
  }
  uint32_t dw[kEmuDigits] = {0u, 0u, 0u, 0u};
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    int x = v[t];
#pragma unroll
    for (int d = 0; d < kEmuDigits; ++d) {
      const int c = static_cast<int>(rint(static_cast<double>(x) * 0.0625));
      dw[d] |= e4m3_of_int(x - 16 * c) << (8 * t);
      x = c;
    }
  }
  uint8_t* dst = chk + (static_cast<int64_t>(q) * nNb * kEmuChkRows + static_cast<int64_t>(nb) * kEmuChkRows) * kpitch + k;
#pragma unroll
  for (int d = 0; d < kEmuChkRows; ++d)
    *reinterpret_cast<uint32_t*>(dst + d * kpitch) = d < kEmuDigits ? dw[d] : 0u;
}

__global__ void emu_convert_kernel(const int64_t* words, double* out, int64_t n) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const __int128 x = (static_cast<__int128>(words[2 * i + 1]) << 64) | static_cast<__int128>(
                         static_cast<uint64_t>(words[2 * i]));
  out[i] = i128_to_f64(x);
}

// ---------------------------------------------------------------------------------------
// Product kernel
// ---------------------------------------------------------------------------------------
struct __align__(1024) EmuSmem {
  uint8_t a[ESTAGES][EBM * EBKB];
  uint8_t b[ESTAGES][EBNM * EBKB];
  uint64_t full[ESTAGES];
  uint64_t empty[ESTAGES];
  uint64_t tfull[2];             // accumulator buffer holds a finished group
  uint64_t tempty[2];            // accumulator buffer read by the 4 epilogue warps
  uint32_t tmem_base;
  int timeout;
  int nflag, first_row, pend_slot, tile_ok;
  double first_delta, first_tau;
};

__device__ void emu_record(const EmuParams& p, int kind, int64_t tr, int64_t tc, int64_t i, int64_t j, double delta,
                           double tau, double before, double after, int nr, int nc) {
  if (p.report == nullptr) return;
  const unsigned slot = atomicAdd(&p.report->n_records, 1u);
  if (slot >= FTBLAS_MAX_RECORDS) {
    atomicOr(&p.report->status, FT_STATUS_RECORDS_TRUNCATED);
    return;
  }
  ft_error_record_t& r = p.report->rec[slot];
  if (p.swap_report) {
    r.tile_row = tc; r.tile_col = tr; r.i = j; r.j = i;
    r.delta_row = 0.0; r.delta_col = delta; r.tau_row = 0.0; r.tau_col = tau;
    r.rows_flagged = nc; r.cols_flagged = nr;
  } else {
    r.tile_row = tr; r.tile_col = tc; r.i = i; r.j = j;
    r.delta_row = delta; r.delta_col = 0.0; r.tau_row = tau; r.tau_col = 0.0;
    r.rows_flagged = nr; r.cols_flagged = nc;
  }
  r.value_before = before;
  r.value_after = after;
  r.kind = kind;
  r.reserved = 0;
}

__device__ void emu_count(const EmuParams& p, uint64_t ft_report_t::*field) {
  if (p.report != nullptr) atomicAdd(reinterpret_cast<unsigned long long*>(&(p.report->*field)), 1ull);
}

// Persistent tile order: groups of 16 row tiles sweep the column tiles (L2 reuse of the
// slices' panels); the last column block, narrower when N is ragged, comes last.
constexpr int kEmuGroupM = 16;
__device__ __forceinline__ void emu_tile_coords(int t, int nMb, int nNb, int& mt, int& nt) {
  const int ncols = nNb - 1;
  if (t >= nMb * ncols) {
    mt = t - nMb * ncols;
    nt = ncols;
    return;
  }
  const int group = t / (kEmuGroupM * ncols);
  const int first_m = group * kEmuGroupM;
  const int gsize = min(kEmuGroupM, nMb - first_m);
  const int in_group = t - group * kEmuGroupM * ncols;
  mt = first_m + in_group % gsize;
  nt = in_group / gsize;
}

// 16 extra expected bytes on the staging barrier of k-tile kt (0: the middle one) of the
// first product of tile (mt, nt) when a stall point (test launches only) names it.
__device__ __forceinline__ uint32_t emu_stall_bytes(const EmuParams& p, int mt, int nt, int kt, int nk) {
  for (int e = 0; e < p.inj.n; ++e) {
    const InjectPoint& ip = p.inj.p[e];
    if (ip.site == kSiteStall && kt == (ip.kt > 0 ? ip.kt : nk / 2) && ip.i / EBM == mt && ip.j / p.bn == nt)
      return 16u;
  }
  return 0u;
}

// Smallest tile column > after of row gi holding an accumulator point of group g, or an
// output point when g is the last group; INT_MAX if none (test launches only).
__device__ __noinline__ int emu_next_inj_col(const EmuParams& p, int64_t gi, int g, int n0, int nJ, int after) {
  int best = INT_MAX;
  for (int e = 0; e < p.inj.n; ++e) {
    const InjectPoint& ip = p.inj.p[e];
    if (ip.i != gi) continue;
    const bool acc = ip.site == kSiteAccum && ip.mode == FT_MODE_BITFLIP && ip.kt == g;
    const bool out = ip.site == kSiteOutput && g == p.s - 1;
    if (!acc && !out) continue;
    const int c = ip.j - n0;
    if (c > after && c < nJ && c < best) best = c;
  }
  return best;
}
__device__ __noinline__ float emu_inject_accum(const EmuParams& p, int64_t gi, int64_t gj, int g, float x) {
  for (int e = 0; e < p.inj.n; ++e) {
    const InjectPoint& ip = p.inj.p[e];
    if (ip.i == gi && ip.j == gj && ip.site == kSiteAccum && ip.mode == FT_MODE_BITFLIP && ip.kt == g)
      x = __uint_as_float(__float_as_uint(x) ^ (1u << (ip.bit & 31)));
  }
  return x;
}
__device__ __noinline__ double emu_inject_output(const EmuParams& p, int64_t gi, int64_t gj, double c) {
  for (int e = 0; e < p.inj.n; ++e) {
    const InjectPoint& ip = p.inj.p[e];
    if (ip.i != gi || ip.j != gj || ip.site != kSiteOutput) continue;
    if (ip.mode == FT_MODE_BITFLIP) {
      c = __longlong_as_double(__double_as_longlong(c) ^ (1ll << (ip.bit & 63)));
    } else {
      const double em = scale_pow2(fabs(c), ip.rel_log2);
      c = ip.sign < 0 ? __dadd_rn(c, -em) : __dadd_rn(c, em);
    }
  }
  return c;
}
// Group 0's predicted row checksum with the checksum-site points of row gi applied.
__device__ __noinline__ int64_t emu_inject_checksum(const EmuParams& p, int64_t gi, int n0, int nJ, int64_t P) {
  for (int e = 0; e < p.inj.n; ++e) {
    const InjectPoint& ip = p.inj.p[e];
    if (ip.site != kSiteChecksumRow || ip.i != gi || ip.j < n0 || ip.j >= n0 + nJ) continue;
    const double m = floor(scale_pow2(fabs(static_cast<double>(P)), ip.rel_log2));
    const int64_t add = m < 1.0 ? 1 : static_cast<int64_t>(m);
    P += ip.sign < 0 ? -add : add;
  }
  return P;
}

__device__ __forceinline__ double gamma64(int n) {
  const double nu = __dmul_rn(static_cast<double>(n), 0x1p-53);
  return __ddiv_rn(nu, __dadd_rn(1.0, -nu));
}

// Persistent product kernel: one CTA per SM loops over output tiles and, per tile, over
// the groups g = 0 .. s-1 (the pairs p + q = g one after another in one accumulator).
template <bool FT>
__global__ void __launch_bounds__(ENTHREADS, 1)
    emu_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                    const __grid_constant__ CUtensorMap tmChk, const __grid_constant__ EmuParams p) {
  constexpr int BN = FT ? kEmuBNProt : kEmuBNPlain, CHK = FT ? kEmuChkRows : 0;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  EmuSmem& sm = *reinterpret_cast<EmuSmem*>(smem_raw);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int nk = (p.K + EBKB - 1) / EBKB;
  const int s = p.s;
  const int ntiles = p.nMb * p.nNb;

  if (t == 0) {
    for (int q = 0; q < ESTAGES; ++q) { mbar_init(&sm.full[q], 1); mbar_init(&sm.empty[q], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&sm.tfull[b], 1); mbar_init(&sm.tempty[b], 4); }
    sm.timeout = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    __syncwarp();
    tmem_alloc(&sm.tmem_base, ETMEM_COLS);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sm.tmem_base;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      tma_prefetch_desc(&tmA);
      tma_prefetch_desc(&tmB);
      if (FT) tma_prefetch_desc(&tmChk);
      const uint32_t bytes = (EBM + BN + CHK) * EBKB;
      uint32_t it = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        int mt, nt;
        emu_tile_coords(tile, p.nMb, p.nNb, mt, nt);
        for (int g = 0; g < s && ok; ++g)
          for (int pa = 0; pa <= g && ok; ++pa) {
            const int qb = g - pa;
            const int ya = static_cast<int>(pa * p.m_pad) + mt * EBM;
            const int yb = static_cast<int>(qb * p.n_pad) + nt * BN;
            const int yc = (qb * p.nNb + nt) * CHK;
            for (int kt = 0; kt < nk; ++kt, ++it) {
              const uint32_t st = it % ESTAGES, u = it / ESTAGES;
              if (u > 0 && !mbar_wait_bounded(&sm.empty[st], (u - 1) & 1, p.wait_limit_ns)) {
                sm.timeout = 1;
                ok = false;
                break;
              }
              const uint32_t extra = (g == 0 && p.inj.n > 0) ? emu_stall_bytes(p, mt, nt, kt, nk) : 0u;
              mbar_arrive_expect_tx(&sm.full[st], bytes + extra);
              const int k0 = kt * EBKB;
              tma_load_2d(sm.a[st], &tmA, &sm.full[st], k0, ya);
              tma_load_2d(sm.b[st], &tmB, &sm.full[st], k0, yb);
              if (FT) tma_load_2d(sm.b[st] + BN * EBKB, &tmChk, &sm.full[st], k0, yc);
            }
          }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issue
    if (lane == 0) {
      const uint32_t idesc = umma_idesc(0u, 0u, EBM, EBNM);  // kind::f8f6f4, E4M3 x E4M3 -> F32
      // A ragged last column block runs narrower MMAs: N1 over its data columns (rounded up
      // to 16) and, protected, N = 16 over stage rows 240..255 (ending with the checksum
      // rows; the data rows among them beyond N are zero-filled by TMA).
      const int nJ_last = p.N - (p.nNb - 1) * BN;
      const int n1_last = (nJ_last + 15) / 16 * 16;
      const bool narrow_last = n1_last + (FT ? 16 : 0) < EBNM;
      const uint32_t idesc_n1 = umma_idesc(0u, 0u, EBM, narrow_last ? n1_last : EBNM);
      const uint32_t idesc_chk = umma_idesc(0u, 0u, EBM, 16);
      uint32_t it = 0, lg = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        int mt, nt;
        emu_tile_coords(tile, p.nMb, p.nNb, mt, nt);
        const bool narrow = narrow_last && nt == p.nNb - 1;
        for (int g = 0; g < s && ok; ++g, ++lg) {
          const uint32_t b = lg & 1, ub = lg >> 1;
          if (ub > 0 && !mbar_wait_bounded(&sm.tempty[b], (ub - 1) & 1, p.wait_limit_ns)) {
            sm.timeout = 1;
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t dcol = tmem + b * EBNM;
          for (int pa = 0; pa <= g && ok; ++pa)
            for (int kt = 0; kt < nk; ++kt, ++it) {
              const uint32_t st = it % ESTAGES, u = it / ESTAGES;
              if (!mbar_wait_bounded(&sm.full[st], u & 1, p.wait_limit_ns)) {
                sm.timeout = 1;
                ok = false;
                break;
              }
              tc_fence_after();
              const uint32_t a0 = smem_addr(sm.a[st]), b0 = smem_addr(sm.b[st]);
#pragma unroll
              for (int kk = 0; kk < EBKB / 32; ++kk) {
                const uint32_t accum = (pa > 0 || kt > 0 || kk > 0) ? 1u : 0u;
                const uint64_t ad = umma_desc_sw128(a0 + kk * 32), bd = umma_desc_sw128(b0 + kk * 32);
                umma_f8(dcol, ad, bd, narrow ? idesc_n1 : idesc, accum);
                if (FT && narrow)
                  umma_f8(dcol + (EBNM - 16), ad, umma_desc_sw128(b0 + (EBNM - 16) * EBKB + kk * 32), idesc_chk, accum);
              }
              umma_commit(&sm.empty[st]);
            }
          // a wait gave up: the group is incomplete and is never handed to the epilogue
          if (!ok) break;
          umma_commit(&sm.tfull[b]);
        }
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue (warps 2..5)
    const int q = warp & 3;
    const int row = q * 32 + lane;
    const int et = t - 64;
    const bool beta_nz = p.beta != 0.0;
    const int shift = -4 * (s + 1);
    // running sums of the groups, per element: H over groups [0, gs), L over [gs, s), both
    // in 64 bits (|H|, |L| < 2^31 16^8 16/15 < 2^63 even for saturated values), so that
    // S = H 16^(s - gs) + L; the output value replaces L after the last group
    const int gs = s / 2;
    int64_t* scrH = p.scratch + static_cast<int64_t>(blockIdx.x) * 2 * BN * EBM;
    int64_t* scr = scrH + BN * EBM;
    uint32_t lg = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
      int mt, nt;
      emu_tile_coords(tile, p.nMb, p.nNb, mt, nt);
      const int m0 = mt * EBM, n0 = nt * BN;
      const int nI = min(EBM, p.M - m0), nJ = min(BN, p.N - n0);
      const int64_t gi = m0 + row;
      const bool row_ok = row < nI;
      const int erow = (row_ok && p.erow[gi] > kExpNone) ? p.erow[gi] : 0;
      const bool rbad = row_ok && p.row_bad[gi];
      bool flagged = false, got_all = true;
      double fdelta = 0.0, ftau = 0.0;
      for (int g = 0; g < s; ++g, ++lg) {
        const uint32_t b = lg & 1, ub = lg >> 1;
        const bool last = g == s - 1;
        // tcgen05.ld is warp-collective: `got` is warp-uniform, and every TMEM load below is
        // executed by all 32 lanes whatever their row. After one wait has given up, later
        // waits are not attempted.
        bool got = *reinterpret_cast<volatile int*>(&sm.timeout) == 0 &&
                   mbar_wait_bounded(&sm.tfull[b], ub & 1, p.wait_limit_ns);
        got = __all_sync(0xffffffffu, got);
        if (!got) { sm.timeout = 1; got_all = false; }
        tc_fence_after();
        const uint32_t trow = tmem + b * EBNM + (static_cast<uint32_t>(q * 32) << 16);
        int64_t R = 0;
        bool invalid = false;
        double V = 0.0, aV = 0.0, Q = 0.0, aQ = 0.0, RC = 0.0, aC = 0.0;
        int inj_c = INT_MAX;
        if (FT && p.inj.n > 0) inj_c = emu_next_inj_col(p, gi, g, n0, nJ, -1);
        if (got) {
          const int nch = (nJ + 7) / 8;
#pragma unroll 1
          for (int ch = 0; ch < nch; ++ch) {
            uint32_t v[8];
            __syncwarp();
            tmem_ld8(trow + ch * 8, v);
            tmem_ld_wait();
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int col = ch * 8 + j;
              if (!row_ok || col >= nJ) continue;
              const int64_t gj = n0 + col;
              float G = __uint_as_float(v[j]);
              const bool at_point = FT && col == inj_c;
              if (at_point) G = emu_inject_accum(p, gi, gj, g, G);
              if (FT) invalid |= !(fabsf(G) <= 16777216.0f && G == rintf(G));
              const int gv = __float2int_rn(G);
              R += gv;
              const int64_t e = static_cast<int64_t>(col) * EBM + row;
              int64_t* slot = (g < gs ? scrH : scr) + e;
              const int64_t X = (g == 0 || g == gs) ? static_cast<int64_t>(gv)
                                                    : static_cast<int64_t>(static_cast<uint64_t>(*slot) << 4) + gv;
              if (!last) {
                *slot = X;
              } else {
                const __int128 S = (static_cast<__int128>(scrH[e]) << (4 * (s - gs))) + X;
                double vv;
                if (rbad || p.col_bad[gj]) vv = __longlong_as_double(0x7ff8000000000000ll);
                else vv = scale_pow2(i128_to_f64(S), erow + p.fcol[gj] + shift);
                const double cin = beta_nz ? p.C[gi + gj * p.ldc] : 0.0;
                double c = __dmul_rn(p.alpha, vv);
                if (beta_nz) c = __dadd_rn(c, __dmul_rn(p.beta, cin));
                if (at_point) c = emu_inject_output(p, gi, gj, c);
                if (FT) {
                  V = __dadd_rn(V, vv); aV = __dadd_rn(aV, fabs(vv));
                  if (beta_nz) { Q = __dadd_rn(Q, cin); aQ = __dadd_rn(aQ, fabs(cin)); }
                  RC = __dadd_rn(RC, c); aC = __dadd_rn(aC, fabs(c));
                  *reinterpret_cast<double*>(slot) = c;  // stored after the tile's checks
                } else {
                  p.C[gi + gj * p.ldc] = c;
                }
              }
              if (at_point) inj_c = emu_next_inj_col(p, gi, g, n0, nJ, col);
            }
          }
          if (FT) {  // group g's predicted row checksum: the four digit columns
            uint32_t vc[8];
            __syncwarp();
            tmem_ld8(trow + BN, vc);
            tmem_ld_wait();
            int64_t P = 0;
#pragma unroll
            for (int d = 0; d < kEmuDigits; ++d)
              P += static_cast<int64_t>(__float2int_rn(__uint_as_float(vc[d]))) << (4 * d);
            if (g == 0 && p.inj.n > 0) P = emu_inject_checksum(p, gi, n0, nJ, P);
            if (row_ok && !flagged && (invalid || R != P)) {
              flagged = true;
              fdelta = static_cast<double>(R - P);
              ftau = 0.0;
            }
          }
        }
        // the accumulator buffer is free for the MMA warp's next-but-one group
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sm.tempty[b]);
        if (FT && last && got && row_ok) {  // the binary64 stage's check
          double Pi = __dmul_rn(p.alpha, V);
          if (beta_nz) Pi = __dadd_rn(Pi, __dmul_rn(p.beta, Q));
          const double tauC = __dmul_rn(__dmul_rn(2.0, gamma64(nJ + 2)),
                                        __dadd_rn(__dadd_rn(__dmul_rn(fabs(p.alpha), aV), __dmul_rn(fabs(p.beta), aQ)), aC));
          const double d = __dadd_rn(RC, -Pi);
          if (!flagged && (!(fabs(d) <= tauC) || isinf(d))) {
            flagged = true;
            fdelta = d;
            ftau = tauC;
          }
        }
      }
      if (!FT) continue;

      // ---------------------------------------------------------- tile classification
      // tile_ok is made uniform over the 128 epilogue threads through shared memory (a
      // warp-local result would split them on the branches below, which hold barriers)
      named_bar(1, 128);
      if (et == 0) { sm.nflag = 0; sm.first_row = INT_MAX; sm.tile_ok = 1; }
      named_bar(1, 128);
      if (!got_all) sm.tile_ok = 0;
      named_bar(1, 128);
      const bool tile_ok = sm.tile_ok != 0;
      const bool tile_bad = p.rowblk_bad[mt] || p.colblk_bad[nt];
      int sub = -1;
      if (tile_ok && !tile_bad && flagged) {
        sub = atomicAdd(&sm.nflag, 1);
        atomicMin(&sm.first_row, row);
      }
      named_bar(1, 128);
      const int nf = sm.nflag;
      if (flagged && row == sm.first_row) { sm.first_delta = fdelta; sm.first_tau = ftau; }
      named_bar(1, 128);
      bool defer = false;
      if (tile_ok && !tile_bad && nf > 0) {
        if (nf <= kEmuPendRows) {
          // flagged rows are not stored: the resolve pass recomputes and stores them
          if (et == 0) sm.pend_slot = static_cast<int>(atomicAdd(&p.pend->count, 1u));
          named_bar(1, 128);
          const int slot = sm.pend_slot;
          if (slot < kEmuPendCap) {
            EmuPendEntry& pe = p.pend->e[slot];
            if (et == 0) { pe.mt = mt; pe.nt = nt; pe.nrows = nf; pe.first_row = sm.first_row; pe.done = 0u; }
            if (sub >= 0) {
              EmuPendRow& pr = pe.r[sub];
              pr.row = row;
              pr.delta = fdelta;
              pr.tau = ftau;
              for (int col = 0; col < nJ; ++col)
                pr.c_computed[col] = *reinterpret_cast<const double*>(scr + static_cast<int64_t>(col) * EBM + row);
              defer = true;
            }
          } else if (et == 0) {  // more flagged tiles in this call than the resolve pass holds
            emu_record(p, FT_KIND_UNCORRECTABLE, mt, nt, m0 + sm.first_row, -1, sm.first_delta, sm.first_tau, 0.0, 0.0,
                       nf, 0);
            emu_count(p, &ft_report_t::detected);
            emu_count(p, &ft_report_t::uncorrectable);
          }
        } else if (et == 0) {  // more flagged rows than the resolve pass recomputes: C as computed
          emu_record(p, FT_KIND_UNCORRECTABLE, mt, nt, m0 + sm.first_row, -1, sm.first_delta, sm.first_tau, 0.0, 0.0,
                     nf, 0);
          emu_count(p, &ft_report_t::detected);
          emu_count(p, &ft_report_t::uncorrectable);
        }
      }
      if (tile_ok && tile_bad && et == 0) {
        emu_record(p, FT_KIND_INPUT_NONFINITE, mt, nt, -1, -1, 0.0, 0.0, 0.0, 0.0, 0, 0);
        emu_count(p, &ft_report_t::input_nonfinite);
      }
      if (tile_ok && row_ok && !defer)
        for (int col = 0; col < nJ; ++col)
          p.C[gi + static_cast<int64_t>(n0 + col) * p.ldc] =
              *reinterpret_cast<const double*>(scr + static_cast<int64_t>(col) * EBM + row);
      if (tile_ok && et == 0) emu_count(p, &ft_report_t::tiles_checked);
      named_bar(1, 128);  // the scratch and the shared state are free for the next tile
    }
  }

  // ------------------------------------------------------------ teardown
  tc_fence_before();
  __syncthreads();
  if (t == 0 && sm.timeout && p.report) atomicOr(&p.report->status, FT_STATUS_TIMEOUT);
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, ETMEM_COLS);
  }
}

// ---------------------------------------------------------------------------------------
// Resolve pass: each flagged row of each pending tile is recomputed exactly from the slices
// (its groups, S, v and C as in the product kernel) and stored; elements whose computed
// value differed are the located errors. Work item = (tile, flagged row, 8 columns); warp
// w takes column 8 g + w, its lanes split K. The CTA finishing a tile's last item
// classifies the tile and writes its records.
// ---------------------------------------------------------------------------------------
constexpr int kEmuColGroups = (kEmuBNProt + 7) / 8;   // 31
constexpr int kEmuItemsPerTile = kEmuPendRows * kEmuColGroups;

__global__ void __launch_bounds__(256) emu_resolve_kernel(const __grid_constant__ EmuParams p) {
  __shared__ int dec[256];
  __shared__ int last;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  dec[threadIdx.x] = int_of_e4m3(threadIdx.x);
  __syncthreads();
  const unsigned npend = min(*reinterpret_cast<volatile const unsigned*>(&p.pend->count), (unsigned)kEmuPendCap);
  const int items = static_cast<int>(npend) * kEmuItemsPerTile;
  const int s = p.s;
  const int shift = -4 * (s + 1);
  const bool beta_nz = p.beta != 0.0;
  const int64_t aslice = p.m_pad * p.kpitch, bslice = p.n_pad * p.kpitch;
  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    EmuPendEntry& pe = p.pend->e[item / kEmuItemsPerTile];
    const int rem = item % kEmuItemsPerTile;
    const int sub = rem / kEmuColGroups, col = (rem % kEmuColGroups) * 8 + warp;
    const int m0 = pe.mt * EBM, n0 = pe.nt * kEmuBNProt;
    const int nJ = min(kEmuBNProt, p.N - n0);
    if (sub < pe.nrows && col < nJ) {
      EmuPendRow& pr = pe.r[sub];
      const int64_t gi = m0 + pr.row, gj = n0 + col;
      const uint8_t* arow = p.aslices + gi * p.kpitch;
      const uint8_t* bcol = p.bslices + gj * p.kpitch;
      int G[kEmuSlicesMax];
#pragma unroll
      for (int g = 0; g < kEmuSlicesMax; ++g) G[g] = 0;
      for (int64_t k = 4 * lane; k < p.kpitch; k += 128) {
        uint32_t aw[kEmuSlicesMax], bw[kEmuSlicesMax];
        for (int x = 0; x < s; ++x) {
          aw[x] = *reinterpret_cast<const uint32_t*>(arow + x * aslice + k);
          bw[x] = *reinterpret_cast<const uint32_t*>(bcol + x * bslice + k);
        }
        for (int by = 0; by < 4; ++by) {
          int bv[kEmuSlicesMax];
          for (int x = 0; x < s; ++x) bv[x] = dec[(bw[x] >> (8 * by)) & 0xffu];
          for (int pa = 0; pa < s; ++pa) {
            const int av = dec[(aw[pa] >> (8 * by)) & 0xffu];
            for (int qb = 0; qb < s - pa; ++qb) G[pa + qb] += av * bv[qb];
          }
        }
      }
      __int128 S = 0;
      for (int g = 0; g < s; ++g) S = S * 16 + __reduce_add_sync(0xffffffffu, G[g]);
      if (lane == 0) {
        const double vv = scale_pow2(i128_to_f64(S), (p.erow[gi] > kExpNone ? p.erow[gi] : 0) + p.fcol[gj] + shift);
        double c = __dmul_rn(p.alpha, vv);
        if (beta_nz) c = __dadd_rn(c, __dmul_rn(p.beta, p.C[gi + gj * p.ldc]));  // the row was not stored: C_in
        pr.c_true[col] = c;
        pr.differs[col] = __double_as_longlong(c) != __double_as_longlong(pr.c_computed[col]) ? 1 : 0;
        p.C[gi + gj * p.ldc] = c;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      last = (atomicAdd(&pe.done, 1u) == static_cast<unsigned>(kEmuItemsPerTile - 1)) ? 1 : 0;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
      __threadfence();
      int located = 0;
      for (int r = 0; r < pe.nrows; ++r)
        for (int c = 0; c < nJ; ++c) located += __ldcg(&pe.r[r].differs[c]);
      emu_count(p, &ft_report_t::detected);
      if (located > 0) {
        emu_count(p, &ft_report_t::corrected);
        for (int r = 0; r < pe.nrows; ++r)
          for (int c = 0; c < nJ; ++c)
            if (__ldcg(&pe.r[r].differs[c]))
              emu_record(p, FT_KIND_CORRECTED, pe.mt, pe.nt, m0 + pe.r[r].row, n0 + c, pe.r[r].delta, pe.r[r].tau,
                         __ldcg(&pe.r[r].c_computed[c]), __ldcg(&pe.r[r].c_true[c]), pe.nrows, located);
      } else {
        emu_count(p, &ft_report_t::checksum_only);
        int fr = 0;
        for (int r = 0; r < pe.nrows; ++r)
          if (pe.r[r].row == pe.first_row) fr = r;
        emu_record(p, FT_KIND_CHECKSUM_ONLY, pe.mt, pe.nt, m0 + pe.first_row, -1, pe.r[fr].delta, pe.r[fr].tau, 0.0,
                   0.0, pe.nrows, 0);
      }
    }
    __syncthreads();
  }
}

}  // namespace

// ---------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------
namespace {
constexpr size_t kAlign = 256;
size_t up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

struct EmuLayout {
  size_t a, b, chk, erow, fcol, row_bad, col_bad, rowblk, colblk, scratch, pend, total;
};
EmuLayout emu_layout(const EmuParams& p, int grid, bool ft) {
  EmuLayout L;
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t at = off; off += up(bytes); return at; };
  L.a = take(static_cast<size_t>(p.s) * p.m_pad * p.kpitch);
  L.b = take(static_cast<size_t>(p.s) * p.n_pad * p.kpitch);
  L.chk = take(ft ? static_cast<size_t>(p.s) * p.nNb * kEmuChkRows * p.kpitch : 0);
  L.erow = take(sizeof(int32_t) * p.m_pad);
  L.fcol = take(sizeof(int32_t) * p.n_pad);
  L.row_bad = take(p.m_pad);
  L.col_bad = take(p.n_pad);
  L.rowblk = take(p.nMb);
  L.colblk = take(p.nNb);
  L.scratch = take(2 * sizeof(int64_t) * static_cast<size_t>(grid) * p.bn * EBM);
  L.pend = take(ft ? sizeof(EmuPending) : 0);
  L.total = off;
  return L;
}
}  // namespace

size_t emu_workspace_bytes(const EmuParams& p, int grid) { return emu_layout(p, grid, p.bn == kEmuBNProt).total; }

void emu_workspace_carve(EmuParams& p, void* ws, int grid, uint8_t** chk_out) {
  const bool ft = p.bn == kEmuBNProt;
  const EmuLayout L = emu_layout(p, grid, ft);
  uint8_t* base = static_cast<uint8_t*>(ws);
  p.aslices = base + L.a;
  p.bslices = base + L.b;
  *chk_out = ft ? base + L.chk : nullptr;
  p.erow = reinterpret_cast<const int32_t*>(base + L.erow);
  p.fcol = reinterpret_cast<const int32_t*>(base + L.fcol);
  p.row_bad = base + L.row_bad;
  p.col_bad = base + L.col_bad;
  p.rowblk_bad = base + L.rowblk;
  p.colblk_bad = base + L.colblk;
  p.scratch = reinterpret_cast<int64_t*>(base + L.scratch);
  p.pend = ft ? reinterpret_cast<EmuPending*>(base + L.pend) : nullptr;
}

cudaError_t launch_emu_split(const EmuParams& p, const EmuSource& a, const EmuSource& b, uint8_t* chk, bool ft,
                             cudaStream_t st) {
  int32_t* erow = const_cast<int32_t*>(p.erow);
  int32_t* fcol = const_cast<int32_t*>(p.fcol);
  uint8_t* row_bad = const_cast<uint8_t*>(p.row_bad);
  uint8_t* col_bad = const_cast<uint8_t*>(p.col_bad);
  uint8_t* rowblk = const_cast<uint8_t*>(p.rowblk_bad);
  uint8_t* colblk = const_cast<uint8_t*>(p.colblk_bad);
  // exponents start below every exponent of a finite nonzero value (bytes 0x80: -2139062144)
  cudaError_t e = cudaMemsetAsync(erow, 0x80, sizeof(int32_t) * p.m_pad, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(fcol, 0x80, sizeof(int32_t) * p.n_pad, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(row_bad, 0, p.m_pad, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(col_bad, 0, p.n_pad, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(rowblk, 0, p.nMb, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(colblk, 0, p.nNb, st);
  if (ft && e == cudaSuccess) e = cudaMemsetAsync(p.pend, 0, 256, st);  // the pending count
  if (e != cudaSuccess) return e;
  const unsigned kchunks = static_cast<unsigned>((p.K + kExpChunk - 1) / kExpChunk);
  auto exps = [&](const EmuSource& src, int32_t* ex, uint8_t* bad, uint8_t* blk, int blk_lines) {
    if (src.ks == 1) {
      emu_exp_kernel<true><<<dim3(static_cast<unsigned>((src.R + 7) / 8), kchunks), 256, 0, st>>>(src, p.K, ex, bad,
                                                                                                  blk, blk_lines);
    } else {
      emu_exp_kernel<false><<<dim3(static_cast<unsigned>((src.R + 31) / 32), kchunks), 256, 0, st>>>(src, p.K, ex, bad,
                                                                                                     blk, blk_lines);
    }
  };
  exps(a, erow, row_bad, rowblk, EBM);
  exps(b, fcol, col_bad, colblk, p.bn);
  const unsigned kt = static_cast<unsigned>((p.kpitch + kSliceK - 1) / kSliceK);
  auto slices = [&](const EmuSource& src, int64_t R_pad, const int32_t* ex, const uint8_t* bad, const uint8_t* out) {
    const dim3 grid(static_cast<unsigned>((R_pad + kSliceRows - 1) / kSliceRows), kt);
    if (src.ks == 1)
      emu_slice_kernel<true><<<grid, 256, 0, st>>>(src, p.K, R_pad, p.kpitch, p.s, ex, bad, const_cast<uint8_t*>(out));
    else
      emu_slice_kernel<false><<<grid, 256, 0, st>>>(src, p.K, R_pad, p.kpitch, p.s, ex, bad, const_cast<uint8_t*>(out));
  };
  slices(a, p.m_pad, erow, row_bad, p.aslices);
  slices(b, p.n_pad, fcol, col_bad, p.bslices);
  if (ft) {
    const dim3 grid(static_cast<unsigned>((p.kpitch / 4 + 255) / 256), static_cast<unsigned>(p.nNb),
                    static_cast<unsigned>(p.s));
    emu_digit_kernel<<<grid, 256, 0, st>>>(p.bslices, p.n_pad, p.kpitch, p.bn, p.nNb, chk);
  }
  return cudaGetLastError();
}

cudaError_t launch_emu_gemm(const EmuParams& p, const CUtensorMap* tmA, const CUtensorMap* tmB,
                            const CUtensorMap* tmChk, bool ft, int grid, cudaStream_t st) {
  const size_t smem = sizeof(EmuSmem);
  cudaError_t e = ft ? cudaFuncSetAttribute(emu_gemm_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                     : cudaFuncSetAttribute(emu_gemm_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kernel_timer_start(st);
  if (ft) emu_gemm_kernel<true><<<grid, ENTHREADS, smem, st>>>(*tmA, *tmB, *tmChk, p);
  else emu_gemm_kernel<false><<<grid, ENTHREADS, smem, st>>>(*tmA, *tmB, *tmA, p);
  kernel_timer_stop(st);
  e = cudaGetLastError();
  if (e != cudaSuccess || !ft) return e;
  int dev = 0, sms = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  emu_resolve_kernel<<<2 * sms, 256, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_emu_convert(const int64_t* words, double* out, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  emu_convert_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, st>>>(words, out, n);
  return cudaGetLastError();
}

}  // namespace ftk
