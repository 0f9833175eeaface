// Reduced-precision ABFT-protected GEMM on the fifth-generation tensor cores (sm_103a):
// BF16 or FP8 E4M3 operands, FP32 accumulation in TMEM, FP32 output (or bfloat16, rounded
// once from the verified FP32 value), FP64 checksum comparison.
//
// FT-BLAS (Zhai et al., ICS '21) has no reduced precision; the checksum relations are those
// of Section II.A, the lazy second side that of Section V.A, and C = beta*C is folded into
// the checksums as in Section V.B.
//
// Structure (persistent: one CTA of 192 threads per SM loops over output tiles; the
// tensor-core tile is 128 x 256 and the TMEM accumulator is double-buffered):
//   warp 0      TMA producer: A (128 x 64) and B (N_data x 64) k-tiles into a 4-stage ring,
//               128-byte swizzled, K-major. Protected launches put the checksum column of
//               B^r = [B, Be] (Section II.A) into the last rows of the same B stage: Be over
//               the tile's data columns, in pieces written by a bandwidth-bound encode
//               pre-pass (ft_tc_encode.cu): 248 data columns and, in rows 248..255, three
//               bfloat16 pieces (hi, mid, lo) of B e, or eight e4m3 pieces.
//   warp 1      TMEM allocation and MMA issue (one thread): 4 x tcgen05.mma M128 N256 K16 per
//               k-tile into one of two 256-column TMEM buffers, so the next tile's product
//               overlaps the previous tile's epilogue. With the checksum column appended, the
//               tensor core produces the pieces of C^r = A (B e) in the last columns with the
//               product itself, at no extra instruction (8 of 256 columns per tile).
//   warps 2..5  epilogue, one TMEM lane (= output row) per thread: C = alpha acc + beta C_in
//               stored in FP32; C^r_ref(i) = sum_j C(i,j) in compensated binary32, compared
//               in binary64 with the predicted checksum against a rigorous bound. A tile
//               with a mismatching row is entered in a pending list.
// After the GEMM, tc_resolve_kernel takes the pending tiles (the lazy second side): it forms
// their column checksums (C^c_ref from the stored tile, C^c = (e^T A) B from global memory
// in binary32) to locate the error. When the columns cannot locate it (rows of very
// different scale), it recomputes the mismatching row and compares element by element. The
// located element is corrected from the row checksum.
//
// Two forms of the product kernel share this structure: tc_gemm_kernel, one CTA per 128-row
// tile as above, and tc_gemm_pair_kernel, a CTA pair (cta_group::2) per 256-row unit with
// each CTA staging its own 128 rows of A and half of B^r in a 6-stage ring, so that a CTA's
// shared-memory traffic per MMA carries half the B operand. Both verify, hand over and
// correct per 128 x BN tile. ftblas_set_tc_cta_group selects the form.
#include <climits>
#include <cstring>

#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "ft_device.cuh"
#include "ft_pair.cuh"
#include "ft_internal.h"
#include "ft_tc.h"
#include "ft_tc_elem.cuh"

namespace ftk {

namespace {

constexpr int BM = kTcBM;            // 128 tile rows (TMEM lanes)
constexpr int BNM = 256;             // MMA N = TMEM columns of one accumulator buffer
constexpr int BKB = 128;             // k-tile depth in bytes (64 BF16 or 128 E4M3)
constexpr int NTHREADS = 192;
constexpr uint32_t TMEM_COLS = 512;   // two accumulator buffers of 256 columns

template <bool FT, int KIND>
struct TcGeom {
  static constexpr int BN = FT ? tc_bn_prot(KIND) : BNM;  // data columns per tile
  static constexpr int CHK = FT ? tc_chk_rows(KIND) : 0;  // checksum rows after them in a B stage
};

// Staging of one CTA. CG = 1: a CTA per 128-row tile, B stages of 256 rows, 4 stages.
// CG = 2: a CTA pair per 256-row unit (cta_group::2); each CTA stages its own 128 rows of A
// and half of B^r (128 rows), 6 stages in the same shared memory.
template <int CG>
struct TcStage {
  static constexpr int kStages = CG == 2 ? 6 : 4;
  static constexpr int kBRows = BNM / CG;
};

template <int CG>
struct __align__(1024) TcSmem {
  uint8_t a[TcStage<CG>::kStages][BM * BKB];
  uint8_t b[TcStage<CG>::kStages][TcStage<CG>::kBRows * BKB];
  uint64_t full[TcStage<CG>::kStages];
  uint64_t empty[TcStage<CG>::kStages];
  uint64_t tfull[2];             // accumulator buffer b holds a finished tile
  uint64_t tempty[2];            // accumulator buffer b has been read by the epilogue warps (of both CTAs)
  uint32_t tmem_base;
  int timeout;
  int nflag_rows, first_row, pend_slot;
  double delta_row, tau_row;
  double pred_row;               // predicted row checksum of the first flagged row
  float cin_col[4][BNM];         // per-warp partial column sums of C_in (beta != 0)
  float cin_col_abs[4][BNM];
};

// MMA shape of a CTA-pair unit whose column block holds nJ data columns. D columns [0, n/2)
// come from the even CTA's B stage rows [0, n/2), D columns [n/2, n) from the odd CTA's.
//   protected, nJ > 120:  n = 256; the even CTA stages data columns 0..127, the odd one
//                         columns 128..247 in rows 0..119 and the checksum rows in 120..127
//                         (D columns 248..255);
//   protected, nJ <= 120 (a ragged last column block): n = 2h, h = nJ rounded up to 8; the
//                         even CTA stages the data columns, the odd one only the checksum rows,
//                         in rows 0..7 (D columns h..h+7; D columns h+8..2h are not used);
//   unprotected:          n = nJ rounded up to 16 (256 for a full block); the odd CTA stages
//                         data columns n/2.. .
struct PairShape {
  int n;        // MMA N
  int chk_col;  // first D column of the checksum pieces (protected)
  int b1_row;   // first data column staged by the odd CTA
  bool b1_data; // the odd CTA stages data columns
};
template <bool FT>
__device__ __forceinline__ PairShape pair_shape(int nJ) {
  PairShape g;
  if (FT) {
    if (nJ <= 120) {
      const int h = (nJ + 7) / 8 * 8;
      g.n = 2 * h; g.chk_col = h; g.b1_row = 0; g.b1_data = false;
    } else {
      g.n = BNM; g.chk_col = BNM - 8; g.b1_row = BNM / 2; g.b1_data = true;
    }
  } else {
    g.n = nJ >= BNM ? BNM : (nJ + 15) / 16 * 16;
    g.chk_col = 0; g.b1_row = g.n / 2; g.b1_data = true;
  }
  return g;
}

// alpha times the per-tensor scales of FP8 operands (device values; absent scales are 1)
__device__ __forceinline__ float alpha_eff(const TcParams& p) {
  float a = p.alpha;
  if (p.a_scale != nullptr) a *= *p.a_scale;
  if (p.b_scale != nullptr) a *= *p.b_scale;
  return a;
}

// Neumaier's compensated summation step (binary32).
__device__ __forceinline__ void neumaier(float& s, float& c, float x) {
  const float t = s + x;
  c += (fabsf(s) >= fabsf(x)) ? ((s - t) + x) : ((x - t) + s);
  s = t;
}

__device__ __forceinline__ double warp_sum_f64(double x) {
#pragma unroll
  for (int w = 16; w >= 1; w >>= 1) x += __shfl_xor_sync(0xffffffffu, x, w);
  return x;
}
__device__ __forceinline__ float warp_sum_up(float x) {
#pragma unroll
  for (int w = 16; w >= 1; w >>= 1) x = __fadd_ru(x, __shfl_xor_sync(0xffffffffu, x, w));
  return x;
}

__device__ __forceinline__ float warp_sum_plain(float x) {
#pragma unroll
  for (int w = 16; w >= 1; w >>= 1) x += __shfl_xor_sync(0xffffffffu, x, w);
  return x;
}

// alpha * acc + beta * C_in with the accumulator- and output-site injections of the current
// plan applied (test launches only; kept out of line).
__device__ __noinline__ float inject_element(const TcParams& p, float alpha, int64_t gi, int64_t gj, float acc,
                                             float cin, bool beta_nz) {
  for (int e = 0; e < p.inj.n; ++e) {
    const InjectPoint& ip = p.inj.p[e];
    if (ip.i == gi && ip.j == gj && ip.site == kSiteAccum && ip.mode == FT_MODE_BITFLIP)
      acc = __uint_as_float(__float_as_uint(acc) ^ (1u << ip.bit));
  }
  float out = beta_nz ? fmaf(alpha, acc, p.beta * cin) : alpha * acc;
  for (int e = 0; e < p.inj.n; ++e) {
    const InjectPoint& ip = p.inj.p[e];
    if (ip.i != gi || ip.j != gj || ip.site != kSiteOutput) continue;
    if (ip.mode == FT_MODE_BITFLIP) {
      out = __uint_as_float(__float_as_uint(out) ^ (1u << ip.bit));
    } else {
      const float em = ldexpf(fabsf(out), ip.rel_log2);
      out = ip.sign < 0 ? out - em : out + em;
    }
  }
  return out;
}

// Smallest tile column > after (tile-local) where row gi holds an accumulator- or output-site
// injection point, INT_MAX if none (test launches only; kept out of line).
__device__ __noinline__ int next_inj_col(const TcParams& p, int64_t gi, int n0, int nJ, int after) {
  int best = INT_MAX;
  for (int e = 0; e < p.inj.n; ++e) {
    const InjectPoint& ip = p.inj.p[e];
    if (ip.i != gi || (ip.site != kSiteAccum && ip.site != kSiteOutput)) continue;
    const int c = ip.j - n0;
    if (c > after && c < nJ && c < best) best = c;
  }
  return best;
}

__device__ __forceinline__ float gamma32_up(float n, float u) {
  const float nu = __fmul_ru(n, u);
  return __fdiv_ru(nu, __fsub_rd(1.0f, nu));
}

__device__ void tc_record(const TcParams& p, int kind, int64_t tr, int64_t tc, int64_t i, int64_t j, double drow,
                          double dcol, double trow, double tcol, double before, double after, int nr, int nc) {
  if (p.report == nullptr) return;
  const unsigned slot = atomicAdd(&p.report->n_records, 1u);
  if (slot >= FTBLAS_MAX_RECORDS) {
    atomicOr(&p.report->status, FT_STATUS_RECORDS_TRUNCATED);
    return;
  }
  ft_error_record_t& r = p.report->rec[slot];
  if (p.swap_report) {
    r.tile_row = tc; r.tile_col = tr; r.i = j; r.j = i;
    r.delta_row = dcol; r.delta_col = drow; r.tau_row = tcol; r.tau_col = trow;
    r.rows_flagged = nc; r.cols_flagged = nr;
  } else {
    r.tile_row = tr; r.tile_col = tc; r.i = i; r.j = j;
    r.delta_row = drow; r.delta_col = dcol; r.tau_row = trow; r.tau_col = tcol;
    r.rows_flagged = nr; r.cols_flagged = nc;
  }
  r.value_before = before;
  r.value_after = after;
  r.kind = kind;
  r.reserved = 0;
}

__device__ void count_kind(const TcParams& p, int kind) {
  if (p.report == nullptr) return;
  atomicAdd(reinterpret_cast<unsigned long long*>(&p.report->detected), 1ull);
  unsigned long long* ctr = (kind == FT_KIND_CORRECTED)
                                ? reinterpret_cast<unsigned long long*>(&p.report->corrected)
                            : (kind == FT_KIND_CHECKSUM_ONLY)
                                ? reinterpret_cast<unsigned long long*>(&p.report->checksum_only)
                                : reinterpret_cast<unsigned long long*>(&p.report->uncorrectable);
  atomicAdd(ctr, 1ull);
}

// Bytes beyond the stage's that the staging barrier of k-tile kt of unit (mu, nt) expects
// (a unit: `rows` rows, one tile or the two tiles of a CTA pair): 16 when a stall point (test
// launches only) names a tile of that unit and k-tile (0: the middle one), so that the barrier
// never completes and the waits on it give up; else 0.
__device__ __forceinline__ uint32_t stall_bytes(const TcParams& p, int mu, int rows, int nt, int kt, int nk, int bn) {
  for (int e = 0; e < p.inj.n; ++e) {
    const InjectPoint& ip = p.inj.p[e];
    if (ip.site == kSiteStall && kt == (ip.kt > 0 ? ip.kt : nk / 2) && ip.i / rows == mu && ip.j / bn == nt)
      return 16u;
  }
  return 0u;
}

// The k-tile of unit (mu, nt) at which a stall point (test launches only) makes the staging
// barrier expect 16 bytes more than arrive, as stall_bytes does, formed once per unit: the
// earliest k-tile named for the unit, or -1. It keeps the per-k-tile work of the producer
// thread at one comparison when injection is on.
__device__ __forceinline__ int stall_ktile(const TcParams& p, int mu, int rows, int nt, int nk, int bn) {
  int kt_min = -1;
  for (int e = 0; e < p.inj.n; ++e) {
    const InjectPoint& ip = p.inj.p[e];
    if (ip.site != kSiteStall || ip.i / rows != mu || ip.j / bn != nt) continue;
    const int kt = ip.kt > 0 ? ip.kt : nk / 2;
    if (kt_min < 0 || kt < kt_min) kt_min = kt;
  }
  return kt_min;
}

// Persistent order of the units (row unit mu, column block nt): groups of kGroupRows rows
// sweep the column blocks, so the CTAs resident at one time share A row panels and B column
// panels in L2. The last column block comes after all the others: when N is not a multiple
// of the tile width its units are narrower and cheaper (narrow MMAs), and placed last they
// fill the final round of the persistent CTAs instead of adding one.
constexpr int kGroupRows = 2048;
__device__ __forceinline__ void tile_coords(int t, int nUb, int nNb, int group_units, int& mu, int& nt) {
  const int ncols = nNb - 1;  // column blocks before the last
  if (t >= nUb * ncols) {
    mu = t - nUb * ncols;
    nt = ncols;
    return;
  }
  const int group = t / (group_units * ncols);
  const int first_m = group * group_units;
  const int gsize = min(group_units, nUb - first_m);
  const int in_group = t - group * group_units * ncols;
  mu = first_m + in_group % gsize;
  nt = in_group / gsize;
}

// Persistent kernel: one CTA per SM loops over output tiles. The TMEM accumulator is double
// buffered (2 x 256 columns): while the epilogue warps verify and store tile t from one
// buffer, the MMA warp accumulates tile t+1 into the other.
template <bool FT, int KIND>
__global__ void __launch_bounds__(NTHREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ CUtensorMap tmChk, const __grid_constant__ TcParams p) {
  constexpr int BN = TcGeom<FT, KIND>::BN, CHK = TcGeom<FT, KIND>::CHK;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  constexpr int STAGES = TcStage<1>::kStages;
  TcSmem<1>& sm = *reinterpret_cast<TcSmem<1>*>(smem_raw);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  using E = Elem<KIND>;
  const int bk_elems = BKB / E::kBytes;
  const int nk = (p.K + bk_elems - 1) / bk_elems;
  const int nMb = (p.M + BM - 1) / BM, nNb = (p.N + BN - 1) / BN;
  const int ntiles = nMb * nNb;

  if (t == 0) {
    for (int s = 0; s < STAGES; ++s) { mbar_init(&sm.full[s], 1); mbar_init(&sm.empty[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&sm.tfull[b], 1); mbar_init(&sm.tempty[b], 4); }
    sm.timeout = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    __syncwarp();
    tmem_alloc(&sm.tmem_base, TMEM_COLS);
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
      const uint32_t bytes = (BM + BN + CHK) * BKB;
      uint32_t it = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        int mt, nt;
        tile_coords(tile, nMb, nNb, kGroupRows / BM, mt, nt);
        for (int kt = 0; kt < nk; ++kt, ++it) {
          const uint32_t s = it % STAGES, u = it / STAGES;
          if (u > 0 && !mbar_wait_bounded(&sm.empty[s], (u - 1) & 1, p.wait_limit_ns)) { sm.timeout = 1; ok = false; break; }
          mbar_arrive_expect_tx(&sm.full[s], bytes + stall_bytes(p, mt, BM, nt, kt, nk, BN));
          const int k0 = kt * bk_elems;
          tma_load_2d(sm.a[s], &tmA, &sm.full[s], k0, mt * BM);
          tma_load_2d(sm.b[s], &tmB, &sm.full[s], k0, nt * BN);
          if (FT) tma_load_2d(sm.b[s] + BN * BKB, &tmChk, &sm.full[s], k0, nt * CHK);
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issue
    if (lane == 0) {
      // kind::f16 with BF16 operands (format 1), or kind::f8f6f4 with E4M3 operands (format 0)
      constexpr uint32_t fmt = KIND == 0 ? 1u : 0u;
      const uint32_t idesc = umma_idesc(fmt, fmt, BM, BNM);
      // A ragged last column block runs narrower MMAs: N1 (its data columns rounded up to 16)
      // over the first stage rows, and, protected, N = 16 over stage rows 240..255, which end
      // with the checksum rows (the data rows among them are beyond N, zero-filled by TMA),
      // into TMEM columns 240..255. The columns in between are left as they were; the
      // epilogue uses only data columns below the tile's width and the checksum columns.
      const int nJ_last = p.N - (nNb - 1) * BN;
      const int n1_last = (nJ_last + 15) / 16 * 16;
      const bool narrow_last = n1_last + (FT ? 16 : 0) < BNM;
      const uint32_t idesc_n1 = umma_idesc(fmt, fmt, BM, narrow_last ? n1_last : BNM);
      const uint32_t idesc_chk = umma_idesc(fmt, fmt, BM, 16);
      uint32_t it = 0, lt = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++lt) {
        int mt, nt;
        tile_coords(tile, nMb, nNb, kGroupRows / BM, mt, nt);
        const bool narrow = narrow_last && nt == nNb - 1;
        const uint32_t b = lt & 1, ub = lt >> 1;
        if (ub > 0 && !mbar_wait_bounded(&sm.tempty[b], (ub - 1) & 1, p.wait_limit_ns)) { sm.timeout = 1; break; }
        tc_fence_after();
        const uint32_t dcol = tmem + b * BNM;
        for (int kt = 0; kt < nk; ++kt, ++it) {
          const uint32_t s = it % STAGES, u = it / STAGES;
          if (!mbar_wait_bounded(&sm.full[s], u & 1, p.wait_limit_ns)) { sm.timeout = 1; ok = false; break; }
          tc_fence_after();
          const uint32_t a0 = smem_addr(sm.a[s]), b0 = smem_addr(sm.b[s]);
#pragma unroll
          for (int kk = 0; kk < BKB / 32; ++kk) {  // one MMA (or two narrow ones) per 32 bytes of K
            const uint32_t accum = (kt > 0 || kk > 0) ? 1u : 0u;
            const uint64_t ad = umma_desc_sw128(a0 + kk * 32), bd = umma_desc_sw128(b0 + kk * 32);
            const uint64_t bd_chk = umma_desc_sw128(b0 + (BNM - 16) * BKB + kk * 32);
            if (KIND == 0) {
              umma_bf16(dcol, ad, bd, narrow ? idesc_n1 : idesc, accum);
              if (FT && narrow) umma_bf16(dcol + (BNM - 16), ad, bd_chk, idesc_chk, accum);
            } else {
              umma_f8(dcol, ad, bd, narrow ? idesc_n1 : idesc, accum);
              if (FT && narrow) umma_f8(dcol + (BNM - 16), ad, bd_chk, idesc_chk, accum);
            }
          }
          umma_commit(&sm.empty[s]);
        }
        // a wait gave up: the accumulator is incomplete, so the tile is never handed to the
        // epilogue (whose own wait then gives up and leaves the tile unstored)
        if (!ok) break;
        umma_commit(&sm.tfull[b]);
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue (warps 2..5)
    const int q = warp & 3;                 // TMEM lane quarter of this warp
    const int row = q * 32 + lane;          // tile row = TMEM lane
    const int ew = warp - 2;                // epilogue warp index 0..3
    const int et = t - 64;                  // epilogue thread index 0..127
    const bool beta_nz = p.beta != 0.0f;
    const float alpha = alpha_eff(p);
    uint32_t lt = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++lt) {
      int mt, nt;
      tile_coords(tile, nMb, nNb, kGroupRows / BM, mt, nt);
      const int m0 = mt * BM, n0 = nt * BN;
      const int nI = min(BM, p.M - m0), nJ = min(BN, p.N - n0);
      const int64_t gi = m0 + row;
      const bool row_ok = row < nI;
      const uint32_t b = lt & 1, ub = lt >> 1;
      // tcgen05.ld is warp-collective (.sync.aligned): every TMEM load below is executed by
      // all 32 lanes of the warp, whatever their row; `got` is made warp-uniform for that.
      const bool got = __all_sync(0xffffffffu, mbar_wait_bounded(&sm.tfull[b], ub & 1, p.wait_limit_ns));
      if (!got) sm.timeout = 1;
      tc_fence_after();
      const uint32_t trow = tmem + b * BNM + (static_cast<uint32_t>(q * 32) << 16);
      float rs = 0.f, rc = 0.f, rabs = 0.f;   // compensated sum of C over the row, upward |C| sum
      float cs = 0.f, cc = 0.f, cabs = 0.f;   // same for C_in
      uint32_t wp[16];  // checksum columns: the pieces' products
#pragma unroll
      for (int q2 = 0; q2 < 16; ++q2) wp[q2] = 0u;
      // Injection points in this tile (test launches only): the per-element injection code
      // is kept out of the hot loop so the epilogue stays small in the instruction cache,
      // which it shares with the producer and MMA warps.
      int inj_c = INT_MAX;  // next tile column of this row holding an injection point
      if (FT && p.inj.n > 0) inj_c = next_inj_col(p, gi, n0, nJ, -1);
      if (got) {
        const int nch = (nJ + 7) / 8;  // chunks of 8 columns holding data (warp-uniform)
#pragma unroll 1
        for (int ch = 0; ch < nch; ++ch) {
          uint32_t v[8];
          __syncwarp();  // reconverge after the previous chunk's per-lane branches
          tmem_ld8(trow + ch * 8, v);
          tmem_ld_wait();
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int col = ch * 8 + j;
            const int64_t gj = n0 + col;
            const bool ok = row_ok && col < nJ;
            float acc = __uint_as_float(v[j]);
            float cin = 0.f;
            if (beta_nz && ok) cin = p.C[gi + gj * p.ldc];
            float out;
            if (FT && col == inj_c) {
              out = inject_element(p, alpha, gi, gj, acc, cin, beta_nz);
              inj_c = next_inj_col(p, gi, n0, nJ, col);
            } else {
              out = beta_nz ? fmaf(alpha, acc, p.beta * cin) : alpha * acc;
            }
            if (ok) p.C[gi + gj * p.ldc] = out;
            if (FT) {
              const float o = ok ? out : 0.f;
              neumaier(rs, rc, o);
              rabs = __fadd_ru(rabs, fabsf(o));
              if (beta_nz) {
                neumaier(cs, cc, cin);
                cabs = __fadd_ru(cabs, fabsf(cin));
                // column sums of C_in over this warp's 32 rows, for the lazy column side
                const float csum = warp_sum_plain(ok ? cin : 0.f);
                const float cabsum = warp_sum_up(fabsf(ok ? cin : 0.f));
                if (lane == 0 && col < BNM) { sm.cin_col[ew][col] = csum; sm.cin_col_abs[ew][col] = cabsum; }
              }
            }
          }
        }
        if (FT) {  // C^r pieces from the checksum columns of B^r
#pragma unroll
          for (int h = 0; h < (E::kPieces + 7) / 8; ++h) {
            uint32_t v8[8];
            __syncwarp();
            tmem_ld8(trow + BN + 8 * h, v8);
            tmem_ld_wait();
#pragma unroll
            for (int q2 = 0; q2 < 8; ++q2) wp[8 * h + q2] = v8[q2];
          }
        }
      }
      // The accumulator buffer is free for the MMA warp's next-but-one tile.
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&sm.tempty[b]);
      if (!FT) continue;

      // -------------------------------------------------------- row verification
      if (et == 0) { sm.nflag_rows = 0; sm.first_row = INT_MAX; }
      named_bar(1, 128);
      double delta = 0.0, tau = 0.0, predicted = 0.0;
      if (got && row_ok) {
        double pr;
        if (KIND == 0) {
          pr = (double)__uint_as_float(wp[0]) + (double)__uint_as_float(wp[1]) + (double)__uint_as_float(wp[2]);
        } else {
          pr = 0.0;
          double sc = 512.0;  // piece scale 2^(9 - 4p)
#pragma unroll
          for (int q2 = 0; q2 < E::kPieces; ++q2, sc *= 0.0625) pr += sc * (double)__uint_as_float(wp[q2]);
        }
        const double cin_sum = (double)cs + (double)cc;
        predicted = (double)alpha * pr + (beta_nz ? (double)p.beta * cin_sum : 0.0);
        for (int e = 0; e < p.inj.n; ++e) {
          const InjectPoint& ip = p.inj.p[e];
          if (ip.site == kSiteChecksumRow && ip.i == gi && ip.j >= n0 && ip.j < n0 + nJ) {
            const double em = ldexp(fabs(predicted), ip.rel_log2);
            predicted = ip.sign < 0 ? predicted - em : predicted + em;
          }
        }
        const double ref = (double)rs + (double)rc;
        delta = ref - predicted;
        // tau = |alpha| P (gamma_K(u_acc) (1 + s) + 2^-20 + gamma_BN(2^-24)) + 2^-23 sum|C| +
        // 2^-21 |beta| sum|C_in|, P an upper bound of sum_k |A(i,k)| sum_{j in tile} |B(k,j)|:
        // gamma_K(u_acc) P bounds the accumulations of the row's outputs, gamma_K(u_acc) s P
        // those of the prediction (s bounds sum_p |piece_p| / |B e|), gamma_BN(2^-24) P the
        // binary32 sum B e over the tile's BN columns, 2^-23 sum|C| the compensated row sum,
        // 2^-21 |beta| sum|C_in| the beta side of the roundings of beta C_in, of the output's
        // multiply-add and of the compensated C_in sum (four times 2^-24, doubled), and
        // 2^-20 P the alpha side of the output rounding, the cross terms and the binary64
        // operations (about 2^-23 P, quadrupled).
        const float P = __fmul_ru(p.rowAbsA[gi], p.maxAbsBe[nt]);
        const float g = gamma32_up((float)p.K, p.u_acc);
        const float genc = gamma32_up((float)BN, 0x1p-24f);
        const float prod = __fmul_ru(__fmul_ru(fabsf(alpha), P),
                                     __fadd_ru(__fadd_ru(__fmul_ru(g, 1.0f + E::kPieceSum), 0x1p-20f), genc));
        const float outp = __fadd_ru(__fmul_ru(0x1p-23f, rabs), __fmul_ru(0x1p-21f, __fmul_ru(fabsf(p.beta), cabs)));
        tau = (double)__fadd_ru(prod, outp);
        if (!(fabs(delta) <= tau) || isinf(delta)) {
          atomicAdd(&sm.nflag_rows, 1);
          atomicMin(&sm.first_row, row);
        }
      }
      named_bar(1, 128);
      if (row_ok && row == sm.first_row) { sm.delta_row = delta; sm.tau_row = tau; sm.pred_row = predicted; }
      __threadfence_block();
      named_bar(1, 128);
      const int nr = sm.nflag_rows;
      if (nr > 0) {
        // A row mismatch. The column checksums that locate it (Section V.A, lazy side) are
        // formed by the resolve pass after every tile is stored, spread over many CTAs; this
        // CTA only hands the tile over (with the column sums of C_in, which it overwrote).
        if (et == 0) sm.pend_slot = (int)atomicAdd(&p.pend->count, 1u);
        named_bar(1, 128);
        const int slot = sm.pend_slot;
        if (slot < kTcPendCap) {
          TcPendingEntry& pe = p.pend->e[slot];
          if (et == 0) {
            pe.mt = mt; pe.nt = nt; pe.nr = nr; pe.first_row = sm.first_row;
            pe.delta_row = sm.delta_row; pe.tau_row = sm.tau_row; pe.pred_row = sm.pred_row; pe.done = 0u;
          }
          if (beta_nz)
            for (int c = et; c < nJ; c += 128) {
              double cs2 = 0.0;
              float ca = 0.f;
              for (int w = 0; w < 4; ++w) { cs2 += (double)sm.cin_col[w][c]; ca = __fadd_ru(ca, sm.cin_col_abs[w][c]); }
              pe.cin_sum[c] = cs2;
              pe.cin_abs[c] = ca;
            }
        } else if (et == 0) {
          // more mismatching tiles in this call than the resolve pass holds: detected, not located
          tc_record(p, FT_KIND_UNCORRECTABLE, mt, nt, m0 + sm.first_row, -1, sm.delta_row, 0.0, sm.tau_row, 0.0,
                    0.0, 0.0, nr, 0);
          count_kind(p, FT_KIND_UNCORRECTABLE);
        }
      }
      if (et == 0 && got && p.report)  // an abandoned tile (a wait gave up) is not counted
        atomicAdd(reinterpret_cast<unsigned long long*>(&p.report->tiles_checked), 1ull);
      named_bar(1, 128);  // every epilogue thread is done with this tile's shared state
    }
  }

  // ------------------------------------------------------------ teardown
  tc_fence_before();
  __syncthreads();
  if (t == 0 && sm.timeout && p.report) atomicOr(&p.report->status, FT_STATUS_TIMEOUT);
  if (warp == 1) {
    __syncwarp();  // tcgen05.dealloc is warp-collective: reconverge after the divergent MMA issue
    tc_fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

// The CTA pair's single-thread loops, the MMA issue (even CTA) and the TMA producer (each
// CTA), are kept out of line (__noinline__). The loops themselves are unchanged; measured, the
// pair kernel then runs 3-10% faster for BF16 and FP8 operands, protected or not, which we
// attribute to instruction fetch (the epilogue warps' verification code is long).
//
// The MMA issue loop.
template <bool FT, int KIND>
__device__ __noinline__ void pair_mma_loop(const TcParams& p, TcSmem<2>& sm, uint32_t tmem, int unit0, int ustep, int nunits, int nUb, int nNb, int nk) {
  constexpr int BN = TcGeom<FT, KIND>::BN;
  constexpr int STAGES = TcStage<2>::kStages;
  // kind::f16 with BF16 operands (format 1), or kind::f8f6f4 with E4M3 operands (format 0)
  constexpr uint32_t fmt = KIND == 0 ? 1u : 0u;
  uint32_t it = 0, lt = 0;
  bool ok = true;
  for (int unit = unit0; unit < nunits && ok; unit += ustep, ++lt) {
    int mu, nt;
    tile_coords(unit, nUb, nNb, kGroupRows / (2 * BM), mu, nt);
    const uint32_t idesc = umma_idesc(fmt, fmt, 2 * BM, pair_shape<FT>(min(BN, p.N - nt * BN)).n);
    const uint32_t b = lt & 1, ub = lt >> 1;
    if (ub > 0 && !mbar_wait_bounded(&sm.tempty[b], (ub - 1) & 1, p.wait_limit_ns)) { sm.timeout = 1; break; }
    tc_fence_after();
    const uint32_t dcol = tmem + b * BNM;
    for (int kt = 0; kt < nk; ++kt, ++it) {
      const uint32_t s = it % STAGES, u = it / STAGES;
      if (!mbar_wait_bounded(&sm.full[s], u & 1, p.wait_limit_ns)) { sm.timeout = 1; ok = false; break; }
      tc_fence_after();
      const uint32_t a0 = smem_addr(sm.a[s]), b0 = smem_addr(sm.b[s]);
#pragma unroll
      for (int kk = 0; kk < BKB / 32; ++kk) {  // one MMA per 32 bytes of K
        const uint32_t accum = (kt > 0 || kk > 0) ? 1u : 0u;
        const uint64_t ad = umma_desc_sw128(a0 + kk * 32), bd = umma_desc_sw128(b0 + kk * 32);
        if (KIND == 0) umma_bf16_pair(dcol, ad, bd, idesc, accum);
        else umma_f8_pair(dcol, ad, bd, idesc, accum);
      }
      umma_commit_pair(&sm.empty[s]);
    }
    // a wait gave up: the accumulator is incomplete, so the unit is never handed to the
    // epilogues (whose own waits then give up and leave the tiles unstored)
    if (!ok) break;
    umma_commit_pair(&sm.tfull[b]);
  }
}

// The TMA producer loop (one thread per CTA).
template <bool FT, int KIND>
__device__ __noinline__ void pair_tma_loop(const TcParams& p, TcSmem<2>& sm, const CUtensorMap* pA, const CUtensorMap* pB, const CUtensorMap* pB2, const CUtensorMap* pChk, int rank, int unit0, int ustep, int nunits, int nUb, int nNb, int nk, int bk_elems) {
  constexpr int BN = TcGeom<FT, KIND>::BN, CHK = TcGeom<FT, KIND>::CHK;
  constexpr int STAGES = TcStage<2>::kStages, BROWS = TcStage<2>::kBRows;
  tma_prefetch_desc(pA);
  tma_prefetch_desc(pB);
  if (FT) { tma_prefetch_desc(pB2); tma_prefetch_desc(pChk); }
  uint32_t it = 0;
  bool ok = true;
  for (int unit = unit0; unit < nunits && ok; unit += ustep) {
    int mu, nt;
    tile_coords(unit, nUb, nNb, kGroupRows / (2 * BM), mu, nt);
    const int mt = 2 * mu + rank;
    const int n0 = nt * BN;
    const PairShape g = pair_shape<FT>(min(BN, p.N - n0));
    // bytes of both CTAs' loads, expected on the even CTA's barrier
    const uint32_t bytes = (2 * BM + BROWS + (FT ? (g.b1_data ? BROWS : CHK) : BROWS)) * BKB;
    const int skt = p.inj.n > 0 ? stall_ktile(p, mu, 2 * BM, nt, nk, BN) : -1;
    for (int kt = 0; kt < nk; ++kt, ++it) {
      const uint32_t s = it % STAGES, u = it / STAGES;
      if (u > 0 && !mbar_wait_bounded(&sm.empty[s], (u - 1) & 1, p.wait_limit_ns)) { sm.timeout = 1; ok = false; break; }
      const int k0 = kt * bk_elems;
      const uint32_t fbar = mapa_shared(smem_addr(&sm.full[s]), 0);
      if (rank == 0) mbar_arrive_expect_tx(&sm.full[s], bytes + (kt == skt ? 16u : 0u));
      // rows beyond M (an odd CTA past the last row tile) read the fill value, zero
      tma_load_2d_pair(sm.a[s], pA, fbar, k0, mt * BM);
      if (rank == 0) {
        tma_load_2d_pair(sm.b[s], pB, fbar, k0, n0);
      } else {
        if (g.b1_data) tma_load_2d_pair(sm.b[s], FT ? pB2 : pB, fbar, k0, n0 + g.b1_row);
        if (FT) tma_load_2d_pair(sm.b[s] + (g.b1_data ? BROWS - CHK : 0) * BKB, pChk, fbar, k0, nt * CHK);
      }
    }
  }
}

// CTA-pair kernel (cta_group::2): a thread-block cluster of two CTAs on one TPC computes each
// 256 x 256 product. Each CTA stages its own 128 rows of A and half of B^r (128 rows: the even
// CTA data columns 0..127, the odd CTA the rest and the checksum rows, as pair_shape gives),
// so a CTA's shared-memory traffic per MMA is half the B operand of the one-CTA kernel. Both
// CTAs' TMA loads complete on the even CTA's staging barrier; the even CTA's MMA warp issues
// M = 256 MMAs over both CTAs' stages and its commits arrive on the barriers of both. Each
// CTA's epilogue verifies and stores its own 128-row tile, so the verification interval, the
// pending list and the resolve pass are those of the one-CTA kernel. The pair loops over units
// (256-row block, column block) in the order of tile_coords.
template <bool FT, int KIND, bool CB>
__global__ void __launch_bounds__(NTHREADS, 1)
    tc_gemm_pair_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                        const __grid_constant__ CUtensorMap tmB2, const __grid_constant__ CUtensorMap tmChk,
                        const __grid_constant__ TcParams p) {
  constexpr int BN = TcGeom<FT, KIND>::BN, CHK = TcGeom<FT, KIND>::CHK;
  constexpr int STAGES = TcStage<2>::kStages, BROWS = TcStage<2>::kBRows;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  TcSmem<2>& sm = *reinterpret_cast<TcSmem<2>*>(smem_raw);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  using E = Elem<KIND>;
  const int bk_elems = BKB / E::kBytes;
  const int nk = (p.K + bk_elems - 1) / bk_elems;
  const int nMb = (p.M + BM - 1) / BM, nNb = (p.N + BN - 1) / BN;
  const int nUb = (nMb + 1) / 2;  // 256-row blocks
  const int nunits = nUb * nNb;
  const int rank = static_cast<int>(cluster_ctarank());
  const int unit0 = static_cast<int>(blockIdx.x) / 2, ustep = static_cast<int>(gridDim.x) / 2;

  if (t == 0) {
    for (int s = 0; s < STAGES; ++s) { mbar_init(&sm.full[s], 1); mbar_init(&sm.empty[s], 1); }
    // tempty: the four epilogue warps of each CTA (the odd CTA's arrive remotely)
    for (int b = 0; b < 2; ++b) { mbar_init(&sm.tfull[b], 1); mbar_init(&sm.tempty[b], 8); }
    sm.timeout = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    __syncwarp();
    tmem_alloc_pair(&sm.tmem_base, TMEM_COLS);
  }
  tc_fence_before();
  cluster_sync();  // the peer's barriers are initialised before any TMA or commit signals them
  tc_fence_after();
  const uint32_t tmem = sm.tmem_base;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) pair_tma_loop<FT, KIND>(p, sm, &tmA, &tmB, &tmB2, &tmChk, rank, unit0, ustep, nunits, nUb, nNb, nk, bk_elems);
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issue (even CTA)
    if (lane == 0 && rank == 0) pair_mma_loop<FT, KIND>(p, sm, tmem, unit0, ustep, nunits, nUb, nNb, nk);
  } else {
    // ------------------------------------------------------------ epilogue (warps 2..5)
    const int q = warp & 3;                 // TMEM lane quarter of this warp
    const int row = q * 32 + lane;          // tile row = TMEM lane
    const int ew = warp - 2;                // epilogue warp index 0..3
    const int et = t - 64;                  // epilogue thread index 0..127
    const bool beta_nz = p.beta != 0.0f;
    const float alpha = alpha_eff(p);
    uint32_t lt = 0;
    for (int unit = unit0; unit < nunits; unit += ustep, ++lt) {
      int mu, nt;
      tile_coords(unit, nUb, nNb, kGroupRows / (2 * BM), mu, nt);
      const int mt = 2 * mu + rank;
      const int m0 = mt * BM, n0 = nt * BN;
      const int nI = min(BM, p.M - m0), nJ = min(BN, p.N - n0);  // nI <= 0: an odd CTA past the last row tile
      const int chk_col = pair_shape<FT>(nJ).chk_col;  // first checksum column in TMEM
      const int64_t gi = m0 + row;
      const bool row_ok = row < nI;
      const uint32_t b = lt & 1, ub = lt >> 1;
      // tcgen05.ld is warp-collective (.sync.aligned): every TMEM load below is executed by
      // all 32 lanes of the warp, whatever their row; `got` is made warp-uniform for that.
      const bool got = __all_sync(0xffffffffu, mbar_wait_bounded(&sm.tfull[b], ub & 1, p.wait_limit_ns));
      if (!got) sm.timeout = 1;
      tc_fence_after();
      const uint32_t trow = tmem + b * BNM + (static_cast<uint32_t>(q * 32) << 16);
      float rs = 0.f, rc = 0.f, rabs = 0.f;   // compensated sum of C over the row, upward |C| sum
      float cs = 0.f, cc = 0.f, cabs = 0.f;   // same for C_in
      uint32_t wp[16];  // checksum columns: the pieces' products
#pragma unroll
      for (int q2 = 0; q2 < 16; ++q2) wp[q2] = 0u;
      // Injection points in this tile (test launches only): the per-element injection code
      // is kept out of the hot loop so the epilogue stays small in the instruction cache,
      // which it shares with the producer and MMA warps.
      int inj_c = INT_MAX;  // next tile column of this row holding an injection point
      if (FT && p.inj.n > 0) inj_c = next_inj_col(p, gi, n0, nJ, -1);
      if (got) {
        const int nch = (nJ + 7) / 8;  // chunks of 8 columns holding data (warp-uniform)
#pragma unroll 1
        for (int ch = 0; ch < nch; ++ch) {
          uint32_t v[8];
          __syncwarp();  // reconverge after the previous chunk's per-lane branches
          tmem_ld8(trow + ch * 8, v);
          tmem_ld_wait();
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int col = ch * 8 + j;
            const int64_t gj = n0 + col;
            const bool ok = row_ok && col < nJ;
            float acc = __uint_as_float(v[j]);
            float cin = 0.f;
            if (beta_nz && ok) {
              if constexpr (CB) cin = __uint_as_float(static_cast<uint32_t>(p.Cb[gi + gj * p.ldcb]) << 16);
              else cin = p.C[gi + gj * p.ldc];
            }
            float out;
            if (FT && col == inj_c) {
              out = inject_element(p, alpha, gi, gj, acc, cin, beta_nz);
              inj_c = next_inj_col(p, gi, n0, nJ, col);
            } else {
              out = beta_nz ? fmaf(alpha, acc, p.beta * cin) : alpha * acc;
            }
            if (ok) {
              if constexpr (CB) {
                // the bfloat16 C, rounded to nearest once; a protected call also keeps the
                // FP32 value, which the resolve pass reads and corrects
                p.Cb[gi + gj * p.ldcb] = __bfloat16_as_ushort(__float2bfloat16_rn(out));
                if (FT) p.C[gi + gj * p.ldc] = out;
              } else {
                p.C[gi + gj * p.ldc] = out;
              }
            }
            if (FT) {
              const float o = ok ? out : 0.f;
              neumaier(rs, rc, o);
              rabs = __fadd_ru(rabs, fabsf(o));
              if (beta_nz) {
                neumaier(cs, cc, cin);
                cabs = __fadd_ru(cabs, fabsf(cin));
                // column sums of C_in over this warp's 32 rows, for the lazy column side
                const float csum = warp_sum_plain(ok ? cin : 0.f);
                const float cabsum = warp_sum_up(fabsf(ok ? cin : 0.f));
                if (lane == 0 && col < BNM) { sm.cin_col[ew][col] = csum; sm.cin_col_abs[ew][col] = cabsum; }
              }
            }
          }
        }
        if (FT) {  // C^r pieces from the checksum columns of B^r
#pragma unroll
          for (int h = 0; h < (E::kPieces + 7) / 8; ++h) {
            uint32_t v8[8];
            __syncwarp();
            tmem_ld8(trow + chk_col + 8 * h, v8);
            tmem_ld_wait();
#pragma unroll
            for (int q2 = 0; q2 < 8; ++q2) wp[8 * h + q2] = v8[q2];
          }
        }
      }
      // The accumulator buffer is free for the MMA warp's next-but-one unit (the barrier is the
      // even CTA's, which issues the MMAs).
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        if (rank != 0) mbar_arrive_cluster(mapa_shared(smem_addr(&sm.tempty[b]), 0));
        else mbar_arrive(&sm.tempty[b]);
      }
      if (!FT) continue;

      // -------------------------------------------------------- row verification
      if (et == 0) { sm.nflag_rows = 0; sm.first_row = INT_MAX; }
      named_bar(1, 128);
      double delta = 0.0, tau = 0.0, predicted = 0.0;
      if (got && row_ok) {
        double pr;
        if (KIND == 0) {
          pr = (double)__uint_as_float(wp[0]) + (double)__uint_as_float(wp[1]) + (double)__uint_as_float(wp[2]);
        } else {
          pr = 0.0;
          double sc = 512.0;  // piece scale 2^(9 - 4p)
#pragma unroll
          for (int q2 = 0; q2 < E::kPieces; ++q2, sc *= 0.0625) pr += sc * (double)__uint_as_float(wp[q2]);
        }
        const double cin_sum = (double)cs + (double)cc;
        predicted = (double)alpha * pr + (beta_nz ? (double)p.beta * cin_sum : 0.0);
        for (int e = 0; e < p.inj.n; ++e) {
          const InjectPoint& ip = p.inj.p[e];
          if (ip.site == kSiteChecksumRow && ip.i == gi && ip.j >= n0 && ip.j < n0 + nJ) {
            const double em = ldexp(fabs(predicted), ip.rel_log2);
            predicted = ip.sign < 0 ? predicted - em : predicted + em;
          }
        }
        const double ref = (double)rs + (double)rc;
        delta = ref - predicted;
        // tau = |alpha| P (gamma_K(u_acc) (1 + s) + 2^-20 + gamma_BN(2^-24)) + 2^-23 sum|C| +
        // 2^-21 |beta| sum|C_in|, P an upper bound of sum_k |A(i,k)| sum_{j in tile} |B(k,j)|:
        // gamma_K(u_acc) P bounds the accumulations of the row's outputs, gamma_K(u_acc) s P
        // those of the prediction (s bounds sum_p |piece_p| / |B e|), gamma_BN(2^-24) P the
        // binary32 sum B e over the tile's BN columns, 2^-23 sum|C| the compensated row sum,
        // 2^-21 |beta| sum|C_in| the beta side of the roundings of beta C_in, of the output's
        // multiply-add and of the compensated C_in sum (four times 2^-24, doubled), and
        // 2^-20 P the alpha side of the output rounding, the cross terms and the binary64
        // operations (about 2^-23 P, quadrupled).
        const float P = __fmul_ru(p.rowAbsA[gi], p.maxAbsBe[nt]);
        const float g = gamma32_up((float)p.K, p.u_acc);
        const float genc = gamma32_up((float)BN, 0x1p-24f);
        const float prod = __fmul_ru(__fmul_ru(fabsf(alpha), P),
                                     __fadd_ru(__fadd_ru(__fmul_ru(g, 1.0f + E::kPieceSum), 0x1p-20f), genc));
        const float outp = __fadd_ru(__fmul_ru(0x1p-23f, rabs), __fmul_ru(0x1p-21f, __fmul_ru(fabsf(p.beta), cabs)));
        tau = (double)__fadd_ru(prod, outp);
        if (!(fabs(delta) <= tau) || isinf(delta)) {
          atomicAdd(&sm.nflag_rows, 1);
          atomicMin(&sm.first_row, row);
        }
      }
      named_bar(1, 128);
      if (row_ok && row == sm.first_row) { sm.delta_row = delta; sm.tau_row = tau; sm.pred_row = predicted; }
      __threadfence_block();
      named_bar(1, 128);
      const int nr = sm.nflag_rows;
      if (nr > 0) {
        // A row mismatch. The column checksums that locate it (Section V.A, lazy side) are
        // formed by the resolve pass after every tile is stored, spread over many CTAs; this
        // CTA only hands the tile over (with the column sums of C_in, which it overwrote).
        if (et == 0) sm.pend_slot = (int)atomicAdd(&p.pend->count, 1u);
        named_bar(1, 128);
        const int slot = sm.pend_slot;
        if (slot < kTcPendCap) {
          TcPendingEntry& pe = p.pend->e[slot];
          if (et == 0) {
            pe.mt = mt; pe.nt = nt; pe.nr = nr; pe.first_row = sm.first_row;
            pe.delta_row = sm.delta_row; pe.tau_row = sm.tau_row; pe.pred_row = sm.pred_row; pe.done = 0u;
          }
          if (beta_nz)
            for (int c = et; c < nJ; c += 128) {
              double cs2 = 0.0;
              float ca = 0.f;
              for (int w = 0; w < 4; ++w) { cs2 += (double)sm.cin_col[w][c]; ca = __fadd_ru(ca, sm.cin_col_abs[w][c]); }
              pe.cin_sum[c] = cs2;
              pe.cin_abs[c] = ca;
            }
        } else if (et == 0) {
          // more mismatching tiles in this call than the resolve pass holds: detected, not located
          tc_record(p, FT_KIND_UNCORRECTABLE, mt, nt, m0 + sm.first_row, -1, sm.delta_row, 0.0, sm.tau_row, 0.0,
                    0.0, 0.0, nr, 0);
          count_kind(p, FT_KIND_UNCORRECTABLE);
        }
      }
      if (et == 0 && got && nI > 0 && p.report)  // an abandoned tile (a wait gave up) is not counted
        atomicAdd(reinterpret_cast<unsigned long long*>(&p.report->tiles_checked), 1ull);
      named_bar(1, 128);  // every epilogue thread is done with this tile's shared state
    }
  }

  // ------------------------------------------------------------ teardown
  // neither CTA leaves (nor frees the pair's TMEM) while the other may still signal its
  // barriers or read its TMEM
  tc_fence_before();
  __syncwarp();
  cluster_sync();
  if (t == 0 && sm.timeout && p.report) atomicOr(&p.report->status, FT_STATUS_TIMEOUT);
  if (warp == 1) {
    __syncwarp();  // tcgen05.dealloc is warp-collective: reconverge after the divergent MMA issue
    tc_fence_after();
    tmem_dealloc_pair(tmem, TMEM_COLS);
  }
}

// ---------------------------------------------------------------------------------------
// Resolve pass: locate and correct the errors of the tiles whose row checksums mismatched
// (run after the GEMM on the same stream; with no such tile every CTA returns at once).
// A work item is (mismatching tile, group of 8 columns); warp w of the CTA takes column
// j = 8 g + w of the tile and forms
//   C^c_ref(j) = sum_i C(i,j) over the stored tile (compensated, warp sum in binary64),
//   C^c(j)     = alpha sum_k (e^T A)(k) B(k,j) [+ beta sum_i C_in(i,j)] (binary32 dot),
//   P_c(j)     = sum_k (sum_i |A(i,k)|) |B(k,j)| (upward),
// and, when exactly one row mismatched and beta == 0, that row's element recomputed,
// alpha sum_k A(i,k) B(k,j), with S = sum_k |A(i,k)||B(k,j)|. The CTA that finishes a
// tile's last group classifies the tile and corrects it.
// ---------------------------------------------------------------------------------------
constexpr int kResolveWarps = 8;

// The lazy side's row-block sums, formed only for the row blocks of pending tiles (after the
// GEMM, before the resolve pass; with no pending tile every CTA returns at once): for the
// 128-row block of each pending tile, e^T A(k) = sum_i A(i,k) (binary32, any order) and
// sum_i |A(i,k)| (upward), into sA / absSA. CTA x takes k = 64 x .. 64 x + 63: thread t loads
// k = 64 x + 8 (t & 7) .. + 7 of rows t >> 3, (t >> 3) + 32, ...; the 32 row groups' partials
// meet in shared memory and are summed in a fixed order. Two pending tiles of one row block
// write the same values.
constexpr int kColsumK = 64;
template <int KIND>
__global__ void __launch_bounds__(256) tc_colsum_kernel(const __grid_constant__ TcParams p) {
  using E = Elem<KIND>;
  __shared__ __align__(16) float red_s[32][kColsumK];
  __shared__ __align__(16) float red_a[32][kColsumK];
  const unsigned npend = min(*reinterpret_cast<volatile const unsigned*>(&p.pend->count), (unsigned)kTcPendCap);
  const int t = threadIdx.x, oct = t & 7, rg = t >> 3;
  const int64_t k = (int64_t)blockIdx.x * kColsumK + oct * 8;
  const uint8_t* A = static_cast<const uint8_t*>(p.A);
  for (unsigned e = 0; e < npend; ++e) {
    const int mt = p.pend->e[e].mt;
    const int m0 = mt * BM, nI = min(BM, p.M - m0);
    float s[8], a[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) { s[q] = 0.f; a[q] = 0.f; }
#pragma unroll
    for (int u = 0; u < BM / 32; ++u) {
      const int i = rg + 32 * u;
      float x[8];
      E::unpack((i < nI && k < p.K) ? E::load_raw(A + (int64_t)(m0 + i) * p.lda * E::kBytes, k, p.K) : E::zero(), x);
#pragma unroll
      for (int q = 0; q < 8; ++q) { s[q] += x[q]; a[q] = __fadd_ru(a[q], fabsf(x[q])); }
    }
    *reinterpret_cast<float4*>(&red_s[rg][oct * 8]) = make_float4(s[0], s[1], s[2], s[3]);
    *reinterpret_cast<float4*>(&red_s[rg][oct * 8 + 4]) = make_float4(s[4], s[5], s[6], s[7]);
    *reinterpret_cast<float4*>(&red_a[rg][oct * 8]) = make_float4(a[0], a[1], a[2], a[3]);
    *reinterpret_cast<float4*>(&red_a[rg][oct * 8 + 4]) = make_float4(a[4], a[5], a[6], a[7]);
    __syncthreads();
    if (t < kColsumK) {
      float S = 0.f, Aab = 0.f;
      for (int g = 0; g < 32; ++g) { S += red_s[g][t]; Aab = __fadd_ru(Aab, red_a[g][t]); }
      const int64_t kk = (int64_t)blockIdx.x * kColsumK + t;
      if (kk < p.K) {
        p.sA[(int64_t)mt * p.sa_pitch + kk] = S;
        p.absSA[(int64_t)mt * p.sa_pitch + kk] = Aab;
      }
    }
    __syncthreads();  // the reduction arrays are reused by the next pending tile
  }
}

struct ResolveShared {
  int last, first_col, first_elem;
  double part_d[kResolveWarps], part_r[kResolveWarps];
  float part_pc[kResolveWarps], part_S[kResolveWarps];
  double cref;
  float cref_abs;
};

// One column j of a mismatching tile, the eight warps splitting K in blocks of 256
// (lane l loads k .. k + 7 of a block with 16-byte loads: B and A rows are 16-byte aligned,
// leading dimensions being multiples of 8; e^T A rows are 32-byte aligned, pitch a multiple
// of 8). Partial sums meet in shared memory; thread 0 forms the comparisons.
template <bool kRecompute, int KIND>
__device__ void resolve_column(const TcParams& p, float alpha, TcPendingEntry& pe, ResolveShared& sh, int mt, int m0,
                               int n0, int nI, int cidx, bool beta_nz) {
  using E = Elem<KIND>;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t gj = n0 + cidx;
  const int64_t gi = m0 + pe.first_row;
  if (warp == 0) {
    float s = 0.f, c = 0.f, a = 0.f;
    for (int i = lane; i < nI; i += 32) {
      const float x = p.C[(int64_t)(m0 + i) + gj * p.ldc];
      neumaier(s, c, x);
      a = __fadd_ru(a, fabsf(x));
    }
    const double cref = warp_sum_f64((double)s + (double)c);
    const float cref_abs = warp_sum_up(a);
    if (lane == 0) { sh.cref = cref; sh.cref_abs = cref_abs; }
  }
  const void* bcol = static_cast<const uint8_t*>(p.B) + gj * p.ldb * E::kBytes;
  const void* arow = static_cast<const uint8_t*>(p.A) + gi * p.lda * E::kBytes;
  const float* sAI = p.sA + (int64_t)mt * p.sa_pitch;
  const float* absAI = p.absSA + (int64_t)mt * p.sa_pitch;
  const int K = p.K, K8 = p.K & ~7;
  float d = 0.f, pc = 0.f, r = 0.f, S = 0.f;
#pragma unroll 2
  for (int k = warp * 256 + lane * 8; k < K8; k += kResolveWarps * 256) {
    float bx[8];
    E::load8(bcol, k, K, bx);
    const float4 s0 = *reinterpret_cast<const float4*>(sAI + k), s1 = *reinterpret_cast<const float4*>(sAI + k + 4);
    const float4 u0 = *reinterpret_cast<const float4*>(absAI + k), u1 = *reinterpret_cast<const float4*>(absAI + k + 4);
    const float sv[8] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
    const float uv[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      d = fmaf(sv[q], bx[q], d);
      pc = __fmaf_ru(uv[q], fabsf(bx[q]), pc);
    }
    if (kRecompute) {
      float ax[8];
      E::load8(arow, k, K, ax);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        r = fmaf(ax[q], bx[q], r);
        S = __fmaf_ru(fabsf(ax[q]), fabsf(bx[q]), S);
      }
    }
  }
  if (warp == kResolveWarps - 1 && K8 + lane < K) {  // ragged end of K, one element per lane
    const int k = K8 + lane;
    const float bx = E::at(bcol, k);
    d = fmaf(sAI[k], bx, d);
    pc = __fmaf_ru(absAI[k], fabsf(bx), pc);
    if (kRecompute) {
      const float ax = E::at(arow, k);
      r = fmaf(ax, bx, r);
      S = __fmaf_ru(fabsf(ax), fabsf(bx), S);
    }
  }
  const double wd = warp_sum_f64((double)d);
  const float wpc = warp_sum_up(pc);
  double wr = 0.0;
  float wS = 0.f;
  if (kRecompute) { wr = warp_sum_f64((double)r); wS = warp_sum_up(S); }
  if (lane == 0) { sh.part_d[warp] = wd; sh.part_pc[warp] = wpc; sh.part_r[warp] = wr; sh.part_S[warp] = wS; }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double dsum = 0.0, rsum = 0.0;
  float Pc = 0.f, Sx = 0.f;
  for (int w = 0; w < kResolveWarps; ++w) {
    dsum += sh.part_d[w]; rsum += sh.part_r[w];
    Pc = __fadd_ru(Pc, sh.part_pc[w]); Sx = __fadd_ru(Sx, sh.part_S[w]);
  }
  const float g = gamma32_up((float)K, p.u_acc);
  const float g24 = gamma32_up((float)K, 0x1p-24f);
  const float genc = gamma32_up((float)BM, 0x1p-24f);  // rounding of e^T A, a binary32 sum over 128 rows
  double cpred = (double)alpha * dsum;
  float cin_abs = 0.f;
  if (beta_nz) {
    cpred += (double)p.beta * pe.cin_sum[cidx];
    cin_abs = pe.cin_abs[cidx];
  }
  const double dcol = sh.cref - cpred;
  // C^c_ref carries the accumulation error gamma_K(u_acc) P_c; C^c (binary32 dot of e^T A
  // with B) adds gamma_K(2^-24) P_c, and e^T A itself, a binary32 sum, gamma_128(2^-24)
  // P_c; 2^-22 P_c covers the alpha side of the output rounding, the cross terms and the
  // binary64 operations. 2^-23 sum|C| is the compensated column sum; the beta side, 34 x
  // 2^-23 |beta| sum|C_in|, covers the per-warp binary32 C_in sums over 32 rows
  // (gamma_31(2^-24)), beta C_in and the output's multiply-add (2 x 2^-24): 33 x 2^-24,
  // doubled.
  const float prod = __fmul_ru(__fmul_ru(fabsf(alpha), Pc), __fadd_ru(__fadd_ru(__fadd_ru(g, g24), 0x1p-22f), genc));
  const float outp = __fmul_ru(0x1p-23f, __fadd_ru(sh.cref_abs, __fmul_ru(__fmul_ru(fabsf(p.beta), cin_abs), 34.0f)));
  const double tauc = (double)__fadd_ru(prod, outp);
  pe.col_delta[cidx] = dcol;
  pe.col_tau[cidx] = tauc;
  pe.col_flag[cidx] = (!(fabs(dcol) <= tauc) || isinf(dcol)) ? 1 : 0;
  if (kRecompute) {
    const double rec = (double)alpha * rsum;
    const double cij = (double)p.C[gi + gj * p.ldc];
    // the recomputation is a binary32 dot product: its rounding, gamma_K(2^-24) S, joins the
    // accumulation's gamma_K(u_acc) S; 2^-23 |C| covers the output's rounding (2^-24,
    // doubled) and 2^-30 S the cross term and the binary64 operations
    const float te = __fadd_ru(__fmul_ru(__fmul_ru(fabsf(alpha), Sx), __fadd_ru(__fadd_ru(g, g24), 0x1p-30f)),
                               __fmul_ru(0x1p-23f, (float)fabs(cij)));
    const double dd = cij - rec;
    pe.elem_flag[cidx] = (!(fabs(dd) <= (double)te) || isinf(dd)) ? 1 : 0;
  }
}

// Classification of one mismatching tile (Section V.A locate, Section VI.C correct):
// one row and one column mismatching locate the error; one row and no column with beta == 0
// falls back to the row recompute; no column otherwise means a fault in the checksum path
// (C kept); anything else is uncorrectable. The located element is corrected from the row
// checksum, C(i,j) = C^r(i) - sum_{j' != j} C(i,j'): equal to C(i,j) - delta_row in exact
// arithmetic, and it never touches the erroneous value.
__device__ void resolve_tile(const TcParams& p, TcPendingEntry& pe, ResolveShared& sh, int mt, int nt, int m0,
                             int n0, int nJ, bool beta_nz) {
  const int c = threadIdx.x, lane = threadIdx.x & 31;
  if (c == 0) { sh.first_col = INT_MAX; sh.first_elem = INT_MAX; }
  __syncthreads();
  const bool cf = c < nJ && __ldcg(&pe.col_flag[c]) != 0;
  if (cf) atomicMin(&sh.first_col, c);
  const int nc = __syncthreads_count(cf);
  const int nr = pe.nr;
  const bool recompute_row = nr == 1 && nc == 0 && !beta_nz;
  const bool ef = recompute_row && c < nJ && __ldcg(&pe.elem_flag[c]) != 0;
  if (ef) atomicMin(&sh.first_elem, c);
  const int ne = __syncthreads_count(ef);
  int located = -1;
  if (nr == 1 && nc == 1) located = sh.first_col;
  else if (recompute_row && ne == 1) located = sh.first_elem;
  if (c >= 32) return;
  const int64_t gi = m0 + pe.first_row;
  double rest = 0.0;
  if (located >= 0)
    for (int j = lane; j < nJ; j += 32)
      if (j != located) rest += (double)__ldcg(&p.C[gi + (int64_t)(n0 + j) * p.ldc]);
  rest = warp_sum_f64(rest);
  if (lane != 0) return;
  int kind;
  double before = 0.0, after = 0.0, dcol = 0.0, tcol = 0.0;
  int64_t gj = -1;
  if (nc > 0) {
    gj = n0 + sh.first_col;
    dcol = __ldcg(&pe.col_delta[sh.first_col]);
    tcol = __ldcg(&pe.col_tau[sh.first_col]);
  }
  if (located >= 0) {
    kind = FT_KIND_CORRECTED;
    gj = n0 + located;
    float* cp = p.C + gi + gj * p.ldc;
    before = (double)__ldcg(cp);
    const float fixed = (float)(pe.pred_row - rest);
    *cp = fixed;
    if (p.Cb != nullptr) p.Cb[gi + gj * p.ldcb] = __bfloat16_as_ushort(__float2bfloat16_rn(fixed));
    after = (double)fixed;
  } else if (nc == 0 && (!recompute_row || ne == 0)) {
    kind = FT_KIND_CHECKSUM_ONLY;
  } else {
    kind = FT_KIND_UNCORRECTABLE;
  }
  const int ncols_rep = nc > 0 ? nc : (recompute_row ? ne : 0);
  tc_record(p, kind, mt, nt, gi, gj, pe.delta_row, dcol, pe.tau_row, tcol, before, after, nr, ncols_rep);
  count_kind(p, kind);
}

template <int KIND>
__global__ void __launch_bounds__(kResolveWarps * 32) tc_resolve_kernel(const __grid_constant__ TcParams p) {
  __shared__ ResolveShared sh;
  const float alpha = alpha_eff(p);
  constexpr int kResolveItems = tc_bn_prot(KIND);  // one column of a pending tile per work item
  const unsigned npend = min(*reinterpret_cast<volatile const unsigned*>(&p.pend->count), (unsigned)kTcPendCap);
  const int items = (int)npend * kResolveItems;
  const bool beta_nz = p.beta != 0.0f;
  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    TcPendingEntry& pe = p.pend->e[item / kResolveItems];
    const int cidx = item % kResolveItems;
    const int mt = pe.mt, nt = pe.nt;
    const int m0 = mt * BM, n0 = nt * kResolveItems;
    const int nI = min(BM, p.M - m0), nJ = min(kResolveItems, p.N - n0);
    if (cidx < nJ) {
      if (pe.nr == 1 && !beta_nz) resolve_column<true, KIND>(p, alpha, pe, sh, mt, m0, n0, nI, cidx, beta_nz);
      else resolve_column<false, KIND>(p, alpha, pe, sh, mt, m0, n0, nI, cidx, beta_nz);
    }
    if (threadIdx.x == 0) {
      __threadfence();  // this column's results before the arrival on the tile counter
      sh.last = (atomicAdd(&pe.done, 1u) == (unsigned)(kResolveItems - 1)) ? 1 : 0;
    }
    __syncthreads();
    if (sh.last) {
      __threadfence();
      resolve_tile(p, pe, sh, mt, nt, m0, n0, nJ, beta_nz);
    }
    __syncthreads();  // the shared state is reused by the next item
  }
}

// C = beta C over an M x N column-major FP32 matrix (beta == 0 writes zeros: C is not read).
__global__ void scale_f32_kernel(float* C, int64_t ldc, int32_t M, int32_t N, float beta) {
  const int64_t total = (int64_t)M * N;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % M, j = e / M;
    float* c = C + i + j * ldc;
    *c = beta == 0.0f ? 0.0f : beta * *c;
  }
}

}  // namespace

cudaError_t launch_scale_f32(float* C, int64_t ldc, int64_t M, int64_t N, float beta, cudaStream_t st) {
  if (M == 0 || N == 0) return cudaSuccess;
  const int64_t total = M * N;
  const int64_t blocks = (total + 255) / 256;
  scale_f32_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(C, ldc, (int32_t)M, (int32_t)N, beta);
  return cudaGetLastError();
}

template <bool FT, int KIND>
static cudaError_t launch_gemm_kind(const TcParams& p, const TcMaps& m, int cg, int sms, cudaStream_t st) {
  const int bn = TcGeom<FT, KIND>::BN;
  const long long nMb = (p.M + BM - 1) / BM, nNb = (p.N + bn - 1) / bn;
  const bool cb = p.Cb != nullptr;
  if (cb && cg != 2) return cudaErrorInvalidValue;
  cudaError_t e;
  if (cg == 2) {
    auto kern = cb ? tc_gemm_pair_kernel<FT, KIND, true> : tc_gemm_pair_kernel<FT, KIND, false>;
    const size_t smem = sizeof(TcSmem<2>);
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2; attr[0].val.clusterDim.y = 1; attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((unsigned)(sms / 2 * 2), 1, 1);
    cfg.blockDim = dim3(NTHREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // CTA pairs resident at once (one per TPC when nothing else occupies the GPU)
    static int max_clusters[2][2][2] = {};
    int& mc = max_clusters[FT ? 1 : 0][KIND][cb ? 1 : 0];
    if (mc == 0) {
      e = cudaOccupancyMaxActiveClusters(&mc, kern, &cfg);
      if (e != cudaSuccess) return e;
      if (mc <= 0) return cudaErrorInvalidConfiguration;
    }
    const long long units = (nMb + 1) / 2 * nNb;
    cfg.gridDim = dim3((unsigned)(2 * (units < mc ? units : mc)), 1, 1);
    kernel_timer_start(st);
    e = cudaLaunchKernelEx(&cfg, kern, m.a, m.b, m.b2, m.chk, p);
    kernel_timer_stop(st);
    if (e == cudaSuccess) e = cudaGetLastError();
  } else {
    const size_t smem = sizeof(TcSmem<1>);
    const long long tiles = nMb * nNb;
    const int grid = (int)(tiles < sms ? tiles : sms);
    e = cudaFuncSetAttribute(tc_gemm_kernel<FT, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kernel_timer_start(st);
    tc_gemm_kernel<FT, KIND><<<grid, NTHREADS, smem, st>>>(m.a, m.b, m.chk, p);
    kernel_timer_stop(st);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess || !FT) return e;
  tc_colsum_kernel<KIND><<<(unsigned)((p.K + kColsumK - 1) / kColsumK), 256, 0, st>>>(p);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  tc_resolve_kernel<KIND><<<2 * sms, kResolveWarps * 32, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_tc_gemm(const TcParams& p, const TcMaps& m, bool ft, int cg, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (p.kind == 0) return ft ? launch_gemm_kind<true, 0>(p, m, cg, sms, st) : launch_gemm_kind<false, 0>(p, m, cg, sms, st);
  return ft ? launch_gemm_kind<true, 1>(p, m, cg, sms, st) : launch_gemm_kind<false, 1>(p, m, cg, sms, st);
}

}  // namespace ftk
