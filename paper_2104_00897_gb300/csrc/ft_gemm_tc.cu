// Reduced-precision ABFT-protected GEMM on the fifth-generation tensor cores (sm_103a):
// BF16 operands, FP32 accumulation in TMEM, FP32 output, FP64 checksum comparison.
//
// FT-BLAS (Zhai et al., ICS '21) has no reduced precision; the checksum relations are those
// of Section II.A, the lazy second side that of Section V.A, and C = beta*C is folded into
// the checksums as in Section V.B.
//
// Structure (persistent: one CTA of 192 threads per SM loops over output tiles; the
// tensor-core tile is 128 x 256 and the TMEM accumulator is double-buffered):
//   warp 0      TMA producer: A (128 x 64) and B (N_data x 64) k-tiles into a 4-stage ring,
//               128-byte swizzled, K-major. Protected launches put the checksum column of
//               B^r = [B, Be] (Section II.A) into rows 240..255 of the same B stage: Be over
//               the tile's 240 data columns, split into three BF16 pieces (hi, mid, lo) by a
//               bandwidth-bound encode pre-pass.
//   warp 1      TMEM allocation and MMA issue (one thread): 4 x tcgen05.mma M128 N256 K16 per
//               k-tile into one of two 256-column TMEM buffers, so the next tile's product
//               overlaps the previous tile's epilogue. With the checksum column appended, the
//               tensor core produces C^r = A (B e) in columns 240..242 with the product
//               itself, at no extra instruction (6.7 % fewer data columns per tile).
//   warps 2..5  epilogue, one TMEM lane (= output row) per thread: C = alpha acc + beta C_in
//               stored in FP32; C^r_ref(i) = sum_j C(i,j) in compensated binary32, compared
//               in binary64 with the predicted checksum against a rigorous bound. Only in a
//               tile with a mismatching row are the column checksums formed (C^c_ref from
//               the stored tile, C^c = (e^T A) B from global memory in binary32)
//               to locate the error; when the columns cannot locate it (rows of very
//               different scale), the mismatching row is recomputed and compared element by
//               element. The located element is corrected from the row checksum.
#include <climits>

#include <cuda_bf16.h>

#include "ft_device.cuh"
#include "ft_internal.h"
#include "ft_tc.h"

namespace ftk {

namespace {

constexpr int BM = kTcBM;            // 128 tile rows (TMEM lanes)
constexpr int BNM = 256;             // MMA N = TMEM columns = B stage rows
constexpr int BKB = 128;             // k-tile depth in bytes (64 BF16)
constexpr int STAGES = 4;
constexpr int NTHREADS = 192;
constexpr int CHK_ROWS = kTcChkRows;  // 16
constexpr uint32_t TMEM_COLS = 512;   // two accumulator buffers of 256 columns
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s per wait; a whole tile takes ~0.1 ms

template <bool FT>
struct TcGeom {
  static constexpr int BN = FT ? kTcBNProt : BNM;  // data columns per tile
};

struct __align__(1024) TcSmem {
  uint8_t a[STAGES][BM * BKB];
  uint8_t b[STAGES][BNM * BKB];
  uint64_t full[STAGES];
  uint64_t empty[STAGES];
  uint64_t tfull[2];             // accumulator buffer b holds a finished tile
  uint64_t tempty[2];            // accumulator buffer b has been read by the 4 epilogue warps
  uint32_t tmem_base;
  int timeout;
  int nflag_rows, first_row, nflag_cols, first_col, nflag_elem, first_elem;
  double delta_row, tau_row, delta_col, tau_col;
  double pred_row;               // predicted row checksum of the first flagged row
  float cin_col[4][BNM];         // per-warp partial column sums of C_in (beta != 0)
  float cin_col_abs[4][BNM];
  double col_delta[BNM];         // lazy column side: C^c_ref - C^c and tau per column
  double col_tau[BNM];
};

__device__ __forceinline__ float bf16_to_f32(uint16_t b) { return __uint_as_float(static_cast<uint32_t>(b) << 16); }

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
__device__ __noinline__ float inject_element(const TcParams& p, int64_t gi, int64_t gj, float acc, float cin,
                                             bool beta_nz) {
  for (int e = 0; e < p.inj.n; ++e) {
    const InjectPoint& ip = p.inj.p[e];
    if (ip.i == gi && ip.j == gj && ip.site == kSiteAccum && ip.mode == FT_MODE_BITFLIP)
      acc = __uint_as_float(__float_as_uint(acc) ^ (1u << ip.bit));
  }
  float out = beta_nz ? fmaf(p.alpha, acc, p.beta * cin) : p.alpha * acc;
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

// Persistent-tile order: groups of kGroupM row tiles sweep all column tiles, so the CTAs
// resident at one time share A row panels and B column panels in L2.
constexpr int kGroupM = 16;
__device__ __forceinline__ void tile_coords(int t, int nMb, int nNb, int& mt, int& nt) {
  const int group = t / (kGroupM * nNb);
  const int first_m = group * kGroupM;
  const int gsize = min(kGroupM, nMb - first_m);
  const int in_group = t - group * kGroupM * nNb;
  mt = first_m + in_group % gsize;
  nt = in_group / gsize;
}

// Persistent kernel: one CTA per SM loops over output tiles. The TMEM accumulator is double
// buffered (2 x 256 columns): while the epilogue warps verify and store tile t from one
// buffer, the MMA warp accumulates tile t+1 into the other.
template <bool FT>
__global__ void __launch_bounds__(NTHREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ CUtensorMap tmChk, const __grid_constant__ TcParams p) {
  constexpr int BN = TcGeom<FT>::BN;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  TcSmem& sm = *reinterpret_cast<TcSmem*>(smem_raw);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int bk_elems = BKB / 2;
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
      const uint32_t bytes = (BM + BN + (FT ? CHK_ROWS : 0)) * BKB;
      uint32_t it = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        int mt, nt;
        tile_coords(tile, nMb, nNb, mt, nt);
        for (int kt = 0; kt < nk; ++kt, ++it) {
          const uint32_t s = it % STAGES, u = it / STAGES;
          if (u > 0 && !mbar_wait_bounded(&sm.empty[s], (u - 1) & 1, kWaitLimitNs)) { sm.timeout = 1; ok = false; break; }
          mbar_arrive_expect_tx(&sm.full[s], bytes);
          const int k0 = kt * bk_elems;
          tma_load_2d(sm.a[s], &tmA, &sm.full[s], k0, mt * BM);
          tma_load_2d(sm.b[s], &tmB, &sm.full[s], k0, nt * BN);
          if (FT) tma_load_2d(sm.b[s] + BN * BKB, &tmChk, &sm.full[s], k0, nt * CHK_ROWS);
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issue
    if (lane == 0) {
      const uint32_t idesc = umma_idesc(1, 1, BM, BNM);
      uint32_t it = 0, lt = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++lt) {
        const uint32_t b = lt & 1, ub = lt >> 1;
        if (ub > 0 && !mbar_wait_bounded(&sm.tempty[b], (ub - 1) & 1, kWaitLimitNs)) { sm.timeout = 1; break; }
        tc_fence_after();
        const uint32_t dcol = tmem + b * BNM;
        for (int kt = 0; kt < nk; ++kt, ++it) {
          const uint32_t s = it % STAGES, u = it / STAGES;
          if (!mbar_wait_bounded(&sm.full[s], u & 1, kWaitLimitNs)) { sm.timeout = 1; ok = false; break; }
          tc_fence_after();
          const uint32_t a0 = smem_addr(sm.a[s]), b0 = smem_addr(sm.b[s]);
#pragma unroll
          for (int kk = 0; kk < BKB / 32; ++kk)
            umma_bf16(dcol, umma_desc_sw128(a0 + kk * 32), umma_desc_sw128(b0 + kk * 32), idesc,
                      (kt > 0 || kk > 0) ? 1u : 0u);
          umma_commit(&sm.empty[s]);
        }
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
    uint32_t lt = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++lt) {
      int mt, nt;
      tile_coords(tile, nMb, nNb, mt, nt);
      const int m0 = mt * BM, n0 = nt * BN;
      const int nI = min(BM, p.M - m0), nJ = min(BN, p.N - n0);
      const int64_t gi = m0 + row;
      const bool row_ok = row < nI;
      const uint32_t b = lt & 1, ub = lt >> 1;
      // tcgen05.ld is warp-collective (.sync.aligned): every TMEM load below is executed by
      // all 32 lanes of the warp, whatever their row; `got` is made warp-uniform for that.
      const bool got = __all_sync(0xffffffffu, mbar_wait_bounded(&sm.tfull[b], ub & 1, kWaitLimitNs));
      if (!got) sm.timeout = 1;
      tc_fence_after();
      const uint32_t trow = tmem + b * BNM + (static_cast<uint32_t>(q * 32) << 16);
      float rs = 0.f, rc = 0.f, rabs = 0.f;   // compensated sum of C over the row, upward |C| sum
      float cs = 0.f, cc = 0.f, cabs = 0.f;   // same for C_in
      uint32_t w4[4] = {0u, 0u, 0u, 0u};
      // Injection points in this tile (test launches only): the per-element injection code
      // is kept out of the hot loop so the epilogue stays small in the instruction cache,
      // which it shares with the producer and MMA warps.
      bool tile_inj = false;
      if (FT)
        for (int e = 0; e < p.inj.n; ++e)
          tile_inj |= p.inj.p[e].i >= m0 && p.inj.p[e].i < m0 + nI && p.inj.p[e].j >= n0 && p.inj.p[e].j < n0 + nJ;
      if (got) {
#pragma unroll 1
        for (int ch = 0; ch < (BN + 7) / 8; ++ch) {
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
            if (FT && tile_inj) out = inject_element(p, gi, gj, acc, cin, beta_nz);
            else out = beta_nz ? fmaf(p.alpha, acc, p.beta * cin) : p.alpha * acc;
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
        if (FT) {
          __syncwarp();
          tmem_ld4(trow + BN, w4);  // C^r pieces from the checksum column of B^r
          tmem_ld_wait();
        }
      }
      // The accumulator buffer is free for the MMA warp's next-but-one tile.
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&sm.tempty[b]);
      if (!FT) continue;

      // -------------------------------------------------------- row verification
      if (et == 0) {
        sm.nflag_rows = 0; sm.first_row = INT_MAX; sm.nflag_cols = 0; sm.first_col = INT_MAX;
        sm.nflag_elem = 0; sm.first_elem = INT_MAX;
      }
      named_bar(1, 128);
      double delta = 0.0, tau = 0.0, predicted = 0.0;
      if (got && row_ok) {
        const double pr = (double)__uint_as_float(w4[0]) + (double)__uint_as_float(w4[1]) +
                          (double)__uint_as_float(w4[2]);
        const double cin_sum = (double)cs + (double)cc;
        predicted = (double)p.alpha * pr + (beta_nz ? (double)p.beta * cin_sum : 0.0);
        for (int e = 0; e < p.inj.n; ++e) {
          const InjectPoint& ip = p.inj.p[e];
          if (ip.site == kSiteChecksumRow && ip.i == gi && ip.j >= n0 && ip.j < n0 + nJ) {
            const double em = ldexp(fabs(predicted), ip.rel_log2);
            predicted = ip.sign < 0 ? predicted - em : predicted + em;
          }
        }
        const double ref = (double)rs + (double)rc;
        delta = ref - predicted;
        // tau = |alpha| P (gamma_K(u_acc) (2 + 2^-7) + 2^-20) + 2 u32 (sum|C| + |beta| sum|C_in|), P an
        // upper bound of sum_k |A(i,k)| sum_{j in tile} |B(k,j)|.
        const float P = __fmul_ru(p.rowAbsA[gi], p.maxAbsBe[nt]);
        const float g = gamma32_up((float)p.K, p.u_acc);
        const float prod = __fmul_ru(__fmul_ru(fabsf(p.alpha), P), __fadd_ru(__fmul_ru(g, 2.0078125f), 0x1p-20f));
        const float outp = __fmul_ru(0x1p-23f, __fadd_ru(rabs, __fmul_ru(fabsf(p.beta), cabs)));
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
        // ------------------------------------------------------ lazy column side (Section V.A)
        // Each warp takes columns ew, ew + 4, ...; its lanes split the rows (C^c_ref) and K
        // (C^c = alpha (e^T A) B(:, j), compensated); partial results are summed in binary64.
        const uint16_t* Bp = static_cast<const uint16_t*>(p.B);
        const float2* sAI = p.sA + (int64_t)mt * p.K;
        const float* absAI = p.absSA + (int64_t)mt * p.K;
        const float g = gamma32_up((float)p.K, p.u_acc);
        const float g24 = gamma32_up((float)p.K, 0x1p-24f);
        for (int cidx = ew; cidx < nJ; cidx += 4) {
          const int64_t gj = n0 + cidx;
          float s = 0.f, c = 0.f, a = 0.f;
          for (int i = lane; i < nI; i += 32) {
            const float x = p.C[(int64_t)(m0 + i) + gj * p.ldc];
            neumaier(s, c, x);
            a = __fadd_ru(a, fabsf(x));
          }
          const double cref = warp_sum_f64((double)s + (double)c);
          const float cref_abs = warp_sum_up(a);
          // binary32 dot products with two independent accumulators (their rounding enters
          // the threshold as gamma_K(2^-24) P_c, next to the accumulation's gamma_K(u_acc) P_c)
          const uint16_t* bcol = Bp + gj * p.ldb;
          float d0 = 0.f, d1 = 0.f, pc0 = 0.f, pc1 = 0.f;
          int k = lane;
          for (; k + 32 < p.K; k += 64) {
            const float b0 = bf16_to_f32(bcol[k]), b1 = bf16_to_f32(bcol[k + 32]);
            d0 = fmaf(sAI[k].x, b0, d0);
            d1 = fmaf(sAI[k + 32].x, b1, d1);
            pc0 = __fmaf_ru(absAI[k], fabsf(b0), pc0);  // sum_k (sum_i |A(i,k)|) |B(k,j)|, upward
            pc1 = __fmaf_ru(absAI[k + 32], fabsf(b1), pc1);
          }
          if (k < p.K) {
            const float b0 = bf16_to_f32(bcol[k]);
            d0 = fmaf(sAI[k].x, b0, d0);
            pc0 = __fmaf_ru(absAI[k], fabsf(b0), pc0);
          }
          double cpred = (double)p.alpha * warp_sum_f64((double)d0 + (double)d1);
          const float Pc = warp_sum_up(__fadd_ru(pc0, pc1));
          float cin_abs = 0.f;
          if (beta_nz) {
            double cin_sum = 0.0;
            for (int w = 0; w < 4; ++w) { cin_sum += (double)sm.cin_col[w][cidx]; cin_abs = __fadd_ru(cin_abs, sm.cin_col_abs[w][cidx]); }
            cpred += (double)p.beta * cin_sum;
          }
          if (lane == 0) {
            const double dcol = cref - cpred;
            // C^c_ref carries the accumulation error gamma_K(u_acc) P_c; C^c (binary32 dot of
            // the rounded e^T A with B) adds gamma_K(2^-24) P_c + 2^-23 P_c; the per-warp C_in
            // partial sums carry gamma_31 (binary32).
            const float prod = __fmul_ru(__fmul_ru(fabsf(p.alpha), Pc), __fadd_ru(__fadd_ru(g, g24), 0x1p-22f));
            const float outp =
                __fmul_ru(0x1p-23f, __fadd_ru(cref_abs, __fmul_ru(__fmul_ru(fabsf(p.beta), cin_abs), 34.0f)));
            const double tauc = (double)__fadd_ru(prod, outp);
            sm.col_delta[cidx] = dcol;
            sm.col_tau[cidx] = tauc;
            if (!(fabs(dcol) <= tauc) || isinf(dcol)) {
              atomicAdd(&sm.nflag_cols, 1);
              atomicMin(&sm.first_col, cidx);
            }
          }
        }
        __threadfence_block();
        named_bar(1, 128);
        const int nc = sm.nflag_cols;
        if (nc > 0 && et == 0) { sm.delta_col = sm.col_delta[sm.first_col]; sm.tau_col = sm.col_tau[sm.first_col]; }
        // ------------------------------------------------------ row-recompute locator
        // One mismatching row and no mismatching column: the column checksums of a tile
        // whose rows differ greatly in scale cannot resolve an error in a small row. Then
        // recompute that row and compare each element with its own bound
        // |alpha| (gamma_K(u_acc) + gamma_K(2^-24) + 2^-30) sum_k |A(i,k)||B(k,j)| + 2^-23 |C(i,j)|.
        const bool recompute_row = (nr == 1 && nc == 0 && !beta_nz);
        if (recompute_row) {
          const int64_t gr = m0 + sm.first_row;
          const uint16_t* arow = static_cast<const uint16_t*>(p.A) + gr * p.lda;
          for (int cidx = ew; cidx < nJ; cidx += 4) {
            const int64_t gj = n0 + cidx;
            const uint16_t* bcol = Bp + gj * p.ldb;
            float d0 = 0.f, d1 = 0.f, s0 = 0.f, s1 = 0.f;
            int k = lane;
            for (; k + 32 < p.K; k += 64) {
              const float a0 = bf16_to_f32(arow[k]), b0 = bf16_to_f32(bcol[k]);
              const float a1 = bf16_to_f32(arow[k + 32]), b1 = bf16_to_f32(bcol[k + 32]);
              d0 = fmaf(a0, b0, d0);
              d1 = fmaf(a1, b1, d1);
              s0 = __fmaf_ru(fabsf(a0), fabsf(b0), s0);
              s1 = __fmaf_ru(fabsf(a1), fabsf(b1), s1);
            }
            if (k < p.K) {
              const float a0 = bf16_to_f32(arow[k]), b0 = bf16_to_f32(bcol[k]);
              d0 = fmaf(a0, b0, d0);
              s0 = __fmaf_ru(fabsf(a0), fabsf(b0), s0);
            }
            const double rec = (double)p.alpha * warp_sum_f64((double)d0 + (double)d1);
            const float S = warp_sum_up(__fadd_ru(s0, s1));
            if (lane == 0) {
              const double cij = (double)p.C[gr + gj * p.ldc];
              // the recomputation is a binary32 dot product: its rounding, gamma_K(2^-24) S,
              // joins the accumulation's gamma_K(u_acc) S
              const float te = __fadd_ru(__fmul_ru(__fmul_ru(fabsf(p.alpha), S), __fadd_ru(__fadd_ru(g, g24), 0x1p-30f)),
                                         __fmul_ru(0x1p-23f, (float)fabs(cij)));
              const double d = cij - rec;
              if (!(fabs(d) <= (double)te) || isinf(d)) {
                atomicAdd(&sm.nflag_elem, 1);
                atomicMin(&sm.first_elem, cidx);
              }
            }
          }
          __threadfence_block();
          named_bar(1, 128);
        }
        if (et == 0) {
          int kind;
          double before = 0.0, after = 0.0;
          const int64_t gi2 = m0 + sm.first_row;
          int located_col = -1;
          if (nr == 1 && nc == 1) located_col = sm.first_col;
          else if (recompute_row && sm.nflag_elem == 1) located_col = sm.first_elem;
          int64_t gj2 = (nc > 0) ? n0 + sm.first_col : -1;
          if (located_col >= 0) {
            kind = FT_KIND_CORRECTED;
            gj2 = n0 + located_col;
            float* cp = p.C + gi2 + gj2 * p.ldc;
            before = (double)*cp;
            // The paper's correction, C(i,j) - delta_row, evaluated as
            // C^r(i) - sum_{j' != j} C(i,j'): equal in exact arithmetic, and it never touches
            // the erroneous value (no cancellation against a huge or non-finite error).
            double rest = 0.0;
            for (int j = 0; j < nJ; ++j)
              if (n0 + j != gj2) rest += (double)p.C[gi2 + (int64_t)(n0 + j) * p.ldc];
            after = sm.pred_row - rest;
            *cp = (float)after;
            after = (double)*cp;
          } else if (nc == 0 && (!recompute_row || sm.nflag_elem == 0)) {
            kind = FT_KIND_CHECKSUM_ONLY;
          } else {
            kind = FT_KIND_UNCORRECTABLE;
          }
          const int ncols_rep = nc > 0 ? nc : (recompute_row ? sm.nflag_elem : 0);
          tc_record(p, kind, mt, nt, gi2, gj2, sm.delta_row, nc > 0 ? sm.delta_col : 0.0, sm.tau_row,
                    nc > 0 ? sm.tau_col : 0.0, before, after, nr, ncols_rep);
          if (p.report) {
            atomicAdd(reinterpret_cast<unsigned long long*>(&p.report->detected), 1ull);
            unsigned long long* ctr = (kind == FT_KIND_CORRECTED)
                                          ? reinterpret_cast<unsigned long long*>(&p.report->corrected)
                                      : (kind == FT_KIND_CHECKSUM_ONLY)
                                          ? reinterpret_cast<unsigned long long*>(&p.report->checksum_only)
                                          : reinterpret_cast<unsigned long long*>(&p.report->uncorrectable);
            atomicAdd(ctr, 1ull);
          }
        }
      }
      if (et == 0 && p.report) atomicAdd(reinterpret_cast<unsigned long long*>(&p.report->tiles_checked), 1ull);
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

// ---------------------------------------------------------------------------------------
// Encode pre-pass (bandwidth-bound). Kernel-frame A is M x K and B is K x N, both
// K-contiguous (row i of A at A + i*lda, column j of B at B + j*ldb). One thread per pair
// of consecutive k; loads are 4-byte BF16 pairs, coalesced along k.
// ---------------------------------------------------------------------------------------
constexpr int ENC_KC = 512;   // k per CTA (256 threads x 2)

__device__ __forceinline__ void load_pair(const uint16_t* row, int64_t k, int32_t K, float& x0, float& x1) {
  // k is even; the pair (k, k+1) is 4-byte aligned because leading dimensions are multiples
  // of 8 elements and base addresses are 16-byte aligned.
  if (k + 1 < K) {
    const uint32_t w = *reinterpret_cast<const uint32_t*>(row + k);
    x0 = __uint_as_float(w << 16);
    x1 = __uint_as_float(w & 0xffff0000u);
  } else {
    x0 = (k < K) ? bf16_to_f32(row[k]) : 0.f;
    x1 = 0.f;
  }
}

// Per 128-row block I: e^T A over the block for each k (hi + lo binary32 pair,
// compensated) and the upward sum of |A| over the block for each k. Streaming, one thread
// per pair of k, no cross-thread reduction.
__global__ void __launch_bounds__(256) encode_rows_kernel(const uint16_t* A, int64_t lda, int32_t M, int32_t K,
                                                           float2* sA, float* absSA) {
  const int I = blockIdx.x;
  const int m0 = I * BM;
  const int nI = min(BM, M - m0);
  const int64_t k = (int64_t)blockIdx.y * ENC_KC + 2 * threadIdx.x;
  if (k >= K) return;
  float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f, a0 = 0.f, a1 = 0.f;
  for (int i = 0; i < nI; ++i) {
    float x0, x1;
    load_pair(A + (int64_t)(m0 + i) * lda, k, K, x0, x1);
    neumaier(s0, c0, x0);
    neumaier(s1, c1, x1);
    a0 = __fadd_ru(a0, fabsf(x0));
    a1 = __fadd_ru(a1, fabsf(x1));
  }
  float h = s0 + c0;
  sA[(int64_t)I * K + k] = make_float2(h, c0 - (h - s0));
  absSA[(int64_t)I * K + k] = a0;
  if (k + 1 < K) {
    h = s1 + c1;
    sA[(int64_t)I * K + k + 1] = make_float2(h, c1 - (h - s1));
    absSA[(int64_t)I * K + k + 1] = a1;
  }
}

// Upward sum_k |A(i,k)| per row: one warp per row, 16-byte loads along the row.
__global__ void __launch_bounds__(256) row_abs_kernel(const uint16_t* A, int64_t lda, int32_t M, int32_t K,
                                                       float* rowAbsA) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * 8 + warp;
  if (i >= M) return;
  const uint16_t* row = A + i * lda;
  float a = 0.f;
  const int K8 = K & ~7;
  for (int k = lane * 8; k < K8; k += 256) {
    const uint4 w = *reinterpret_cast<const uint4*>(row + k);  // rows are 16-byte aligned
    const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      a = __fadd_ru(a, fabsf(__uint_as_float(ws[h] << 16)));
      a = __fadd_ru(a, fabsf(__uint_as_float(ws[h] & 0xffff0000u)));
    }
  }
  for (int k = K8 + lane; k < K; k += 32) a = __fadd_ru(a, fabsf(bf16_to_f32(row[k])));
  a = warp_sum_up(a);
  if (lane == 0) rowAbsA[i] = a;
}

// Per block J of `bn` columns: B e over the block for each k, split into three BF16 pieces
// written to rows J*16 + {0, 1, 2} of the checksum operand (K-contiguous, pitch kpitch),
// and max_k of the upward |B| sum over the block (maxAbsBe[J]). Streaming, one thread per
// pair of k.
__global__ void __launch_bounds__(256) encode_cols_kernel(const uint16_t* B, int64_t ldb, int32_t N, int32_t K,
                                                           int32_t bn, uint16_t* chk, int64_t kpitch, float* maxAbsBe) {
  const int J = blockIdx.x;
  const int n0 = J * bn;
  const int nJ = min(bn, N - n0);
  const int64_t k = (int64_t)blockIdx.y * ENC_KC + 2 * threadIdx.x;
  float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f, a0 = 0.f, a1 = 0.f;
  if (k < K) {
    for (int j = 0; j < nJ; ++j) {
      float x0, x1;
      load_pair(B + (int64_t)(n0 + j) * ldb, k, K, x0, x1);
      neumaier(s0, c0, x0);
      neumaier(s1, c1, x1);
      a0 = __fadd_ru(a0, fabsf(x0));
      a1 = __fadd_ru(a1, fabsf(x1));
    }
    auto split_store = [&](float s, float c, int64_t kk) {
      // three bfloat16 pieces, each the nearest bfloat16 of the remainder of s + c
      const float x = s + c;
      const float xr = c - (x - s);
      const __nv_bfloat16 h = __float2bfloat16_rn(x);
      const float r1 = (x - __bfloat162float(h)) + xr;
      const __nv_bfloat16 m = __float2bfloat16_rn(r1);
      const float r2 = r1 - __bfloat162float(m);
      const __nv_bfloat16 l = __float2bfloat16_rn(r2);
      chk[(int64_t)(J * CHK_ROWS + 0) * kpitch + kk] = __bfloat16_as_ushort(h);
      chk[(int64_t)(J * CHK_ROWS + 1) * kpitch + kk] = __bfloat16_as_ushort(m);
      chk[(int64_t)(J * CHK_ROWS + 2) * kpitch + kk] = __bfloat16_as_ushort(l);
    };
    split_store(s0, c0, k);
    if (k + 1 < K) split_store(s1, c1, k + 1);
  }
  float mx = fmaxf(k < K ? a0 : 0.f, k + 1 < K ? a1 : 0.f);
#pragma unroll
  for (int w = 16; w >= 1; w >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, w));
  if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<unsigned int*>(&maxAbsBe[J]), __float_as_uint(mx));
}

}  // namespace

size_t tc_workspace_bytes(int32_t M, int32_t N, int32_t K) {
  const int64_t nMb = (M + BM - 1) / BM, nNb = (N + kTcBNProt - 1) / kTcBNProt;
  const int64_t kpitch = (K + 7) / 8 * 8;
  auto up = [](int64_t x) { return (x + 255) / 256 * 256; };
  return up(nNb * CHK_ROWS * kpitch * 2) + up(nMb * (int64_t)K * 8) + up(nMb * (int64_t)K * 4) + up(M * 4) + up(nNb * 4);
}

TcWorkspace tc_workspace_carve(void* base, int32_t M, int32_t N, int32_t K) {
  const int64_t nMb = (M + BM - 1) / BM, nNb = (N + kTcBNProt - 1) / kTcBNProt;
  const int64_t kpitch = (K + 7) / 8 * 8;
  auto up = [](int64_t x) { return (x + 255) / 256 * 256; };
  char* c = static_cast<char*>(base);
  TcWorkspace w;
  w.chk = reinterpret_cast<uint16_t*>(c); c += up(nNb * CHK_ROWS * kpitch * 2);
  w.kpitch = kpitch;
  w.sA = reinterpret_cast<float2*>(c); c += up(nMb * (int64_t)K * 8);
  w.absSA = reinterpret_cast<float*>(c); c += up(nMb * (int64_t)K * 4);
  w.rowAbsA = reinterpret_cast<float*>(c); c += up(M * 4);
  w.maxAbsBe = reinterpret_cast<float*>(c); c += up(nNb * 4);
  w.bytes = static_cast<size_t>(c - static_cast<char*>(base));
  return w;
}

cudaError_t launch_tc_encode(const TcParams& p, const TcWorkspace& w, void* ws_base, cudaStream_t st) {
  const int nMb = (p.M + BM - 1) / BM, nNb = (p.N + kTcBNProt - 1) / kTcBNProt, nkc = (p.K + ENC_KC - 1) / ENC_KC;
  // zero the checksum operand (its rows 3..15 stay zero) and the block maxima
  cudaError_t e = cudaMemsetAsync(ws_base, 0, w.bytes, st);
  if (e != cudaSuccess) return e;
  encode_rows_kernel<<<dim3(nMb, nkc), 256, 0, st>>>(static_cast<const uint16_t*>(p.A), p.lda, p.M, p.K, w.sA,
                                                      w.absSA);
  row_abs_kernel<<<(p.M + 7) / 8, 256, 0, st>>>(static_cast<const uint16_t*>(p.A), p.lda, p.M, p.K, w.rowAbsA);
  encode_cols_kernel<<<dim3(nNb, nkc), 256, 0, st>>>(static_cast<const uint16_t*>(p.B), p.ldb, p.N, p.K, kTcBNProt,
                                                      w.chk, w.kpitch, w.maxAbsBe);
  return cudaGetLastError();
}

cudaError_t launch_tc_gemm(const TcParams& p, const CUtensorMap* tmA, const CUtensorMap* tmB, const CUtensorMap* tmChk,
                           bool ft, cudaStream_t st) {
  const size_t smem = sizeof(TcSmem);
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int bn = ft ? kTcBNProt : BNM;
  const long long tiles = (long long)((p.M + BM - 1) / BM) * ((p.N + bn - 1) / bn);
  const int grid = (int)(tiles < sms ? tiles : sms);
  if (ft) {
    e = cudaFuncSetAttribute(tc_gemm_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    tc_gemm_kernel<true><<<grid, NTHREADS, smem, st>>>(*tmA, *tmB, *tmChk, p);
  } else {
    e = cudaFuncSetAttribute(tc_gemm_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    tc_gemm_kernel<false><<<grid, NTHREADS, smem, st>>>(*tmA, *tmB, *tmChk, p);
  }
  return cudaGetLastError();
}

}  // namespace ftk
