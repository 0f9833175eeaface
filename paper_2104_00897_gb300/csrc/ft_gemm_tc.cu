// Reduced-precision ABFT-protected GEMM on the fifth-generation tensor cores (sm_103a):
// BF16 operands, FP32 accumulation in TMEM, FP32 output, FP64 checksum comparison.
//
// FT-BLAS (Zhai et al., ICS '21) has no reduced precision; the checksum relations are those
// of Section II.A, the lazy second side that of Section V.A, and C = beta*C is folded into
// the checksums as in Section V.B.
//
// Structure (one 128 x 256 output tile per CTA, 192 threads):
//   warp 0      TMA producer: A (128 x 64), B (256 x 64) and the checksum operand (16 x 64)
//               k-tiles into a 4-stage ring, 128-byte swizzled, K-major;
//   warp 1      TMEM allocation and MMA issue (one thread): per k-tile 4 x
//               tcgen05.mma M128 N256 K16 into TMEM columns [0, 256) and, when protected,
//               4 x M128 N16 K16 of A against the checksum operand into columns [256, 272):
//               the row checksum C^r = A (B e) is produced by the tensor core itself;
//   warps 2..5  epilogue, one TMEM lane (= output row) per thread: C = alpha acc + beta C_in,
//               stored in FP32; the reference row checksum C^r_ref(i) = sum_j C(i,j) in
//               compensated binary32; compared in binary64 with the predicted checksum;
//               only when a row mismatches, the column checksums of the tile are formed
//               (C^c_ref from the stored tile, C^c = (e^T A) B from global memory in
//               compensated binary32) to locate the error, which is then corrected from
//               the row checksum.
// The checksum operand holds B e of the tile's 256 columns, split into three BF16 pieces
// (hi, mid, lo), prepared by a bandwidth-bound pre-pass that also forms the magnitude
// bounds for the threshold and e^T A per 128-row block for the column side.
#include <climits>

#include <cuda_bf16.h>

#include "ft_device.cuh"
#include "ft_internal.h"
#include "ft_tc.h"

namespace ftk {

namespace {

constexpr int BM = kTcBM, BN = kTcBN, BKB = 128;  // BKB: k-tile depth in bytes (64 BF16)
constexpr int STAGES = 4;
constexpr int NTHREADS = 192;
constexpr int CHK_ROWS = kTcChkRows;
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t kChkCol = 256;                  // TMEM column of the checksum accumulators
constexpr uint64_t kWaitLimitNs = 2000000000ull;   // 2 s per wait; a whole tile takes ~0.1 ms

struct __align__(1024) TcSmem {
  uint8_t a[STAGES][BM * BKB];
  uint8_t b[STAGES][BN * BKB];
  uint8_t chk[STAGES][CHK_ROWS * BKB];
  uint64_t full[STAGES];
  uint64_t empty[STAGES];
  uint64_t accum;
  uint32_t tmem_base;
  int timeout;
  int nflag_rows, first_row, nflag_cols, first_col;
  int nonfinite;
  double delta_row, tau_row, delta_col, tau_col;
  double pred_row;               // predicted row checksum of the first flagged row
  float cin_col[4][BN];          // per-warp partial column sums of C_in (beta != 0)
  float cin_col_abs[4][BN];
  double col_delta[BN];          // lazy column side: C^c_ref - C^c and tau per column
  double col_tau[BN];
};

__device__ __forceinline__ float bf16_to_f32(uint16_t b) { return __uint_as_float(static_cast<uint32_t>(b) << 16); }

// Neumaier's compensated summation step (binary32).
__device__ __forceinline__ void neumaier(float& s, float& c, float x) {
  const float t = s + x;
  c += (fabsf(s) >= fabsf(x)) ? ((s - t) + x) : ((x - t) + s);
  s = t;
}

// Error-free product a*b = p + e (binary32, via fused multiply-add).
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = a * b;
  e = fmaf(a, b, -p);
}

// Warp transpose-reduction: lane l ends with sum over lanes of v[l] (31 shuffles).
__device__ __forceinline__ float warp_column_sum(float (&v)[32], int lane) {
#pragma unroll
  for (int w = 16; w >= 1; w >>= 1) {
#pragma unroll
    for (int i = 0; i < w; ++i) {
      const bool up = (lane & w) != 0;
      const float send = up ? v[i] : v[i + w];
      const float keep = up ? v[i + w] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, w);
    }
  }
  return v[0];
}
__device__ __forceinline__ float warp_column_sum_up(float (&v)[32], int lane) {
#pragma unroll
  for (int w = 16; w >= 1; w >>= 1) {
#pragma unroll
    for (int i = 0; i < w; ++i) {
      const bool up = (lane & w) != 0;
      const float send = up ? v[i] : v[i + w];
      const float keep = up ? v[i + w] : v[i];
      v[i] = __fadd_ru(keep, __shfl_xor_sync(0xffffffffu, send, w));
    }
  }
  return v[0];
}

__device__ __forceinline__ float gamma32_up(float n, float u) {
  const float nu = __fmul_ru(n, u);
  return __fdiv_ru(nu, __fsub_rd(1.0f, nu));
}

__device__ __forceinline__ float ldg_bf16(const uint16_t* p, int64_t idx) { return bf16_to_f32(p[idx]); }

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

template <bool FT>
__global__ void __launch_bounds__(NTHREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ CUtensorMap tmChk, const __grid_constant__ TcParams p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  TcSmem& sm = *reinterpret_cast<TcSmem*>(smem_raw);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int nI = min(BM, p.M - m0), nJ = min(BN, p.N - n0);
  const int bk_elems = BKB / 2;
  const int nk = (p.K + bk_elems - 1) / bk_elems;

  if (t == 0) {
    for (int s = 0; s < STAGES; ++s) { mbar_init(&sm.full[s], 1); mbar_init(&sm.empty[s], 1); }
    mbar_init(&sm.accum, 1);
    sm.timeout = 0; sm.nflag_rows = 0; sm.first_row = INT_MAX; sm.nflag_cols = 0; sm.first_col = INT_MAX;
    sm.nonfinite = 0;
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
      for (int kt = 0; kt < nk; ++kt) {
        const int s = kt % STAGES, u = kt / STAGES;
        if (u > 0 && !mbar_wait_bounded(&sm.empty[s], (u - 1) & 1, kWaitLimitNs)) { sm.timeout = 1; break; }
        mbar_arrive_expect_tx(&sm.full[s], bytes);
        const int k0 = kt * bk_elems;
        tma_load_2d(sm.a[s], &tmA, &sm.full[s], k0, m0);
        tma_load_2d(sm.b[s], &tmB, &sm.full[s], k0, n0);
        if (FT) tma_load_2d(sm.chk[s], &tmChk, &sm.full[s], k0, blockIdx.y * CHK_ROWS);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issue
    if (lane == 0) {
      const uint32_t idesc = umma_idesc(1, 1, BM, BN);
      const uint32_t idesc_chk = umma_idesc(1, 1, BM, CHK_ROWS);
      int kt = 0;
      for (; kt < nk; ++kt) {
        const int s = kt % STAGES, u = kt / STAGES;
        if (!mbar_wait_bounded(&sm.full[s], u & 1, kWaitLimitNs)) { sm.timeout = 1; break; }
        tc_fence_after();
        const uint32_t a0 = smem_addr(sm.a[s]), b0 = smem_addr(sm.b[s]), c0 = smem_addr(sm.chk[s]);
#pragma unroll
        for (int kk = 0; kk < BKB / 32; ++kk) {
          const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
          const uint64_t ad = umma_desc_sw128(a0 + kk * 32);
          umma_bf16(tmem, ad, umma_desc_sw128(b0 + kk * 32), idesc, acc);
          if (FT) umma_bf16(tmem + kChkCol, ad, umma_desc_sw128(c0 + kk * 32), idesc_chk, acc);
        }
        umma_commit(&sm.empty[s]);
      }
      umma_commit(&sm.accum);
    }
  } else {
    // ------------------------------------------------------------ epilogue (warps 2..5)
    const int q = warp & 3;                 // TMEM lane quarter of this warp
    const int row = q * 32 + lane;          // tile row = TMEM lane
    const int64_t gi = m0 + row;
    const bool row_ok = row < nI;
    const int ew = warp - 2;                // epilogue warp index 0..3
    const uint32_t trow = tmem + (static_cast<uint32_t>(q * 32) << 16);
    // tcgen05.ld is warp-collective (.sync.aligned): every TMEM load below is executed by all
    // 32 lanes of the warp, whatever their row; `got` is made warp-uniform for that reason.
    const bool got = __all_sync(0xffffffffu, mbar_wait_bounded(&sm.accum, 0, kWaitLimitNs));
    if (!got) sm.timeout = 1;
    tc_fence_after();
    const bool beta_nz = p.beta != 0.0f;
    float rs = 0.f, rc = 0.f, rabs = 0.f;   // compensated sum of C over the row, upward |C| sum
    float cs = 0.f, cc = 0.f, cabs = 0.f;   // same for C_in
    if (got) {
      for (int ch = 0; ch < BN / 32; ++ch) {
        uint32_t v[32];
        __syncwarp();  // reconverge after the previous chunk's per-lane branches
        tmem_ld32(trow + ch * 32, v);
        tmem_ld_wait();
        float cinv[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int col = ch * 32 + j;
          const int64_t gj = n0 + col;
          const bool ok = row_ok && col < nJ;
          float acc = __uint_as_float(v[j]);
          float cin = 0.f;
          if (beta_nz && ok) cin = p.C[gi + gj * p.ldc];
          if (FT && p.inj.n > 0) {
            for (int e = 0; e < p.inj.n; ++e) {
              const InjectPoint& ip = p.inj.p[e];
              if (ip.i == gi && ip.j == gj && ip.site == kSiteAccum && ip.mode == FT_MODE_BITFLIP)
                acc = __uint_as_float(__float_as_uint(acc) ^ (1u << ip.bit));
            }
          }
          float out = beta_nz ? fmaf(p.alpha, acc, p.beta * cin) : p.alpha * acc;
          if (FT && p.inj.n > 0) {
            for (int e = 0; e < p.inj.n; ++e) {
              const InjectPoint& ip = p.inj.p[e];
              if (ip.i != gi || ip.j != gj || ip.site != kSiteOutput) continue;
              if (ip.mode == FT_MODE_BITFLIP) out = __uint_as_float(__float_as_uint(out) ^ (1u << ip.bit));
              else {
                const float em = ldexpf(fabsf(out), ip.rel_log2);
                out = ip.sign < 0 ? out - em : out + em;
              }
            }
          }
          if (ok) p.C[gi + gj * p.ldc] = out;
          if (FT) {
            const float o = ok ? out : 0.f;
            neumaier(rs, rc, o);
            rabs = __fadd_ru(rabs, fabsf(o));
            if (beta_nz) { neumaier(cs, cc, cin); cabs = __fadd_ru(cabs, fabsf(cin)); }
          }
          cinv[j] = cin;
        }
        if (FT && beta_nz) {
          // per-warp column sums of C_in for the lazy column side
          float w1[32], w2[32];
#pragma unroll
          for (int j = 0; j < 32; ++j) { w1[j] = cinv[j]; w2[j] = fabsf(cinv[j]); }
          const float colsum = warp_column_sum(w1, lane);
          const float colabs = warp_column_sum_up(w2, lane);
          sm.cin_col[ew][ch * 32 + lane] = colsum;
          sm.cin_col_abs[ew][ch * 32 + lane] = colabs;
        }
      }
    }
    if (FT) {
      // -------------------------------------------------------- row verification
      double delta = 0.0, tau = 0.0, predicted = 0.0;
      bool flagged = false;
      uint32_t w4[4] = {0u, 0u, 0u, 0u};
      if (got) {  // warp-uniform
        __syncwarp();
        tmem_ld4(trow + kChkCol, w4);
        tmem_ld_wait();
      }
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
        const float P = __fmul_ru(p.rowAbsA[gi], p.maxAbsBe[blockIdx.y]);
        const float g = gamma32_up((float)p.K, p.u_acc);
        const float prod = __fmul_ru(__fmul_ru(fabsf(p.alpha), P), __fadd_ru(__fmul_ru(g, 2.0078125f), 0x1p-20f));
        const float outp = __fmul_ru(0x1p-23f, __fadd_ru(rabs, __fmul_ru(fabsf(p.beta), cabs)));
        tau = (double)__fadd_ru(prod, outp);
        flagged = !(fabs(delta) <= tau) || isinf(delta);
        if (flagged) {
          atomicAdd(&sm.nflag_rows, 1);
          atomicMin(&sm.first_row, row);
        }
      }
      named_bar(1, 128);
      if (row_ok && row == sm.first_row) { sm.delta_row = delta; sm.tau_row = tau; sm.pred_row = predicted; }
      __threadfence_block();
      named_bar(1, 128);
      const int nr = sm.nflag_rows;
      const int64_t trr = blockIdx.x, tcc = blockIdx.y;
      if (nr > 0) {
        // ------------------------------------------------------ lazy column side (Section V.A)
        for (int cidx = t - 64; cidx < BN; cidx += 128) {
          if (cidx >= nJ) continue;
          const int64_t gj = n0 + cidx;
          float s = 0.f, c = 0.f, a = 0.f;
          for (int i = 0; i < nI; ++i) {
            const float x = p.C[(int64_t)(m0 + i) + gj * p.ldc];
            neumaier(s, c, x);
            a = __fadd_ru(a, fabsf(x));
          }
          // C^c(j) = alpha sum_k (e^T A)(k) B(k, j): compensated dot product (Dot2).
          const uint16_t* bcol = static_cast<const uint16_t*>(p.B) + gj * p.ldb;
          float ds = 0.f, dc = 0.f;
          for (int k = 0; k < p.K; ++k) {
            const float2 sa = p.sA[(int64_t)blockIdx.x * p.K + k];
            const float b = ldg_bf16(bcol, k);
            float p1, e1, p2, e2;
            two_prod(sa.x, b, p1, e1);
            two_prod(sa.y, b, p2, e2);
            neumaier(ds, dc, p1);
            dc += e1 + p2 + e2;
          }
          double cpred = (double)p.alpha * ((double)ds + (double)dc);
          float cin_abs = 0.f;
          if (beta_nz) {
            double cin_sum = 0.0;
            for (int w = 0; w < 4; ++w) { cin_sum += (double)sm.cin_col[w][cidx]; cin_abs = __fadd_ru(cin_abs, sm.cin_col_abs[w][cidx]); }
            cpred += (double)p.beta * cin_sum;
          }
          const double dcol = ((double)s + (double)c) - cpred;
          const float P = __fmul_ru(p.colAbsB[gj], p.maxAbsAe[blockIdx.x]);
          const float g = gamma32_up((float)p.K, p.u_acc);
          // C^c is formed in compensated arithmetic here; the C^c_ref side carries the
          // accumulation error, the partial C_in sums carry gamma_31 (binary32).
          const float prod = __fmul_ru(__fmul_ru(fabsf(p.alpha), P), __fadd_ru(g, 0x1p-30f));
          const float outp = __fmul_ru(0x1p-23f, __fadd_ru(a, __fmul_ru(__fmul_ru(fabsf(p.beta), cin_abs), 34.0f)));
          const double tauc = (double)__fadd_ru(prod, outp);
          const bool fl = !(fabs(dcol) <= tauc) || isinf(dcol);
          sm.col_delta[cidx] = dcol;
          sm.col_tau[cidx] = tauc;
          if (fl) {
            atomicAdd(&sm.nflag_cols, 1);
            atomicMin(&sm.first_col, cidx);
          }
        }
        __threadfence_block();
        named_bar(1, 128);
        if (sm.first_col < BN) { sm.delta_col = sm.col_delta[sm.first_col]; sm.tau_col = sm.col_tau[sm.first_col]; }
        const int nc = sm.nflag_cols;
        if (t == 64) {
          int kind;
          double before = 0.0, after = 0.0;
          int64_t gi2 = nr > 0 ? m0 + sm.first_row : -1;
          int64_t gj2 = nc > 0 ? n0 + sm.first_col : -1;
          if (nr == 1 && nc == 1) {
            kind = FT_KIND_CORRECTED;
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
          } else if (nc == 0) {
            kind = FT_KIND_CHECKSUM_ONLY;
          } else {
            kind = FT_KIND_UNCORRECTABLE;
          }
          tc_record(p, kind, trr, tcc, gi2, gj2, sm.delta_row, nc > 0 ? sm.delta_col : 0.0, sm.tau_row,
                    nc > 0 ? sm.tau_col : 0.0, before, after, nr, nc);
          if (p.report) {
            atomicAdd(reinterpret_cast<unsigned long long*>(&p.report->detected), 1ull);
            unsigned long long* ctr = (nr == 1 && nc == 1) ? reinterpret_cast<unsigned long long*>(&p.report->corrected)
                                      : (nc == 0) ? reinterpret_cast<unsigned long long*>(&p.report->checksum_only)
                                                  : reinterpret_cast<unsigned long long*>(&p.report->uncorrectable);
            atomicAdd(ctr, 1ull);
          }
        }
      }
      if (t == 64 && p.report) atomicAdd(reinterpret_cast<unsigned long long*>(&p.report->tiles_checked), 1ull);
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
// K-contiguous (row i of A at A + i*lda, column j of B at B + j*ldb).
// ---------------------------------------------------------------------------------------

// Per 128-row block I and 1024-wide k chunk: e^T A over the block for each k (as an
// unevaluated hi + lo binary32 pair, compensated), the upward sum of |A| over the block
// (max over k -> maxAbsAe[I]) and per-row upward partial sums of |A| over the chunk.
constexpr int ENC_KC = 1024;

__global__ void __launch_bounds__(256) encode_rows_kernel(const uint16_t* A, int64_t lda, int32_t M, int32_t K,
                                                           float2* sA, float* rowAbsPart, float* maxAbsAe) {
  const int I = blockIdx.x, kc = blockIdx.y;
  const int m0 = I * BM, k0 = kc * ENC_KC;
  const int nI = min(BM, M - m0), kn = min(ENC_KC, K - k0);
  __shared__ float tile[BM][65];
  float rowabs = 0.f;    // thread t < 128: row t
  float colmax = 0.f;
  for (int kb = 0; kb < kn; kb += 64) {
    const int kw = min(64, kn - kb);
    for (int idx = threadIdx.x; idx < BM * 64; idx += 256) {
      const int r = idx / 64, kk = idx % 64;
      tile[r][kk] = (r < nI && kk < kw) ? bf16_to_f32(A[(int64_t)(m0 + r) * lda + k0 + kb + kk]) : 0.f;
    }
    __syncthreads();
    if (threadIdx.x < BM) {
      for (int kk = 0; kk < 64; ++kk) rowabs = __fadd_ru(rowabs, fabsf(tile[threadIdx.x][kk]));
    } else if (threadIdx.x < BM + 64) {
      const int kk = threadIdx.x - BM;
      if (kk < kw) {
        float s = 0.f, c = 0.f, a = 0.f;
        for (int r = 0; r < BM; ++r) { neumaier(s, c, tile[r][kk]); a = __fadd_ru(a, fabsf(tile[r][kk])); }
        const float hi = s + c;
        const float lo = c - (hi - s);
        sA[(int64_t)I * K + k0 + kb + kk] = make_float2(hi, lo);
        colmax = fmaxf(colmax, a);
      }
    }
    __syncthreads();
  }
  if (threadIdx.x < BM && threadIdx.x < nI) rowAbsPart[(int64_t)kc * M + m0 + threadIdx.x] = rowabs;
  if (threadIdx.x >= BM && threadIdx.x < BM + 64)
    atomicMax(reinterpret_cast<unsigned int*>(&maxAbsAe[I]), __float_as_uint(colmax));
}

// Per 256-column block J and k chunk: B e over the block for each k, split into three
// BF16 pieces written to rows J*16 + {0, 1, 2} of the checksum operand (K-contiguous,
// pitch kpitch); the upward |B| sum over the block (max over k -> maxAbsBe[J]); per-column
// upward partial sums of |B| over the chunk.
__global__ void __launch_bounds__(256) encode_cols_kernel(const uint16_t* B, int64_t ldb, int32_t N, int32_t K,
                                                           uint16_t* chk, int64_t kpitch, float* colAbsPart,
                                                           float* maxAbsBe) {
  const int J = blockIdx.x, kc = blockIdx.y;
  const int n0 = J * BN, k0 = kc * ENC_KC;
  const int nJ = min(BN, N - n0), kn = min(ENC_KC, K - k0);
  __shared__ float tile[BN][33];
  float colabs = 0.f;  // thread t: column t (256 threads = 256 columns)
  float kmax = 0.f;
  for (int kb = 0; kb < kn; kb += 32) {
    const int kw = min(32, kn - kb);
    for (int idx = threadIdx.x; idx < BN * 32; idx += 256) {
      const int c = idx / 32, kk = idx % 32;
      tile[c][kk] = (c < nJ && kk < kw) ? bf16_to_f32(B[(int64_t)(n0 + c) * ldb + k0 + kb + kk]) : 0.f;
    }
    __syncthreads();
    for (int kk = 0; kk < 32; ++kk) colabs = __fadd_ru(colabs, fabsf(tile[threadIdx.x][kk]));
    if (threadIdx.x < 32 && threadIdx.x < kw) {
      const int kk = threadIdx.x;
      float s = 0.f, c = 0.f, a = 0.f;
      for (int col = 0; col < BN; ++col) { neumaier(s, c, tile[col][kk]); a = __fadd_ru(a, fabsf(tile[col][kk])); }
      // split s + c into three bfloat16 pieces, each the nearest bfloat16 of the remainder
      const float x = s + c;
      const float xr = c - (x - s);
      const __nv_bfloat16 h = __float2bfloat16_rn(x);
      const float r1 = (x - __bfloat162float(h)) + xr;
      const __nv_bfloat16 m = __float2bfloat16_rn(r1);
      const float r2 = r1 - __bfloat162float(m);
      const __nv_bfloat16 l = __float2bfloat16_rn(r2);
      const int64_t k = k0 + kb + kk;
      chk[(int64_t)(J * CHK_ROWS + 0) * kpitch + k] = __bfloat16_as_ushort(h);
      chk[(int64_t)(J * CHK_ROWS + 1) * kpitch + k] = __bfloat16_as_ushort(m);
      chk[(int64_t)(J * CHK_ROWS + 2) * kpitch + k] = __bfloat16_as_ushort(l);
      kmax = fmaxf(kmax, a);
    }
    __syncthreads();
  }
  if (threadIdx.x < nJ) colAbsPart[(int64_t)kc * N + n0 + threadIdx.x] = colabs;
  if (threadIdx.x < 32) atomicMax(reinterpret_cast<unsigned int*>(&maxAbsBe[J]), __float_as_uint(kmax));
}

// Upward sum of the per-chunk partials.
__global__ void finalize_abs_kernel(const float* part, int nparts, int32_t n, float* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int c = 0; c < nparts; ++c) s = __fadd_ru(s, part[(int64_t)c * n + i]);
    out[i] = s;
  }
}

}  // namespace

size_t tc_workspace_bytes(int32_t M, int32_t N, int32_t K) {
  const int64_t nMb = (M + BM - 1) / BM, nNb = (N + BN - 1) / BN, nkc = (K + ENC_KC - 1) / ENC_KC;
  const int64_t kpitch = (K + 7) / 8 * 8;
  auto up = [](int64_t x) { return (x + 255) / 256 * 256; };
  return up(nNb * CHK_ROWS * kpitch * 2) + up(nMb * (int64_t)K * 8) + up(nkc * (int64_t)M * 4) + up(nkc * (int64_t)N * 4) +
         up(M * 4) + up(N * 4) + up(nMb * 4) + up(nNb * 4);
}

TcWorkspace tc_workspace_carve(void* base, int32_t M, int32_t N, int32_t K) {
  const int64_t nMb = (M + BM - 1) / BM, nNb = (N + BN - 1) / BN, nkc = (K + ENC_KC - 1) / ENC_KC;
  const int64_t kpitch = (K + 7) / 8 * 8;
  auto up = [](int64_t x) { return (x + 255) / 256 * 256; };
  char* c = static_cast<char*>(base);
  TcWorkspace w;
  w.chk = reinterpret_cast<uint16_t*>(c); c += up(nNb * CHK_ROWS * kpitch * 2);
  w.kpitch = kpitch;
  w.sA = reinterpret_cast<float2*>(c); c += up(nMb * (int64_t)K * 8);
  w.rowAbsPart = reinterpret_cast<float*>(c); c += up(nkc * (int64_t)M * 4);
  w.colAbsPart = reinterpret_cast<float*>(c); c += up(nkc * (int64_t)N * 4);
  w.rowAbsA = reinterpret_cast<float*>(c); c += up(M * 4);
  w.colAbsB = reinterpret_cast<float*>(c); c += up(N * 4);
  w.maxAbsAe = reinterpret_cast<float*>(c); c += up(nMb * 4);
  w.maxAbsBe = reinterpret_cast<float*>(c); c += up(nNb * 4);
  w.bytes = static_cast<size_t>(c - static_cast<char*>(base));
  return w;
}

cudaError_t launch_tc_encode(const TcParams& p, const TcWorkspace& w, void* ws_base, cudaStream_t st) {
  const int nMb = (p.M + BM - 1) / BM, nNb = (p.N + BN - 1) / BN, nkc = (p.K + ENC_KC - 1) / ENC_KC;
  cudaError_t e = cudaMemsetAsync(ws_base, 0, w.bytes, st);  // zero pieces rows 3..15 and the maxima
  if (e != cudaSuccess) return e;
  encode_rows_kernel<<<dim3(nMb, nkc), 256, 0, st>>>(static_cast<const uint16_t*>(p.A), p.lda, p.M, p.K, w.sA,
                                                      w.rowAbsPart, w.maxAbsAe);
  encode_cols_kernel<<<dim3(nNb, nkc), 256, 0, st>>>(static_cast<const uint16_t*>(p.B), p.ldb, p.N, p.K, w.chk,
                                                      w.kpitch, w.colAbsPart, w.maxAbsBe);
  finalize_abs_kernel<<<(p.M + 255) / 256, 256, 0, st>>>(w.rowAbsPart, nkc, p.M, w.rowAbsA);
  finalize_abs_kernel<<<(p.N + 255) / 256, 256, 0, st>>>(w.colAbsPart, nkc, p.N, w.colAbsB);
  return cudaGetLastError();
}

cudaError_t launch_tc_gemm(const TcParams& p, const CUtensorMap* tmA, const CUtensorMap* tmB, const CUtensorMap* tmChk,
                           bool ft, cudaStream_t st) {
  dim3 grid((p.M + BM - 1) / BM, (p.N + BN - 1) / BN);
  const size_t smem = sizeof(TcSmem);
  if (ft) {
    cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    tc_gemm_kernel<true><<<grid, NTHREADS, smem, st>>>(*tmA, *tmB, *tmChk, p);
  } else {
    cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    tc_gemm_kernel<false><<<grid, NTHREADS, smem, st>>>(*tmA, *tmB, *tmChk, p);
  }
  return cudaGetLastError();
}

}  // namespace ftk
