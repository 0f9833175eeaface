// FP64 ABFT-protected GEMM for sm_103a (FT-BLAS, Zhai et al., ICS '21, Sections II.A, V).
//
// One CTA computes one output tile over all of K, 128 x 128 (or 64 x 64 where 128-edge
// tiles would leave SMs idle); that tile is the verification interval. Per k-tile (32 deep) the operand tiles are staged in shared memory by TMA
// (3-stage mbarrier ring; a cooperative-load fallback covers pointers or leading dimensions
// TMA cannot address). While staged they are reused, as the paper's fused packing reuses
// each loaded element (Section V.B):
//   E1  warp reductions give this k-tile's checksum row of A^c = [A; e^T A] (e^T A over the
//       tile's rows) and checksum column of B^r = [B, Be] (Be over the tile's columns);
//   E2  the predicted checksums accumulate C^r(i) += A(i,k) (Be)(k) and
//       C^c(j) += (e^T A)(k) B(k,j), with upward-rounded binary32 magnitudes for the
//       threshold;
//   MMA the product, by one of two FP64 engines sharing this code: DFMA (8x8 register
//       micro-tile of fused multiply-adds per thread) or DMMA (mma.sync.m8n8k4.f64 tensor
//       core fragments). On GB300 both issue to the same FP64 pipe, so checksum work costs
//       exactly its operation count: 2 (BM + BN) FP64 operations per k (E1's two sums, E2's
//       two fused multiply-adds) against BM BN for the product, 1/32 at 128 x 128 and 1/16
//       at 64 x 64.
// Epilogue: C = alpha*acc + beta*C_in in registers; reference checksums C^r_ref, C^c_ref
// from those registers (Section V.B reuses C at register level); compare with the
// predicted ones against the rigorous round-off threshold; exactly one flagged row and
// one flagged column locate the error (Section V.A), which is corrected by recomputing
// that element with the identical instruction sequence (bit-exact fault-free value);
// other patterns are classified and reported. Then the tile is stored.
// Online verification (optional, Section V.A): every kc_tiles k-tiles the same comparison
// runs on the partial product (raw accumulators against the predicted partial checksums,
// threshold for the k done so far); one flagged row and column are corrected there by
// recomputing that accumulator over those k, so each interval tolerates one error.
#include <climits>

#include "ft_device.cuh"
#include "ft_internal.h"

namespace ftk {

namespace {

constexpr int BK = kDBK, STAGES = kDStages, NT = kDThreads;
// Shared memory of one CTA for engine E (tile E::BM x E::BN).
template <class E>
struct __align__(1024) DSmem {
  double a[STAGES][E::BM * BK];
  double b[STAGES][BK * E::BN];
  double encA[BK];        // e^T A over the tile's rows, per k of the current k-tile
  double encB[BK];        // B e over the tile's columns
  float encA_abs[BK];     // upward-rounded e^T |A|
  float encB_abs[BK];     // upward-rounded |B| e
  uint64_t full[STAGES];
  int timeout;
  int nonfinite;
  int first_row, first_col;
  double delta_row, delta_col;
  double tau_row, tau_col;
  int recompute;          // 1: the located element must be recomputed
  int loc_i, loc_j;       // tile-local location
  // online verification scratch: per-slot row / column sums of the raw accumulators
  double mrs[E::ROW_SLOTS * E::BM], mra[E::ROW_SLOTS * E::BM];  // [ROW_SLOTS][BM] sums, upward sums of |.|
  double mcs[E::COL_SLOTS * E::BN], mca[E::COL_SLOTS * E::BN];  // [COL_SLOTS][BN]
};

// Operand element (i, k) of the staged A tile and (k, j) of the staged B tile.
// (TBM, TBN: the tile's rows and columns, the strides of the M- and N-contiguous layouts.)
template <bool AK, int TBM>
__device__ __forceinline__ double lds_a(const double* sA, int i, int k) {
  return AK ? sA[i * BK + k] : sA[k * TBM + i];
}
template <bool BKM, int TBN>
__device__ __forceinline__ double lds_b(const double* sB, int k, int j) {
  return BKM ? sB[j * BK + k] : sB[k * TBN + j];
}

// Kernel-frame global operand access (recompute and fallback loads).
__device__ __forceinline__ double ldg_a(const DgemmParams& p, int64_t i, int64_t k) {
  return p.a_kmajor ? p.A[k + i * p.lda] : p.A[i + k * p.lda];
}
__device__ __forceinline__ double ldg_b(const DgemmParams& p, int64_t k, int64_t j) {
  return p.b_kmajor ? p.B[k + j * p.ldb] : p.B[j + k * p.ldb];
}

// ---------------------------------------------------------------------------------------
// Product engines. Each thread owns NR x NC accumulators at tile rows row(t, r) and tile
// columns col(t, c); threads sharing a row (column) have distinct row_slot (col_slot).
// ---------------------------------------------------------------------------------------
// NR x NC accumulators per thread: a 16 NR x 16 NC tile (128 x 128 for 8 x 8, 64 x 64 for 4 x 4).
template <int NR_, int NC_>
struct EngineDFMA {
  static constexpr int NR = NR_, NC = NC_;
  static constexpr int BM = 16 * NR, BN = 16 * NC;
  // Lanes l and l^16 share rows (reduced by one xor shuffle); the 8 warps then hold 8
  // partials per row. A column belongs to one half-warp (xor 1, 2, 4, 8): one partial.
  static constexpr int ROW_SLOTS = 8, COL_SLOTS = 1;
  static constexpr int ROW_XOR = 16, COL_XOR = 15;  // lane bits over which to reduce
  __device__ static int row(int t, int r) { return (t & 15) + 16 * r; }
  __device__ static int col(int t, int c) { return (t >> 4) + 16 * c; }
  __device__ static int row_slot(int t) { return t >> 5; }
  __device__ static int col_slot(int t) { return 0; }

  template <bool AK, bool BKM>
  __device__ static void ktile(double (&acc)[NR][NC], const double* sA, const double* sB, int t) {
    const int tr = t & 15, tc = t >> 4;
#pragma unroll 2
    for (int k = 0; k < BK; ++k) {
      double a[NR], b[NC];
#pragma unroll
      for (int r = 0; r < NR; ++r) a[r] = lds_a<AK, BM>(sA, tr + 16 * r, k);
#pragma unroll
      for (int c = 0; c < NC; ++c) b[c] = lds_b<BKM, BN>(sB, k, tc + 16 * c);
#pragma unroll
      for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
    }
  }

  // Fault-free value of acc at kernel-frame element (gi, gj): the same fused multiply-add
  // chain in ascending k (the zero-filled padding of the last k-tile adds exact zeros).
  // Called by the owning thread only; returns true if this thread produced the value.
  __device__ static bool recompute(const DgemmParams& p, int64_t gi, int64_t gj, int t, int li, int lj,
                                   double& out, int64_t kmin, int64_t kmax) {
    bool mine = false;
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
      for (int c = 0; c < NC; ++c) mine |= (row(t, r) == li && col(t, c) == lj);
    if (!mine) return false;
    double acc = 0.0;
    for (int64_t k = kmin; k < kmax; ++k) acc = fma(ldg_a(p, gi, k), ldg_b(p, k, gj), acc);
    out = acc;
    return true;
  }
};

__device__ __forceinline__ void dmma884(double& d0, double& d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}

struct EngineDMMA {
  // 8 warps as 4 (rows) x 2 (columns); warp tile 32 x 64 = 4 x 8 fragments of 8 x 8.
  // m8n8k4 fragments: A(g, q), B(q, g), C(g, 2q + e) with g = lane / 4, q = lane % 4.
  static constexpr int NR = 4, NC = 16;
  static constexpr int BM = 128, BN = 128;
  // Rows are shared by the 4 lanes with equal g (xor 1, 2) and by the 2 column warps;
  // columns by the 8 lanes with equal q (xor 4, 8, 16) and by the 4 row warps.
  static constexpr int ROW_SLOTS = 2, COL_SLOTS = 4;
  static constexpr int ROW_XOR = 3, COL_XOR = 28;
  __device__ static int wm(int t) { return (t >> 5) & 3; }
  __device__ static int wn(int t) { return t >> 7; }
  __device__ static int g(int t) { return (t & 31) >> 2; }
  __device__ static int q(int t) { return t & 3; }
  __device__ static int row(int t, int r) { return 32 * wm(t) + 8 * r + g(t); }
  __device__ static int col(int t, int c) { return 64 * wn(t) + 8 * (c >> 1) + 2 * q(t) + (c & 1); }
  __device__ static int row_slot(int t) { return wn(t); }
  __device__ static int col_slot(int t) { return wm(t); }

  template <bool AK, bool BKM>
  __device__ static void ktile(double (&acc)[NR][NC], const double* sA, const double* sB, int t) {
    const int r0 = 32 * wm(t) + g(t), c0 = 64 * wn(t) + g(t), qq = q(t);
#pragma unroll 2
    for (int k = 0; k < BK; k += 4) {
      double a[NR], b[NC / 2];
#pragma unroll
      for (int mb = 0; mb < NR; ++mb) a[mb] = lds_a<AK, BM>(sA, r0 + 8 * mb, k + qq);
#pragma unroll
      for (int nb = 0; nb < NC / 2; ++nb) b[nb] = lds_b<BKM, BN>(sB, k + qq, c0 + 8 * nb);
#pragma unroll
      for (int mb = 0; mb < NR; ++mb)
#pragma unroll
        for (int nb = 0; nb < NC / 2; ++nb) dmma884(acc[mb][2 * nb], acc[mb][2 * nb + 1], a[mb], b[nb]);
    }
  }

  // Warp-cooperative recompute of the 8 x 8 fragment holding the element, with the same
  // mma sequence over k < kmax in chunks of 4 (out-of-range operands are the zeros TMA filled).
  __device__ static bool recompute(const DgemmParams& p, int64_t gi, int64_t gj, int t, int li, int lj,
                                   double& out, int64_t kmin, int64_t kmax) {
    const int w_row = li / 32, w_col = lj / 64;
    if (wm(t) != w_row || wn(t) != w_col) return false;  // warp-uniform
    const int64_t rb = gi - (li % 8), cb = gj - (lj % 8);  // fragment origin, kernel frame
    const int64_t ra = rb + g(t), cbb = cb + g(t);
    double d0 = 0.0, d1 = 0.0;
    for (int64_t k0 = kmin; k0 < kmax; k0 += 4) {
      const int64_t k = k0 + q(t);
      const double a = (ra < p.M && k < p.K) ? ldg_a(p, ra, k) : 0.0;
      const double b = (cbb < p.N && k < p.K) ? ldg_b(p, k, cbb) : 0.0;
      dmma884(d0, d1, a, b);
    }
    const int my_row = li % 8 == g(t);
    const int my_col = (lj % 8) / 2 == q(t);
    if (my_row && my_col) {
      out = (lj & 1) ? d1 : d0;
      return true;
    }
    return false;
  }
};


// Butterfly sum over the lane bits in `mask` (plain and upward-rounded).
__device__ __forceinline__ void xor_reduce(double& s, double& a, int mask) {
#pragma unroll
  for (int b = 1; b < 32; b <<= 1) {
    if (mask & b) {
      s += __shfl_xor_sync(0xffffffffu, s, b);
      a = __dadd_ru(a, __shfl_xor_sync(0xffffffffu, a, b));
    }
  }
}

// Row and column sums (and upward-rounded sums of magnitudes) of val(r, c) over the
// tile, written as per-slot partials: srow/arow[ROW_SLOTS][BM], scol/acol[COL_SLOTS][BN].
template <class E, class F>
__device__ __forceinline__ void tile_sums(F val, int t, double* srow, double* arow, double* scol, double* acol) {
  constexpr int BM = E::BM, BN = E::BN;
  const int lane = t & 31;
#pragma unroll
  for (int r = 0; r < E::NR; ++r) {
    double s = 0.0, a = 0.0;
#pragma unroll
    for (int c = 0; c < E::NC; ++c) { const double x = val(r, c); s += x; a = __dadd_ru(a, fabs(x)); }
    xor_reduce(s, a, E::ROW_XOR);
    if ((lane & E::ROW_XOR) == 0) { srow[E::row_slot(t) * BM + E::row(t, r)] = s; arow[E::row_slot(t) * BM + E::row(t, r)] = a; }
  }
#pragma unroll
  for (int c = 0; c < E::NC; ++c) {
    double s = 0.0, a = 0.0;
#pragma unroll
    for (int r = 0; r < E::NR; ++r) { const double x = val(r, c); s += x; a = __dadd_ru(a, fabs(x)); }
    xor_reduce(s, a, E::COL_XOR);
    if ((lane & E::COL_XOR) == 0) { scol[E::col_slot(t) * BN + E::col(t, c)] = s; acol[E::col_slot(t) * BN + E::col(t, c)] = a; }
  }
}

// Upward-rounded gamma_n = n u / (1 - n u), u = 2^-53, in binary64.
__device__ __forceinline__ double gamma_up64(int64_t n) {
  const double nu = __dmul_ru((double)n, 0x1p-53);
  return __ddiv_ru(nu, __dsub_rd(1.0, nu));
}

__device__ void write_record(const DgemmParams& p, int kind, int64_t tr, int64_t tc, int64_t i, int64_t j,
                             double drow, double dcol, double trow, double tcol, double before, double after,
                             int nr, int nc) {
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

// Cooperative (non-TMA) load of one k-tile into the same smem layout TMA produces.
template <class E, bool AK, bool BKM>
__device__ void load_ktile_plain(const DgemmParams& p, double* sA, double* sB, int m0, int n0, int k0, int t) {
  constexpr int BM = E::BM, BN = E::BN;
  for (int idx = t; idx < BM * BK; idx += NT) {
    int i, k;
    if (AK) { i = idx / BK; k = idx % BK; } else { k = idx / BM; i = idx % BM; }
    const int64_t gi = m0 + i, gk = k0 + k;
    sA[idx] = (gi < p.M && gk < p.K) ? ldg_a(p, gi, gk) : 0.0;
  }
  for (int idx = t; idx < BK * BN; idx += NT) {
    int k, j;
    if (BKM) { j = idx / BK; k = idx % BK; } else { k = idx / BN; j = idx % BN; }
    const int64_t gk = k0 + k, gj = n0 + j;
    sB[idx] = (gk < p.K && gj < p.N) ? ldg_b(p, gk, gj) : 0.0;
  }
}

// Bytes beyond the stage's that the staging barrier of k-tile kt of the tile at (m0, n0)
// expects: 16 when a stall point (test launches only) names that tile and k-tile, so that the
// barrier never completes and the waits on it give up; else 0.
template <class E>
__device__ __forceinline__ uint32_t stall_bytes(const DgemmParams& p, int m0, int n0, int kt, int kstar_tile) {
  for (int e = 0; e < p.inj.n; ++e) {
    const InjectPoint& ip = p.inj.p[e];
    if (ip.site == kSiteStall && kt == (ip.kt > 0 ? ip.kt : kstar_tile) && ip.i >= m0 && ip.i < m0 + E::BM &&
        ip.j >= n0 && ip.j < n0 + E::BN)
      return 16u;
  }
  return 0u;
}

template <class E, bool AK, bool BKM>
__device__ __forceinline__ void issue_ktile(DSmem<E>& sm, const CUtensorMap* tmA, const CUtensorMap* tmB, int s,
                                            int m0, int n0, int k0, uint32_t extra_bytes) {
  constexpr uint32_t kStageBytes = (E::BM * BK + BK * E::BN) * sizeof(double);
  mbar_arrive_expect_tx(&sm.full[s], kStageBytes + extra_bytes);
  if (AK) tma_load_2d(sm.a[s], tmA, &sm.full[s], k0, m0);
  else tma_load_2d(sm.a[s], tmA, &sm.full[s], m0, k0);
  if (BKM) tma_load_2d(sm.b[s], tmB, &sm.full[s], k0, n0);
  else tma_load_2d(sm.b[s], tmB, &sm.full[s], n0, k0);
}

// Online verification of the partial product over k < kp (Section V.A): reference sums of
// the raw accumulators against the running predictions pred (C^r or C^c without alpha,
// beta) with tau = 2 [gamma_{kp + n + 3} P + gamma_n sum |acc|], P the running magnitude
// bound. One flagged row and one flagged column: the accumulator at their crossing is
// recomputed over k < kp with the product's own instruction sequence and a corrected record
// written; other patterns are left to the finished tile's check. All threads of the CTA
// call it (it synchronises).
template <class E>
__device__ __forceinline__ void online_check(const DgemmParams& p, double (&acc)[E::NR][E::NC], double pred, float pmag,
                                          DSmem<E>& sm, int t, int m0, int n0, int nI, int nJ, int64_t kmin,
                                          int64_t kp) {
  constexpr int BM = E::BM, BN = E::BN;
  tile_sums<E>([&](int r, int c) { return acc[r][c]; }, t, sm.mrs, sm.mra, sm.mcs, sm.mca);
  const bool huge = __syncthreads_or(!isfinite(pmag));  // binary32 bound overflowed: skip
  if (huge) return;
  // one row (t < BM) or one column (BM <= t < BM + BN) per thread; threads beyond idle
  const bool is_row = t < BM, active = t < BM + BN;
  const int idx = is_row ? t : (active ? t - BM : 0);
  const int nslots = is_row ? E::ROW_SLOTS : E::COL_SLOTS;
  const int extent = is_row ? BM : BN;
  const double* ps = is_row ? sm.mrs : sm.mcs;
  const double* pa = is_row ? sm.mra : sm.mca;
  double ref = 0.0, R = 0.0;
  for (int sl = 0; sl < nslots; ++sl) {
    ref += ps[sl * extent + idx];
    R = __dadd_ru(R, pa[sl * extent + idx]);
  }
  const double delta = ref - pred;
  const int n_other = is_row ? nJ : nI;
  double tau = __fma_ru(gamma_up64(kp + n_other + 3), (double)pmag, __dmul_ru(gamma_up64(n_other), R));
  tau = __dmul_ru(2.0, tau);
  const bool valid = active && idx < (is_row ? nI : nJ);
  const bool flagged = valid && (!(fabs(delta) <= tau) || isinf(delta));
  if (flagged) atomicMin(is_row ? &sm.first_row : &sm.first_col, idx);
  const int nr = __syncthreads_count(is_row && flagged);
  const int nc = __syncthreads_count(!is_row && flagged);
  if (flagged && is_row && idx == sm.first_row) { sm.delta_row = delta; sm.tau_row = tau; }
  if (flagged && !is_row && idx == sm.first_col) { sm.delta_col = delta; sm.tau_col = tau; }
  __syncthreads();
  if (nr == 1 && nc == 1 && sm.nonfinite == 0) {
    const int li = sm.first_row, lj = sm.first_col;
    const int64_t gi = m0 + li, gj = n0 + lj;
    double fixed;
    if (E::recompute(p, gi, gj, t, li, lj, fixed, kmin, kp)) {
      double before = 0.0;
#pragma unroll
      for (int r = 0; r < E::NR; ++r)
#pragma unroll
        for (int c = 0; c < E::NC; ++c)
          if (E::row(t, r) == li && E::col(t, c) == lj) { before = acc[r][c]; acc[r][c] = fixed; }
      write_record(p, FT_KIND_CORRECTED, blockIdx.x, blockIdx.y, gi, gj, sm.delta_row, sm.delta_col, sm.tau_row,
                   sm.tau_col, before, fixed, 1, 1);
      if (p.report) {
        atomicAdd(reinterpret_cast<unsigned long long*>(&p.report->detected), 1ull);
        atomicAdd(reinterpret_cast<unsigned long long*>(&p.report->corrected), 1ull);
      }
    }
  }
  __syncthreads();
  if (t == 0) { sm.first_row = INT_MAX; sm.first_col = INT_MAX; }
  __syncthreads();
}

template <class E, bool AK, bool BKM, bool FT>
__global__ void __launch_bounds__(NT, 1)
    dgemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                 const __grid_constant__ DgemmParams p) {
  constexpr int BM = E::BM, BN = E::BN;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  DSmem<E>& sm = *reinterpret_cast<DSmem<E>*>(smem_raw);
  const int t = threadIdx.x;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int nk = (p.K + BK - 1) / BK;
  const int kstar_tile = nk / 2;
  // k-tiles this tile needs: all of them, or the range a triangular operand leaves nonzero
  // (op(A) upper: k >= i; lower: k <= i; op(B) upper: k <= j; lower: k >= j).
  int kb = 0, ke = nk;
  if (p.tri_a == 1) kb = m0 / BK;
  if (p.tri_a == 2) ke = min(ke, (m0 + BM + BK - 1) / BK);
  if (p.tri_b == 1) ke = min(ke, (n0 + BN + BK - 1) / BK);
  if (p.tri_b == 2) kb = max(kb, n0 / BK);
  const int nl = ke > kb ? ke - kb : 0;  // k-tiles in range
  const int64_t k_lo = (int64_t)kb * BK, k_hi = min((int64_t)ke * BK, (int64_t)p.K);
  const int nI = min(BM, p.M - m0), nJ = min(BN, p.N - n0);

  if (t == 0) {
    for (int s = 0; s < STAGES; ++s) mbar_init(&sm.full[s], 1);
    sm.timeout = 0; sm.nonfinite = 0;
    sm.first_row = INT_MAX; sm.first_col = INT_MAX;
    sm.recompute = 0;
    fence_mbar_init();
    if (p.use_tma) {
      tma_prefetch_desc(&tmA);
      tma_prefetch_desc(&tmB);
      for (int s = 0; s < STAGES && s < nl; ++s)
        issue_ktile<E, AK, BKM>(sm, &tmA, &tmB, s, m0, n0, (kb + s) * BK, stall_bytes<E>(p, m0, n0, kb + s, kstar_tile));
    }
  }
  __syncthreads();

  double acc[E::NR][E::NC];
#pragma unroll
  for (int r = 0; r < E::NR; ++r)
#pragma unroll
    for (int c = 0; c < E::NC; ++c) acc[r][c] = 0.0;
  double pred = 0.0;  // t < 128: alpha-free C^r(i = t) partial; t >= 128: C^c(j = t - 128)
  float pmag = 0.0f;  // upward-rounded magnitude sum for the threshold

  int kt = kb;
  for (; kt < ke; ++kt) {
    const int lt = kt - kb;  // position in this tile's k-range: stage and phase
    const int s = lt % STAGES;
    if (p.use_tma) {
      if (!mbar_wait_bounded(&sm.full[s], (lt / STAGES) & 1, p.wait_limit_ns)) sm.timeout = 1;
    } else {
      load_ktile_plain<E, AK, BKM>(p, sm.a[s], sm.b[s], m0, n0, kt * BK, t);
    }
    __syncthreads();
    if (sm.timeout) break;
    const double* sA = sm.a[s];
    const double* sB = sm.b[s];

    if (FT) {
      // Accumulator injection after bk * kt products, kt = the point's k-tile or floor(nk / 2)
      // (test launches only).
      if (p.inj.n > 0) {
        for (int e = 0; e < p.inj.n; ++e) {
          const InjectPoint& ip = p.inj.p[e];
          if (ip.site != kSiteAccum || ip.mode != FT_MODE_BITFLIP) continue;
          if (kt != (ip.kt > 0 ? ip.kt : kstar_tile)) continue;
          const int li = ip.i - m0, lj = ip.j - n0;
          if (li < 0 || li >= nI || lj < 0 || lj >= nJ) continue;
#pragma unroll
          for (int r = 0; r < E::NR; ++r)
#pragma unroll
            for (int c = 0; c < E::NC; ++c)
              if (E::row(t, r) == li && E::col(t, c) == lj) acc[r][c] = flip_bit_f64(acc[r][c], ip.bit);
        }
      }
      // E1: e^T A (k = s < BK) and B e (k = s - BK) for this k-tile; 4 lanes per sum.
      {
        const int sidx = t >> 2, part = t & 3;
        double v = 0.0;
        float va = 0.0f;
        if (sidx < BK) {
#pragma unroll 8
          for (int qq = 0; qq < BM / 4; ++qq) {
            const double x = lds_a<AK, BM>(sA, part + 4 * qq, sidx);
            v += x;
            va = add_up(va, abs_up(x));
          }
        } else {
#pragma unroll 8
          for (int qq = 0; qq < BN / 4; ++qq) {
            const double x = lds_b<BKM, BN>(sB, sidx - BK, part + 4 * qq);
            v += x;
            va = add_up(va, abs_up(x));
          }
        }
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        v += __shfl_xor_sync(0xffffffffu, v, 2);
        va = add_up(va, __shfl_xor_sync(0xffffffffu, va, 1));
        va = add_up(va, __shfl_xor_sync(0xffffffffu, va, 2));
        if (part == 0) {
          if (sidx < BK) { sm.encA[sidx] = v; sm.encA_abs[sidx] = va; }
          else { sm.encB[sidx - BK] = v; sm.encB_abs[sidx - BK] = va; }
          if (!isfinite(v)) sm.nonfinite = 1;
        }
      }
      __syncthreads();
      // E2: C^r(i) += sum_k A(i,k) (Be)(k) for i = t; C^c(j) += sum_k (e^T A)(k) B(k,j) for
      // j = t - BM (threads from BM + BN on are idle). The k order is rotated by lane to
      // spread shared-memory banks.
      if (t < BM) {
#pragma unroll 8
        for (int kk = 0; kk < BK; ++kk) {
          const int k = (kk + t) & (BK - 1);
          const double x = lds_a<AK, BM>(sA, t, k);
          pred = fma(x, sm.encB[k], pred);
          pmag = fma_up(abs_up(x), sm.encB_abs[k], pmag);
        }
      } else if (t < BM + BN) {
        const int j = t - BM;
#pragma unroll 8
        for (int kk = 0; kk < BK; ++kk) {
          const int k = (kk + t) & (BK - 1);
          const double y = lds_b<BKM, BN>(sB, k, j);
          pred = fma(sm.encA[k], y, pred);
          pmag = fma_up(sm.encA_abs[k], abs_up(y), pmag);
        }
      }
    }

    E::template ktile<AK, BKM>(acc, sA, sB, t);
    __syncthreads();
    if (p.use_tma && t == 0 && lt + STAGES < nl)
      issue_ktile<E, AK, BKM>(sm, &tmA, &tmB, s, m0, n0, (kt + STAGES) * BK,
                              stall_bytes<E>(p, m0, n0, kt + STAGES, kstar_tile));
    if (FT && p.kc_tiles > 0 && (kt + 1) % p.kc_tiles == 0 && kt + 1 < ke)
      online_check<E>(p, acc, pred, pmag, sm, t, m0, n0, nI, nJ, k_lo, (int64_t)(kt + 1) * BK);
  }

  if (sm.timeout) {
    // Abandon the tile: wait (bounded) for copies this CTA still has in flight, then
    // report. The output tile is not written.
    if (t == 0) {
      if (p.use_tma)
        for (int k2 = kt; k2 < ke && k2 < kt + STAGES; ++k2)
          (void)mbar_wait_bounded(&sm.full[(k2 - kb) % STAGES], ((k2 - kb) / STAGES) & 1, p.wait_limit_ns);
      if (p.report) atomicOr(&p.report->status, FT_STATUS_TIMEOUT);
    }
    return;
  }

  // ---------------------------------------------------------------- epilogue: C in registers
  const bool beta_nz = (p.beta != 0.0);
  auto cin_at = [&](int li, int lj) -> double {
    return (li < nI && lj < nJ) ? p.C[(int64_t)(m0 + li) + (int64_t)(n0 + lj) * p.ldc] : 0.0;
  };
  // Partial-sum arrays overlay the operand ring (every copy has landed and been read).
  double* rsum = sm.a[0];                 // [ROW_SLOTS][BM]  sum of C over the row
  double* rabs = rsum + E::ROW_SLOTS * BM;  //                  upward sum of |C|
  double* rcin = rabs + E::ROW_SLOTS * BM;  //                  sum of C_in
  double* rabc = rcin + E::ROW_SLOTS * BM;  //                  upward sum of |C_in|
  double* csum = rabc + E::ROW_SLOTS * BM;  // [COL_SLOTS][BN]
  double* cabs = csum + E::COL_SLOTS * BN;
  double* ccin = cabs + E::COL_SLOTS * BN;
  double* cabc = ccin + E::COL_SLOTS * BN;
  double* slow = cabc + E::COL_SLOTS * BN;  // [2][kSlowChunk] threshold slow path
  constexpr int kSlowChunk = 1024;
  static_assert(4 * (E::ROW_SLOTS * BM + E::COL_SLOTS * BN) + 2 * kSlowChunk <= STAGES * BM * BK,
                "epilogue scratch exceeds the A ring");
  if (FT) {
    // beta*C_in enters the predicted checksums (Section V.B): its row and column sums.
    if (beta_nz) {
      tile_sums<E>([&](int r, int c) { return cin_at(E::row(t, r), E::col(t, c)); }, t, rcin, rabc, ccin, cabc);
    } else {
      tile_sums<E>([&](int, int) { return 0.0; }, t, rcin, rabc, ccin, cabc);
    }
  }
#pragma unroll
  for (int r = 0; r < E::NR; ++r)
#pragma unroll
    for (int c = 0; c < E::NC; ++c)
      acc[r][c] = beta_nz ? fma(p.alpha, acc[r][c], p.beta * cin_at(E::row(t, r), E::col(t, c))) : p.alpha * acc[r][c];

  if (FT) {
    // Output-site injection (test launches only).
    for (int e = 0; e < p.inj.n; ++e) {
      const InjectPoint& ip = p.inj.p[e];
      if (ip.site != kSiteOutput) continue;
      const int li = ip.i - m0, lj = ip.j - n0;
      if (li < 0 || li >= nI || lj < 0 || lj >= nJ) continue;
#pragma unroll
      for (int r = 0; r < E::NR; ++r)
#pragma unroll
        for (int c = 0; c < E::NC; ++c)
          if (E::row(t, r) == li && E::col(t, c) == lj) {
            double v = acc[r][c];
            if (ip.mode == FT_MODE_BITFLIP) v = flip_bit_f64(v, ip.bit);
            else {
              const double em = ldexp(fabs(v), ip.rel_log2);
              v = ip.sign < 0 ? v - em : v + em;
            }
            acc[r][c] = v;
          }
    }
    // Reference checksums C^r_ref, C^c_ref from the registers (Section V.B).
    tile_sums<E>([&](int r, int c) { return acc[r][c]; }, t, rsum, rabs, csum, cabs);
    __syncthreads();

    // One row (t < BM) or one column (BM <= t < BM + BN) per thread; threads beyond idle.
    const bool is_row = t < BM, active = t < BM + BN;
    const int idx = is_row ? t : (active ? t - BM : 0);
    const int nslots = is_row ? E::ROW_SLOTS : E::COL_SLOTS;
    const int extent = is_row ? BM : BN;
    const double* ps = is_row ? rsum : csum;
    const double* pa = is_row ? rabs : cabs;
    const double* pc = is_row ? rcin : ccin;
    const double* pac = is_row ? rabc : cabc;
    double ref = 0.0, cin_sum = 0.0, R = 0.0, Q = 0.0;
    for (int sl = 0; sl < nslots; ++sl) {
      ref += ps[sl * extent + idx];
      cin_sum += pc[sl * extent + idx];
      R = __dadd_ru(R, pa[sl * extent + idx]);
      Q = __dadd_ru(Q, pac[sl * extent + idx]);
    }
    // The binary32 magnitude sum from the mainloop overflows only for huge operands; then
    // the tile recomputes it in binary64 (upward) from global memory.
    double P = (double)pmag;
    if (__syncthreads_or(!isfinite(pmag))) {
      double* sabsB = slow;               // upward sum_{j in tile} |B(k, j)|
      double* sabsA = slow + kSlowChunk;  // upward sum_{i in tile} |A(i, k)|
      P = 0.0;
      for (int64_t k0 = 0; k0 < p.K; k0 += kSlowChunk) {
        const int kc = (int)((p.K - k0) < kSlowChunk ? (p.K - k0) : kSlowChunk);
        for (int kk = t; kk < kc; kk += NT) {
          double sb = 0.0, sa = 0.0;
          for (int j = 0; j < nJ; ++j) sb = __dadd_ru(sb, fabs(ldg_b(p, k0 + kk, n0 + j)));
          for (int i = 0; i < nI; ++i) sa = __dadd_ru(sa, fabs(ldg_a(p, m0 + i, k0 + kk)));
          sabsB[kk] = sb;
          sabsA[kk] = sa;
        }
        __syncthreads();
        if (active && idx < (is_row ? nI : nJ)) {
          for (int kk = 0; kk < kc; ++kk) {
            const double x = is_row ? fabs(ldg_a(p, m0 + idx, k0 + kk)) : fabs(ldg_b(p, k0 + kk, n0 + idx));
            P = __fma_ru(x, is_row ? sabsB[kk] : sabsA[kk], P);
          }
        }
        __syncthreads();
      }
    }
    double predicted = beta_nz ? fma(p.alpha, pred, p.beta * cin_sum) : p.alpha * pred;
    if (beta_nz && !isfinite(cin_sum)) sm.nonfinite = 1;
    for (int e = 0; e < p.inj.n; ++e) {  // checksum-path injection (test launches only)
      const InjectPoint& ip = p.inj.p[e];
      const bool hit_row = ip.site == kSiteChecksumRow && is_row && ip.i == m0 + idx && ip.j >= n0 && ip.j < n0 + nJ;
      const bool hit_col = ip.site == kSiteChecksumCol && !is_row && ip.j == n0 + idx && ip.i >= m0 && ip.i < m0 + nI;
      if (hit_row || hit_col) {
        if (ip.mode == FT_MODE_BITFLIP) predicted = flip_bit_f64(predicted, ip.bit);
        else {
          const double em = ldexp(fabs(predicted), ip.rel_log2);
          predicted = ip.sign < 0 ? predicted - em : predicted + em;
        }
      }
    }
    const double delta = ref - predicted;
    // tau = 2 [gamma_{K+n+3} (|alpha| P + |beta| Q) + gamma_n R], n = entries summed, all
    // rounded upward: a rigorous bound on |delta| for an error-free tile.
    const int n_other = is_row ? nJ : nI;
    const double g1 = gamma_up64((int64_t)p.K + n_other + 3), g2 = gamma_up64(n_other);
    double tau = __fma_ru(fabs(p.alpha), P, __dmul_ru(fabs(p.beta), Q));
    tau = __fma_ru(g1, tau, __dmul_ru(g2, R));
    tau = __dmul_ru(2.0, tau);
    const bool valid = active && idx < (is_row ? nI : nJ);
    // Flagged: |delta| > tau, or delta not finite (NaN, or infinite even against tau = inf).
    const bool flagged = valid && (!(fabs(delta) <= tau) || isinf(delta));
    if (flagged) atomicMin(is_row ? &sm.first_row : &sm.first_col, idx);
    const int nr = __syncthreads_count(is_row && flagged);
    const int nc = __syncthreads_count(!is_row && flagged);
    if (valid && is_row && idx == sm.first_row) { sm.delta_row = delta; sm.tau_row = tau; }
    if (valid && !is_row && idx == sm.first_col) { sm.delta_col = delta; sm.tau_col = tau; }
    __syncthreads();

    const bool nonfinite = sm.nonfinite != 0;
    const int64_t tr = blockIdx.x, tc = blockIdx.y;
    if (!nonfinite && nr == 1 && nc == 1) {
      // Located at the crossing of the flagged row and column; recompute it.
      const int li = sm.first_row, lj = sm.first_col;
      const int64_t gi = m0 + li, gj = n0 + lj;
      double acc_fixed;
      const bool mine = E::recompute(p, gi, gj, t, li, lj, acc_fixed, k_lo, k_hi);
      if (mine) {
        const double cin = beta_nz ? p.C[gi + gj * p.ldc] : 0.0;
        const double fixed = beta_nz ? fma(p.alpha, acc_fixed, p.beta * cin) : p.alpha * acc_fixed;
        double before = 0.0;
#pragma unroll
        for (int r = 0; r < E::NR; ++r)
#pragma unroll
          for (int c = 0; c < E::NC; ++c)
            if (E::row(t, r) == li && E::col(t, c) == lj) { before = acc[r][c]; acc[r][c] = fixed; }
        write_record(p, FT_KIND_CORRECTED, tr, tc, gi, gj, sm.delta_row, sm.delta_col, sm.tau_row, sm.tau_col,
                     before, fixed, nr, nc);
      }
    } else if (t == 0 && (nonfinite || nr > 0 || nc > 0)) {
      const int kind = nonfinite ? FT_KIND_INPUT_NONFINITE
                       : (nr == 0 || nc == 0) ? FT_KIND_CHECKSUM_ONLY
                                              : FT_KIND_UNCORRECTABLE;
      const int64_t gi = nr > 0 ? m0 + sm.first_row : -1;
      const int64_t gj = nc > 0 ? n0 + sm.first_col : -1;
      write_record(p, kind, tr, tc, gi, gj, nr > 0 ? sm.delta_row : 0.0, nc > 0 ? sm.delta_col : 0.0,
                   nr > 0 ? sm.tau_row : 0.0, nc > 0 ? sm.tau_col : 0.0, 0.0, 0.0, nr, nc);
    }
    if (t == 0 && p.report) {
      atomicAdd(reinterpret_cast<unsigned long long*>(&p.report->tiles_checked), 1ull);
      if (nonfinite) {
        atomicAdd(reinterpret_cast<unsigned long long*>(&p.report->input_nonfinite), 1ull);
      } else if (nr > 0 || nc > 0) {
        atomicAdd(reinterpret_cast<unsigned long long*>(&p.report->detected), 1ull);
        unsigned long long* ctr = (nr == 1 && nc == 1) ? reinterpret_cast<unsigned long long*>(&p.report->corrected)
                                  : (nr == 0 || nc == 0) ? reinterpret_cast<unsigned long long*>(&p.report->checksum_only)
                                                         : reinterpret_cast<unsigned long long*>(&p.report->uncorrectable);
        atomicAdd(ctr, 1ull);
      }
    }
  }

  // Store the tile.
#pragma unroll
  for (int c = 0; c < E::NC; ++c) {
#pragma unroll
    for (int r = 0; r < E::NR; ++r) {
      const int li = E::row(t, r), lj = E::col(t, c);
      if (li < nI && lj < nJ) p.C[(int64_t)(m0 + li) + (int64_t)(n0 + lj) * p.ldc] = acc[r][c];
    }
  }
}

// Full n x n copy T of a symmetric (mode 0) or triangular (mode 1) matrix stored in one
// triangle of X (layout col/row-major, leading dimension ldx), written in the same layout
// with leading dimension n.
//   mode 0: T(r,c) = X(r,c) when (r,c) lies in the stored triangle, else X(c,r);
//   mode 1: T = op(X) with the other triangle zero; unit_diag puts 1 on the diagonal.
__global__ void expand_kernel(const double* X, int64_t ldx, int32_t row_major, int64_t n, int32_t mode,
                              int32_t upper, int32_t trans, int32_t unit_diag, double* T) {
  const int64_t total = n * n;
  auto at = [&](int64_t r, int64_t c) { return row_major ? X[r * ldx + c] : X[r + c * ldx]; };
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    // e runs along the contiguous dimension of T
    const int64_t r = row_major ? e / n : e % n, c = row_major ? e % n : e / n;
    double v;
    if (mode == 0) {
      const bool stored = upper ? (r <= c) : (r >= c);
      v = stored ? at(r, c) : at(c, r);
    } else {
      const int64_t p = trans ? c : r, q = trans ? r : c;  // op(X)(r,c) = X(p,q)
      const bool in_tri = upper ? (p <= q) : (p >= q);
      v = (r == c && unit_diag) ? 1.0 : (in_tri ? at(p, q) : 0.0);
    }
    T[row_major ? r * n + c : r + c * n] = v;
  }
}

__global__ void scale_kernel(double* C, int64_t ldc, int32_t M, int32_t N, double beta) {
  const int64_t total = (int64_t)M * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % M, j = e / M;
    double* c = C + i + j * ldc;
    *c = (beta == 0.0) ? 0.0 : beta * *c;
  }
}

template <class E, bool AK, bool BKM, bool FT>
cudaError_t launch_one(const DgemmParams& p, const CUtensorMap* tmA, const CUtensorMap* tmB, cudaStream_t st) {
  auto kern = dgemm_kernel<E, AK, BKM, FT>;
  // Set on every launch: the attribute is per device and the call costs microseconds.
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(DSmem<E>));
  if (e != cudaSuccess) return e;
  dim3 grid((p.M + E::BM - 1) / E::BM, (p.N + E::BN - 1) / E::BN);
  kernel_timer_start(st);
  kern<<<grid, NT, sizeof(DSmem<E>), st>>>(*tmA, *tmB, p);
  kernel_timer_stop(st);
  return cudaGetLastError();
}

template <class E, bool FT>
cudaError_t launch_layout(const DgemmParams& p, const CUtensorMap* tmA, const CUtensorMap* tmB, cudaStream_t st) {
  if (p.a_kmajor) {
    return p.b_kmajor ? launch_one<E, true, true, FT>(p, tmA, tmB, st) : launch_one<E, true, false, FT>(p, tmA, tmB, st);
  }
  return p.b_kmajor ? launch_one<E, false, true, FT>(p, tmA, tmB, st) : launch_one<E, false, false, FT>(p, tmA, tmB, st);
}

}  // namespace

cudaError_t launch_dgemm(const DgemmParams& p, const CUtensorMap* tmA, const CUtensorMap* tmB, bool ft, int engine,
                         int tile_edge, cudaStream_t stream) {
  if (engine == kEngineDMMA) {
    if (tile_edge != EngineDMMA::BM) return cudaErrorInvalidValue;
    return ft ? launch_layout<EngineDMMA, true>(p, tmA, tmB, stream) : launch_layout<EngineDMMA, false>(p, tmA, tmB, stream);
  }
  using Dfma128 = EngineDFMA<8, 8>;
  using Dfma64 = EngineDFMA<4, 4>;
  if (tile_edge == Dfma64::BM) {
    return ft ? launch_layout<Dfma64, true>(p, tmA, tmB, stream) : launch_layout<Dfma64, false>(p, tmA, tmB, stream);
  }
  if (tile_edge != Dfma128::BM) return cudaErrorInvalidValue;
  return ft ? launch_layout<Dfma128, true>(p, tmA, tmB, stream) : launch_layout<Dfma128, false>(p, tmA, tmB, stream);
}

cudaError_t launch_scale(double* C, int64_t ldc, int32_t M, int32_t N, double beta, cudaStream_t stream) {
  const int64_t total = (int64_t)M * N;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks < 1) blocks = 1;
  scale_kernel<<<blocks, 256, 0, stream>>>(C, ldc, M, N, beta);
  return cudaGetLastError();
}

cudaError_t launch_expand(const double* X, int64_t ldx, bool row_major, int64_t n, int mode, bool upper, bool trans,
                          bool unit_diag, double* T, cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  int64_t blocks = (n * n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  expand_kernel<<<(unsigned)blocks, 256, 0, stream>>>(X, ldx, row_major ? 1 : 0, n, mode, upper ? 1 : 0,
                                                      trans ? 1 : 0, unit_diag ? 1 : 0, T);
  return cudaGetLastError();
}

}  // namespace ftk
