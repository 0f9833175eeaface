// FT-DTRSM building blocks (the paper's Level-3 family beside GEMM): the strided copy that
// brings B into the column-major solve frame, the protected diagonal-block solve, and the
// merge of the per-step reports. The blocked substitution itself (host side) runs its
// trailing updates through the protected FP64 GEMM.
//
// Diagonal-block solve with a checksum (Section II.A applied to T X = R): for an n x n
// triangular block T and right-hand sides R, e^T (T X) = (e^T T) X must equal e^T R for
// every column. Columns are independent, so a column whose checksum mismatches is solved
// again from the untouched R (same arithmetic: the fault-free result bit for bit); several
// faulty columns are all corrected.
//
// The substitution is blocked by kBlk rows. Each diagonal kBlk x kBlk block is solved by
// kGroups threads per column: the owner of row r forms x_r = w_r / T(r,r) (as w_r times the
// reciprocal, one rounding more than a division, inside the checksum's bound), broadcasts it
// by warp shuffle, and each thread eliminates it from its own rows of the block. Then the
// rows still to come are updated by all threads, each output as a kBlk-term fused
// multiply-add chain in ascending k, four rows per thread at a time so that four
// independent chains hide the FP64 latency. On GB300's FP64 pipe the updates, which hold
// almost all the work, then keep every warp busy. The one-thread re-solve of a column uses
// exactly the same arithmetic, so its result is the fault-free one bit for bit.
#include <climits>

#include "ft_device.cuh"
#include "ft_internal.h"

namespace ftk {

namespace {

constexpr int kLeaf = kTrsmLeaf;  // diagonal block edge (<= 128)
constexpr int kCols = 64;         // right-hand sides per CTA
constexpr int kThreads = 256;     // all threads stage, update and write back
constexpr int kBlk = 16;          // rows per diagonal block of the blocked substitution
constexpr int kGroups = kThreads / kCols;  // threads sharing one column (its rows by residue)
static_assert(kGroups * kCols == kThreads && 32 % kGroups == 0, "a column's threads share one warp");


// dst(r, c) = scale * src[r * rs + c * cs], dst column-major with leading dimension ld.
// 32 x 32 tiles; when the source is contiguous along c the tile goes through shared memory
// so that both the loads and the stores are coalesced.
__global__ void copy2d_kernel(const double* src, int64_t rs, int64_t cs, double* dst, int64_t ld, int64_t rows,
                              int64_t cols, double scale) {
  __shared__ double tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32, c0 = (int64_t)blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  if (rs == 1 || cs != 1) {
    for (int q = ty; q < 32; q += 8) {
      const int64_t r = r0 + tx, c = c0 + q;
      if (r < rows && c < cols) dst[r + c * ld] = scale * src[r * rs + c * cs];
    }
    return;
  }
  for (int q = ty; q < 32; q += 8) {
    const int64_t r = r0 + q, c = c0 + tx;
    tile[q][tx] = (r < rows && c < cols) ? src[r * rs + c] : 0.0;
  }
  __syncthreads();
  for (int q = ty; q < 32; q += 8) {
    const int64_t r = r0 + tx, c = c0 + q;
    if (r < rows && c < cols) dst[r + c * ld] = scale * tile[tx][q];
  }
}

__device__ __forceinline__ double gamma_up64(int64_t n) {
  const double nu = __dmul_ru((double)n, 0x1p-53);
  return __ddiv_ru(nu, __dsub_rd(1.0, nu));
}

// The triangle of the block packed by columns: lower, column r holds rows r..n-1 from
// r n - r (r - 1) / 2; upper, column r holds rows 0..r from r (r + 1) / 2.
__device__ __forceinline__ int packed(int s, int r, int n, bool lower) {
  return lower ? r * n - r * (r - 1) / 2 + (s - r) : r * (r + 1) / 2 + s;
}

struct LeafSmem {
  double T[kLeaf * (kLeaf + 1) / 2];  // the block's triangle, packed by columns
  double w[kLeaf][kCols];             // w[row][column]: right-hand side, then solution
  double wf[kLeaf][kCols];            // a faulty solution kept while its column is solved again
  double tsum[kLeaf], tabs[kLeaf];    // column sums of T and of |T|
  double inv_d[kLeaf];                // 1 / T(r,r)
};

// Element (s, r) of the block (in its stored triangle).
__device__ __forceinline__ double tri(const LeafSmem& sm, int s, int r, int n, bool lower) {
  return sm.T[packed(s, r, n, lower)];
}

// Rows [r0, r1) of diagonal block b in solve order: lower (forward) from the top, upper
// (backward) from the bottom.
__device__ __forceinline__ void block_rows(int bi, int n, bool lower, int& r0, int& r1) {
  const int nb = (n + kBlk - 1) / kBlk;
  const int b = lower ? bi : nb - 1 - bi;
  r0 = b * kBlk;
  r1 = min(n, r0 + kBlk);
}

// Substitution within diagonal block [r0, r1) for column t held in sm.w[.][t], by one thread:
// x_r = w_r (1 / T(r,r)), then w_s -= T(s,r) x_r for the block's rows still to come, in the
// order of the CTA-wide version below (the re-solve of a column).
__device__ void solve_diag_block(LeafSmem& sm, int t, int r0, int r1, int n, bool lower) {
  for (int q = r0; q < r1; ++q) {
    const int r = lower ? q : r0 + r1 - 1 - q;
    const double x = sm.w[r][t] * sm.inv_d[r];
    sm.w[r][t] = x;
    if (lower) {
      for (int s2 = r + 1; s2 < r1; ++s2) sm.w[s2][t] = fma(-tri(sm, s2, r, n, lower), x, sm.w[s2][t]);
    } else {
      for (int s2 = r0; s2 < r; ++s2) sm.w[s2][t] = fma(-tri(sm, s2, r, n, lower), x, sm.w[s2][t]);
    }
  }
}

// The same substitution by the kGroups threads of column c (lanes kGroups c .. kGroups c +
// kGroups - 1 of one warp): thread g owns the rows r with r % kGroups == g, forms x_r for
// those and updates only those, and each x_r reaches the others by a warp shuffle. Every
// element receives its updates in the same order as in solve_diag_block. An injection point
// at row inj_r flips bit inj_bit of x_r right after it is formed (test launches only).
__device__ void solve_diag_block_par(LeafSmem& sm, int c, int g, int r0, int r1, int n, bool lower, int inj_r,
                                     int inj_bit) {
  const int lane = threadIdx.x & 31;
  for (int q = r0; q < r1; ++q) {
    const int r = lower ? q : r0 + r1 - 1 - q;
    const int owner = r % kGroups;
    double x = 0.0;
    if (g == owner) {
      x = sm.w[r][c] * sm.inv_d[r];
      if (r == inj_r) x = __longlong_as_double(__double_as_longlong(x) ^ (1ll << inj_bit));
      sm.w[r][c] = x;
    }
    x = __shfl_sync(0xffffffffu, x, (lane & ~(kGroups - 1)) | owner);
    // this thread's rows only (a predicated-off FMA would still take a slot of the FP64 pipe)
    if (lower) {
      const int first = r + 1 + ((g - (r + 1)) % kGroups + kGroups) % kGroups;
      for (int s2 = first; s2 < r1; s2 += kGroups) sm.w[s2][c] = fma(-tri(sm, s2, r, n, lower), x, sm.w[s2][c]);
    } else {
      const int first = r0 + ((g - r0) % kGroups + kGroups) % kGroups;
      for (int s2 = first; s2 < r; s2 += kGroups) sm.w[s2][c] = fma(-tri(sm, s2, r, n, lower), x, sm.w[s2][c]);
    }
  }
}

// Update of row `row` of column t by diagonal block [r0, r1): w_row -= sum_k T(row,k) x_k as
// one fused multiply-add chain in ascending k (x_k = sm.w[k][t], already solved).
__device__ __forceinline__ void update_row(LeafSmem& sm, int t, int row, int r0, int r1, int n, bool lower) {
  double acc = sm.w[row][t];
  for (int k = r0; k < r1; ++k) acc = fma(-tri(sm, row, k, n, lower), sm.w[k][t], acc);
  sm.w[row][t] = acc;
}

// Rows a diagonal block updates: lower, those after it; upper, those before it.
__device__ __forceinline__ void update_range(int r0, int r1, int n, bool lower, int& lo, int& hi) {
  lo = lower ? r1 : 0;
  hi = lower ? n : r0;
}

// The whole blocked substitution of column t by one thread, with the arithmetic of the
// CTA-wide solve (the re-solve of a column whose checksum mismatched).
__device__ void solve_column(LeafSmem& sm, int t, int n, bool lower) {
  const int nb = (n + kBlk - 1) / kBlk;
  for (int bi = 0; bi < nb; ++bi) {
    int r0, r1, lo, hi;
    block_rows(bi, n, lower, r0, r1);
    solve_diag_block(sm, t, r0, r1, n, lower);
    update_range(r0, r1, n, lower, lo, hi);
    for (int row = lo; row < hi; ++row) update_row(sm, t, row, r0, r1, n, lower);
  }
}

// One CTA: kCols right-hand sides of the n x n diagonal block at T (column-major, ld ldt);
// W (column-major, ld ldw) is overwritten with the solution. rep: this step's report.
__global__ void __launch_bounds__(kThreads) trsm_leaf_kernel(const double* T, int64_t ldt, double* W, int64_t ldw,
                                                             int n, int64_t nrhs, int lower, ft_report_t* rep,
                                                             InjectList inj) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  LeafSmem& sm = *reinterpret_cast<LeafSmem*>(smem_raw);
  const int tid = threadIdx.x;
  const int64_t j0 = (int64_t)blockIdx.x * kCols;
  const int ncols = (int)min((int64_t)kCols, nrhs - j0);
  const bool low = lower != 0;
  // stage the triangle (coalesced along each column) and the right-hand sides
  for (int r = 0; r < n; ++r) {
    const int lo = low ? r : 0, hi = low ? n : r + 1;  // stored rows of column r
    for (int s2 = lo + tid; s2 < hi; s2 += kThreads) sm.T[packed(s2, r, n, low)] = T[s2 + (int64_t)r * ldt];
  }
  for (int e = tid; e < n * kCols; e += kThreads) {
    const int r = e % n, c = e / n;
    sm.w[r][c] = c < ncols ? W[r + (j0 + c) * ldw] : 0.0;
  }
  __syncthreads();
  for (int c = tid; c < n; c += kThreads) {
    const double* col = sm.T + packed(low ? c : 0, c, n, low);
    const int len = low ? n - c : c + 1;
    double s = 0.0, a = 0.0;
    for (int q = 0; q < len; ++q) { s += col[q]; a = __dadd_ru(a, fabs(col[q])); }
    sm.tsum[c] = s;
    sm.tabs[c] = a;
    sm.inv_d[c] = 1.0 / tri(sm, c, c, n, low);
  }
  __syncthreads();
  // the right-hand side's sums (threads t < kCols), read before the substitution overwrites
  // the column
  const int t = tid;
  const int64_t j = j0 + t;
  const bool jok = t < kCols && t < ncols;
  double rsum = 0.0, rabs = 0.0;
  if (t < kCols)
    for (int r = 0; r < n; ++r) { rsum += sm.w[r][t]; rabs = __dadd_ru(rabs, fabs(sm.w[r][t])); }
  // this thread's column in the diagonal solves (kGroups lanes per column) and its injection
  // point
  const int dc = tid / kGroups, dg = tid % kGroups;
  int inj_r = -1, inj_bit = 0;
  for (int e = 0; e < inj.n; ++e)
    if (dc < ncols && inj.p[e].j == j0 + dc && inj.p[e].i >= 0 && inj.p[e].i < n &&
        inj.p[e].mode == FT_MODE_BITFLIP) {
      inj_r = inj.p[e].i;
      inj_bit = inj.p[e].bit;
    }
  __syncthreads();
  // blocked substitution: each diagonal block by kGroups threads per column, then the updates
  // of the rows still to come by all threads (kGroups threads per column, interleaved rows);
  // the solved values of the block are held in registers for the updates
  const int nb = (n + kBlk - 1) / kBlk;
  const int uc = tid % kCols, ug = tid / kCols;
  for (int bi = 0; bi < nb; ++bi) {
    int r0, r1, lo, hi;
    block_rows(bi, n, low, r0, r1);
    solve_diag_block_par(sm, dc, dg, r0, r1, n, low, inj_r, inj_bit);
    __syncthreads();
    update_range(r0, r1, n, low, lo, hi);
    double xk[kBlk];
#pragma unroll
    for (int k = 0; k < kBlk; ++k) xk[k] = r0 + k < r1 ? sm.w[r0 + k][uc] : 0.0;
    // four rows at a time: four independent chains hide the FP64 latency; each row's chain is
    // that of update_row
    constexpr int kRows = 4;
    for (int row = lo + ug; row < hi; row += kGroups * kRows) {
      double acc[kRows];
#pragma unroll
      for (int q = 0; q < kRows; ++q) {
        const int rr = row + q * kGroups;
        acc[q] = rr < hi ? sm.w[rr][uc] : 0.0;
      }
#pragma unroll
      for (int k = 0; k < kBlk; ++k) {
        if (r0 + k < r1) {
#pragma unroll
          for (int q = 0; q < kRows; ++q) {
            const int rr = row + q * kGroups;
            if (rr < hi) acc[q] = fma(-tri(sm, rr, r0 + k, n, low), xk[k], acc[q]);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < kRows; ++q) {
        const int rr = row + q * kGroups;
        if (rr < hi) sm.w[rr][uc] = acc[q];
      }
    }
    __syncthreads();
  }
  if (jok) {
    // e^T T x against e^T r: tau = 2 gamma_{2n+2} (sum_s (e^T|T|)_s |x_s| + sum |r|), a bound on
    // the substitution's residual (componentwise backward error gamma_n |T| |x|) plus the
    // rounding of both sums.
    double chk = 0.0, mag = 0.0;
    for (int s2 = 0; s2 < n; ++s2) {
      const double x = sm.w[s2][t];
      chk = fma(sm.tsum[s2], x, chk);
      mag = __fma_ru(sm.tabs[s2], fabs(x), mag);
    }
    const double delta = chk - rsum;
    const double tau = __dmul_ru(2.0, __dmul_ru(gamma_up64(2 * (int64_t)n + 2), __dadd_ru(mag, rabs)));
    if (!(fabs(delta) <= tau) || isinf(delta)) {
      // keep the faulty solution, solve again from the untouched right-hand side in W
      for (int r = 0; r < n; ++r) { sm.wf[r][t] = sm.w[r][t]; sm.w[r][t] = W[r + j * ldw]; }
      solve_column(sm, t, n, low);
      int first = -1;  // where the fault entered: the first row, in solve order, that differs
      for (int q = 0; q < n && first < 0; ++q) {
        const int r = low ? q : n - 1 - q;
        if (__double_as_longlong(sm.wf[r][t]) != __double_as_longlong(sm.w[r][t])) first = r;
      }
      if (rep) {
        atomicAdd(reinterpret_cast<unsigned long long*>(&rep->detected), 1ull);
        atomicAdd(reinterpret_cast<unsigned long long*>(&rep->corrected), 1ull);
        const unsigned slot = atomicAdd(&rep->n_records, 1u);
        if (slot < FTBLAS_MAX_RECORDS) {
          ft_error_record_t& rc = rep->rec[slot];
          rc.tile_row = 0; rc.tile_col = blockIdx.x;
          rc.i = first; rc.j = j;
          rc.delta_row = 0.0; rc.delta_col = delta; rc.tau_row = 0.0; rc.tau_col = tau;
          rc.value_before = first >= 0 ? sm.wf[first][t] : 0.0;
          rc.value_after = first >= 0 ? sm.w[first][t] : 0.0;
          rc.rows_flagged = 0; rc.cols_flagged = 1;
          rc.kind = FT_KIND_CORRECTED;
          rc.reserved = 0;
        } else {
          atomicOr(&rep->status, FT_STATUS_RECORDS_TRUNCATED);
        }
      }
    }
  }
  if (rep && tid == 0) atomicAdd(reinterpret_cast<unsigned long long*>(&rep->tiles_checked), 1ull);
  __syncthreads();
  for (int e = tid; e < n * ncols; e += kThreads) {  // coalesced write-back
    const int r = e % n, c = e / n;
    W[r + (j0 + c) * ldw] = sm.w[r][c];
  }
}

// Sum the step reports into `out` (zeroed by the caller): counters added, status ORed,
// records concatenated in step order with coordinates moved from each step's frame
// (rows + row_off[p]) to the caller's (swapped when `swap`).
__global__ void report_merge_kernel(const ft_report_t* parts, const int64_t* row_off, int nparts, ft_report_t* out,
                                    int swap) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  unsigned n = 0;
  for (int q = 0; q < nparts; ++q) {
    const ft_report_t& r = parts[q];
    out->tiles_checked += r.tiles_checked;
    out->detected += r.detected;
    out->corrected += r.corrected;
    out->uncorrectable += r.uncorrectable;
    out->checksum_only += r.checksum_only;
    out->input_nonfinite += r.input_nonfinite;
    out->status |= r.status;
    const unsigned m = r.n_records < FTBLAS_MAX_RECORDS ? r.n_records : FTBLAS_MAX_RECORDS;
    for (unsigned k = 0; k < m; ++k) {
      if (n >= FTBLAS_MAX_RECORDS) { out->status |= FT_STATUS_RECORDS_TRUNCATED; break; }
      ft_error_record_t rc = r.rec[k];
      const int64_t i = rc.i >= 0 ? rc.i + row_off[q] : -1, j = rc.j;
      rc.i = swap ? j : i;
      rc.j = swap ? i : j;
      out->rec[n++] = rc;
    }
  }
  out->n_records = n;
}

}  // namespace

cudaError_t launch_copy2d(const double* src, int64_t rs, int64_t cs, double* dst, int64_t ld, int64_t rows,
                          int64_t cols, double scale, cudaStream_t st) {
  if (rows == 0 || cols == 0) return cudaSuccess;
  // gridDim.y is at most 65535: wider copies go in column chunks of 65535 x 32
  constexpr int64_t kChunk = 65535 * 32;
  for (int64_t c0 = 0; c0 < cols; c0 += kChunk) {
    const int64_t nc = cols - c0 < kChunk ? cols - c0 : kChunk;
    dim3 grid((unsigned)((rows + 31) / 32), (unsigned)((nc + 31) / 32));
    copy2d_kernel<<<grid, dim3(32, 8), 0, st>>>(src + c0 * cs, rs, cs, dst + c0 * ld, ld, rows, nc, scale);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_trsm_leaf(const double* T, int64_t ldt, double* W, int64_t ldw, int n, int64_t nrhs, bool lower,
                             ft_report_t* rep, const InjectList& inj, cudaStream_t st) {
  if (n == 0 || nrhs == 0) return cudaSuccess;
  const size_t smem = sizeof(LeafSmem);
  cudaError_t e = cudaFuncSetAttribute(trsm_leaf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  trsm_leaf_kernel<<<(unsigned)((nrhs + kCols - 1) / kCols), kThreads, smem, st>>>(T, ldt, W, ldw, n, nrhs,
                                                                                      lower ? 1 : 0, rep, inj);
  return cudaGetLastError();
}

cudaError_t launch_report_merge(const ft_report_t* parts, const int64_t* row_off, int nparts, ft_report_t* out,
                                bool swap, cudaStream_t st) {
  report_merge_kernel<<<1, 32, 0, st>>>(parts, row_off, nparts, out, swap ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace ftk
