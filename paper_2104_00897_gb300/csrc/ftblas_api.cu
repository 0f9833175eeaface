// Host side of the C ABI declared in include/ftblas.h: argument validation (BLAS xerbla
// style), the layout/transpose mapping to the column-major kernel frame, TMA descriptors,
// the injection plan, and the host-buffer variant. No compute happens here: every step of
// the product, encode, verification and correction runs in the kernels.
#include <cudaTypedefs.h>

#include <atomic>
#include <cstring>
#include <mutex>
#include <vector>

#include "ft_emu.h"
#include "ft_internal.h"
#include "ft_tc.h"

using namespace ftk;

namespace {

thread_local int g_last_cuda_error = 0;
thread_local int g_last_used_tma = -1;
std::atomic<int> g_fp64_engine{kEngineDFMA};
std::atomic<int> g_tc_cta_group{0};  // 0: the library's choice (CTA pairs); 1 or 2 forced
std::atomic<int> g_fp64_tile{0};  // 0: fp64_tile_edge decides; else the forced DFMA tile edge
std::atomic<int64_t> g_kc_interval{0};
std::atomic<int> g_emu_slices{kEmuSlicesDefault};

// ------------------------------------------------------------------ injection plan state
std::mutex g_inj_mu;
bool g_inj_on = false;
ft_inject_t g_inj;
uint64_t g_launch = 0;

int record_cuda(cudaError_t e) {
  if (e == cudaSuccess) return 0;
  g_last_cuda_error = static_cast<int>(e);
  return FTBLAS_STATUS_CUDA_ERROR;
}

// SMs of the current device; 152 (GB300) when no device answers, so that the geometry
// queries also work on a machine without a GPU.
int current_sm_count() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
      v > 0)
    return v;
  (void)cudaGetLastError();
  return 152;
}

// SplitMix64 step (Steele, Lea and Flood, OOPSLA 2014).
uint64_t splitmix_next(uint64_t& s) {
  s += 0x9E3779B97F4A7C15ull;
  uint64_t z = s;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct CallerPoint {
  int64_t i, j;
  int32_t site, mode, bit, rel_log2, sign, kt;
};

// The points injected into this launch, in the caller's coordinates. The seeded draw is
// the one documented beside ftblas_set_injection in the header.
int plan_injections(int64_t M, int64_t N, int64_t tile_rows, int64_t tile_cols, CallerPoint* out) {
  std::lock_guard<std::mutex> lk(g_inj_mu);
  const uint64_t launch = g_launch++;
  if (!g_inj_on) return 0;
  const ft_inject_t& c = g_inj;
  int n = 0;
  if (c.n_fixed > 0) {
    for (int q = 0; q < c.n_fixed && n < kMaxInject; ++q) {
      const ft_inject_point_t& f = c.fixed[q];
      if (f.i < 0 || f.i >= M || f.j < 0 || f.j >= N) continue;
      out[n++] = CallerPoint{f.i, f.j, f.site, f.mode, f.bit, f.rel_log2, f.sign, f.k_tile};
    }
    return n;
  }
  if (c.every_n_launches <= 0 || c.errors_per_launch <= 0) return 0;
  const uint64_t every = static_cast<uint64_t>(c.every_n_launches);
  if (launch % every != c.seed % every) return 0;
  const int64_t tr = (M + tile_rows - 1) / tile_rows, tc = (N + tile_cols - 1) / tile_cols;
  const int64_t ntiles = tr * tc;
  int64_t want = c.errors_per_launch;
  if (want > ntiles) want = ntiles;
  if (want > kMaxInject) want = kMaxInject;
  uint64_t st = c.seed ^ (launch * 0xD1B54A32D192ED03ull);
  while (n < want) {
    const uint64_t t = splitmix_next(st) % static_cast<uint64_t>(ntiles);
    const uint64_t ri = splitmix_next(st), rj = splitmix_next(st), rb = splitmix_next(st);
    const uint64_t rp = splitmix_next(st), rs = splitmix_next(st);
    const int64_t trow = static_cast<int64_t>(t) % tr, tcol = static_cast<int64_t>(t) / tr;
    bool dup = false;
    for (int q = 0; q < n; ++q)
      if (out[q].i / tile_rows == trow && out[q].j / tile_cols == tcol) dup = true;
    if (dup) continue;
    const int64_t rows = (trow == tr - 1) ? M - trow * tile_rows : tile_rows;
    const int64_t cols = (tcol == tc - 1) ? N - tcol * tile_cols : tile_cols;
    CallerPoint& pnt = out[n++];
    pnt.i = trow * tile_rows + static_cast<int64_t>(ri % static_cast<uint64_t>(rows));
    pnt.j = tcol * tile_cols + static_cast<int64_t>(rj % static_cast<uint64_t>(cols));
    pnt.site = c.site;
    pnt.mode = c.mode;
    pnt.bit = c.bit_lo + static_cast<int32_t>(rb % static_cast<uint64_t>(c.bit_hi - c.bit_lo + 1));
    pnt.rel_log2 = c.log2_lo + static_cast<int32_t>(rp % static_cast<uint64_t>(c.log2_hi - c.log2_lo + 1));
    pnt.sign = (rs & 1) ? -1 : 1;
    pnt.kt = 0;
  }
  return n;
}

// ------------------------------------------------------------------ TMA descriptors
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// 2-D FP64 tensor map: `inner` contiguous elements, `outer` lines `ld` elements apart.
bool make_map_f64(CUtensorMap* map, const void* base, int64_t inner, int64_t outer, int64_t ld, uint32_t box_inner,
                  uint32_t box_outer) {
  auto fn = encode_fn();
  if (!fn) return false;
  if ((reinterpret_cast<uintptr_t>(base) & 15u) != 0) return false;
  if (((ld * 8) & 15) != 0 || ld * 8 >= (int64_t(1) << 40)) return false;
  if (inner <= 0 || outer <= 0 || inner > (int64_t(1) << 32) || outer > (int64_t(1) << 32)) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(inner), static_cast<cuuint64_t>(outer)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld * 8)};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// 2-D 16-bit tensor map with 128-byte swizzle: `inner` K-contiguous elements per line.
// 2-D map of 2-byte (BF16) or 1-byte (FP8) elements, 128-byte swizzle: the box's inner
// extent is 128 bytes (one swizzle row). Leading dimensions must be a multiple of 16 bytes
// and the base 16-byte aligned (else false: the caller reports FTBLAS_STATUS_NOT_SUPPORTED).
bool make_map_sw128(CUtensorMap* map, int elem_bytes, const void* base, int64_t inner, int64_t outer,
                    int64_t ld_elems, uint32_t box_outer) {
  auto fn = encode_fn();
  if (!fn) return false;
  if ((reinterpret_cast<uintptr_t>(base) & 15u) != 0) return false;
  if (((ld_elems * elem_bytes) & 15) != 0 || ld_elems * elem_bytes >= (int64_t(1) << 40)) return false;
  if (inner <= 0 || outer <= 0 || inner > (int64_t(1) << 32) || outer > (int64_t(1) << 32)) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(inner), static_cast<cuuint64_t>(outer)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld_elems * elem_bytes)};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(128 / elem_bytes), box_outer};
  cuuint32_t estr[2] = {1, 1};
  const CUtensorMapDataType dt = elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8;
  CUresult r = fn(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// ------------------------------------------------------------------ validation
struct Frame {
  // kernel frame (column-major): C' = alpha op(A') op(B') + beta C'
  int64_t M, N;
  const void* A;
  int64_t lda;
  const void* B;
  int64_t ldb;
  bool a_kmajor, b_kmajor, swap;
};

int validate(int layout, int ta, int tb, int64_t M, int64_t N, int64_t K, const void* A, int64_t lda, const void* B,
             int64_t ldb, const void* C, int64_t ldc, bool need_ab) {
  if (layout != FTBLAS_ROW_MAJOR && layout != FTBLAS_COL_MAJOR) return -1;
  if (ta != FTBLAS_NO_TRANS && ta != FTBLAS_TRANS) return -2;
  if (tb != FTBLAS_NO_TRANS && tb != FTBLAS_TRANS) return -3;
  if (M < 0) return -4;
  if (N < 0) return -5;
  if (K < 0) return -6;
  const bool col = layout == FTBLAS_COL_MAJOR;
  // rows / cols of the stored A and B
  const int64_t a_rows = (ta == FTBLAS_NO_TRANS) ? M : K, a_cols = (ta == FTBLAS_NO_TRANS) ? K : M;
  const int64_t b_rows = (tb == FTBLAS_NO_TRANS) ? K : N, b_cols = (tb == FTBLAS_NO_TRANS) ? N : K;
  const int64_t need_lda = col ? (a_rows > 1 ? a_rows : 1) : (a_cols > 1 ? a_cols : 1);
  const int64_t need_ldb = col ? (b_rows > 1 ? b_rows : 1) : (b_cols > 1 ? b_cols : 1);
  const int64_t need_ldc = col ? (M > 1 ? M : 1) : (N > 1 ? N : 1);
  if (need_ab && A == nullptr) return -8;
  if (lda < need_lda) return -9;
  if (need_ab && B == nullptr) return -10;
  if (ldb < need_ldb) return -11;
  if (M > 0 && N > 0 && C == nullptr) return -13;
  if (ldc < need_ldc) return -14;
  return 0;
}

Frame map_frame(int layout, int ta, int tb, int64_t M, int64_t N, const void* A, int64_t lda, const void* B,
                int64_t ldb) {
  Frame f;
  if (layout == FTBLAS_COL_MAJOR) {
    f = Frame{M, N, A, lda, B, ldb, ta == FTBLAS_TRANS, tb == FTBLAS_NO_TRANS, false};
  } else {
    // C^T = op(B)^T op(A)^T over the same memory read column-major.
    f = Frame{N, M, B, ldb, A, lda, tb == FTBLAS_TRANS, ta == FTBLAS_NO_TRANS, true};
  }
  return f;
}

constexpr int64_t kMaxDim = (int64_t(1) << 31) - 256;

}  // namespace

int ftk::fp64_tile_edge(int64_t M, int64_t N, int engine, int sm_count) {
  if (engine == kEngineDMMA || M <= 0 || N <= 0 || sm_count <= 0) return kDBM;
  // busy fraction of the SMs over the waves of one CTA per tile, divided by the work per
  // product operation (1 + 4 / edge: encode and predicted checksums over the tile's edges)
  auto score = [&](int64_t e) {
    const int64_t tiles = ((M + e - 1) / e) * ((N + e - 1) / e);
    const int64_t waves = (tiles + sm_count - 1) / sm_count;
    return (double)tiles / (double)(waves * sm_count) / (1.0 + 4.0 / (double)e);
  };
  return score(kDBSmall) > 1.03 * score(kDBM) ? kDBSmall : kDBM;
}

namespace {

// The FP64 tile edge of a kernel-frame M x N call: DMMA's only edge, the forced DFMA edge
// (ftblas_set_fp64_tile), else the rule of fp64_tile_edge.
int chosen_fp64_edge(int64_t M, int64_t N, int engine) {
  if (engine == kEngineDMMA) return kDBM;
  const int forced = g_fp64_tile.load();
  return forced != 0 ? forced : fp64_tile_edge(M, N, engine, current_sm_count());
}

// tri_a / tri_b: op(A) / op(B) triangular in the caller's frame (0 no, 1 upper, 2 lower):
// the kernel then runs, per tile, only the k-tiles the nonzero triangle reaches.
int dgemm_impl(int layout, int ta, int tb, int64_t M, int64_t N, int64_t K, double alpha, const double* A,
               int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc, void* stream,
               ft_report_t* report, bool ft, int tri_a = 0, int tri_b = 0) {
  const bool need_ab = (K > 0 && alpha != 0.0 && M > 0 && N > 0);
  int v = validate(layout, ta, tb, M, N, K, A, lda, B, ldb, C, ldc, need_ab);
  if (v != 0) return v;
  if (M > kMaxDim || N > kMaxDim || K > kMaxDim) return FTBLAS_STATUS_NOT_SUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (ft && report != nullptr) {
    if (int e = record_cuda(cudaMemsetAsync(report, 0, sizeof(ft_report_t), st))) return e;
  }
  if (M == 0 || N == 0) return 0;
  const Frame f = map_frame(layout, ta, tb, M, N, A, lda, B, ldb);
  const int engine = g_fp64_engine.load();
  const int edge = chosen_fp64_edge(f.M, f.N, engine);  // square tiles
  CallerPoint pts[kMaxInject];
  int npts = 0;
  if (ft) npts = plan_injections(M, N, edge, edge, pts);
  if (K == 0 || alpha == 0.0) return record_cuda(launch_scale(C, ldc, (int32_t)f.M, (int32_t)f.N, beta, st));

  DgemmParams p;
  std::memset(&p, 0, sizeof(p));
  p.M = (int32_t)f.M; p.N = (int32_t)f.N; p.K = (int32_t)K;
  p.alpha = alpha; p.beta = beta;
  p.A = static_cast<const double*>(f.A); p.lda = f.lda;
  p.B = static_cast<const double*>(f.B); p.ldb = f.ldb;
  p.C = C; p.ldc = ldc;
  p.a_kmajor = f.a_kmajor; p.b_kmajor = f.b_kmajor;
  p.report = ft ? report : nullptr;
  p.swap_report = f.swap;
  {
    // row-major: the kernel frame computes C^T = op(B)^T op(A)^T, and a transpose swaps
    // upper and lower
    auto flip = [](int t) { return t == 1 ? 2 : (t == 2 ? 1 : 0); };
    p.tri_a = f.swap ? flip(tri_b) : tri_a;
    p.tri_b = f.swap ? flip(tri_a) : tri_b;
  }
  {
    const int64_t kc = g_kc_interval.load();
    p.kc_tiles = (ft && kc > 0) ? (int32_t)((kc + kDBK - 1) / kDBK) : 0;
  }
  p.inj.n = 0;
  bool stall = false;
  for (int q = 0; q < npts; ++q) {
    InjectPoint& ip = p.inj.p[p.inj.n++];
    const CallerPoint& c = pts[q];
    ip.i = (int32_t)(f.swap ? c.j : c.i);
    ip.j = (int32_t)(f.swap ? c.i : c.j);
    ip.site = c.site == FT_SITE_CHECKSUM ? (f.swap ? kSiteChecksumCol : kSiteChecksumRow)
              : c.site == FT_SITE_STALL  ? kSiteStall
                                         : c.site;
    ip.mode = c.mode; ip.bit = c.bit; ip.rel_log2 = c.rel_log2; ip.sign = c.sign; ip.kt = c.kt;
    stall |= c.site == FT_SITE_STALL;
  }
  // a bounded wait normally gives up after 4 s (a k-tile takes about 0.1 ms); with a stall
  // point planned, after 20 ms, so that its test ends quickly
  p.wait_limit_ns = stall ? 20000000ull : 4000000000ull;
  CUtensorMap tmA, tmB;
  std::memset(&tmA, 0, sizeof(tmA));
  std::memset(&tmB, 0, sizeof(tmB));
  const uint32_t be = (uint32_t)edge;
  bool ok = f.a_kmajor ? make_map_f64(&tmA, f.A, K, f.M, f.lda, kDBK, be)
                       : make_map_f64(&tmA, f.A, f.M, K, f.lda, be, kDBK);
  ok = ok && (f.b_kmajor ? make_map_f64(&tmB, f.B, K, f.N, f.ldb, kDBK, be)
                         : make_map_f64(&tmB, f.B, f.N, K, f.ldb, be, kDBK));
  p.use_tma = ok ? 1 : 0;
  g_last_used_tma = p.use_tma;
  return record_cuda(launch_dgemm(p, &tmA, &tmB, ft, engine, edge, st));
}

// ------------------------------------------------------------------ FT-DSYMM, FT-DTRMM
// Both run the protected FP64 GEMM on a full copy of the symmetric or triangular operand
// (the analogue of the paper's symmetric / triangular packing before the Level-3 kernel).
int dsymm_impl(int layout, int side, int uplo, int64_t M, int64_t N, double alpha, const double* A, int64_t lda,
               const double* B, int64_t ldb, double beta, double* C, int64_t ldc, void* stream, ft_report_t* report) {
  if (layout != FTBLAS_ROW_MAJOR && layout != FTBLAS_COL_MAJOR) return -1;
  if (side != FTBLAS_LEFT && side != FTBLAS_RIGHT) return -2;
  if (uplo != FTBLAS_UPPER && uplo != FTBLAS_LOWER) return -3;
  if (M < 0) return -4;
  if (N < 0) return -5;
  const bool col = layout == FTBLAS_COL_MAJOR;
  const int64_t dim = side == FTBLAS_LEFT ? M : N;
  const bool need = M > 0 && N > 0 && alpha != 0.0;
  if (need && A == nullptr) return -7;
  if (lda < (dim > 1 ? dim : 1)) return -8;
  if (need && B == nullptr) return -9;
  const int64_t ld_mn = col ? M : N;
  if (ldb < (ld_mn > 1 ? ld_mn : 1)) return -10;
  if (M > 0 && N > 0 && C == nullptr) return -12;
  if (ldc < (ld_mn > 1 ? ld_mn : 1)) return -13;
  if (M > kMaxDim || N > kMaxDim) return FTBLAS_STATUS_NOT_SUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!need) {  // quick returns: an empty product (K = 0) gives C = beta C, or nothing
    const int64_t l1 = ld_mn > 1 ? ld_mn : 1;
    return dgemm_impl(layout, FTBLAS_NO_TRANS, FTBLAS_NO_TRANS, M, N, 0, 0.0, nullptr, l1, nullptr, l1, beta, C, ldc,
                      stream, report, true);
  }
  double* S = nullptr;
  if (ws_alloc(reinterpret_cast<void**>(&S), (size_t)(dim * dim) * 8, st) != cudaSuccess)
    return FTBLAS_STATUS_ALLOC_FAILED;
  int rc = record_cuda(launch_expand(A, lda, !col, dim, 0, uplo == FTBLAS_UPPER, false, false, S, st));
  if (rc == 0) {
    rc = side == FTBLAS_LEFT
             ? dgemm_impl(layout, FTBLAS_NO_TRANS, FTBLAS_NO_TRANS, M, N, M, alpha, S, dim, B, ldb, beta, C, ldc,
                          stream, report, true)
             : dgemm_impl(layout, FTBLAS_NO_TRANS, FTBLAS_NO_TRANS, M, N, N, alpha, B, ldb, S, dim, beta, C, ldc,
                          stream, report, true);
  }
  cudaFreeAsync(S, st);
  return rc;
}

// FT-DTRMM's tiles do unequal work: each visits only the k-tiles its triangle leaves
// nonzero, from all of K down to one. The kernel's launch order, which the block scheduler
// follows, runs row tiles fastest and column tiles slowest. So the heaviest tiles come
// first, and the lightest fill the last wave, exactly when the triangular operand is the
// kernel frame's op(B) and is lower (column tile j needs k >= j). With the triangular
// operand as the kernel's op(A), heavy and light tiles alternate. As op(B) upper, the
// heaviest come last. Running the product in the other storage layout transposes the
// kernel frame: op(A) becomes op(B) and upper becomes lower. Each element keeps the same
// products in the same k order, so the values are unchanged. The cost is a transposing
// copy of B in and of the result out.
// Placement score: 2 for op(B) lower, 1 for op(A), 0 for op(B) upper.
int tri_placement_score(bool on_a, int t) { return on_a ? 1 : (t == 2 ? 2 : 0); }

bool use_other_layout(bool col, bool left, int tri) {
  auto flip = [](int t) { return t == 1 ? 2 : 1; };
  // in the caller's layout: column-major puts op(A) of a left product in the kernel's op(A);
  // row-major swaps the kernel's operands and transposes them
  const bool on_a = col == left;
  const int t = col ? tri : flip(tri);
  return tri_placement_score(!on_a, flip(t)) > tri_placement_score(on_a, t);
}

int dtrmm_other_layout(bool col, int side, int uplo, int transa, int diag, int64_t M, int64_t N, double alpha,
                       const double* A, int64_t lda, double* B, int64_t ldb, cudaStream_t st, ft_report_t* report,
                       int tri, int64_t rows, int64_t cols) {
  // B's storage holds `cols` lines of `rows` contiguous elements; in the other layout the
  // copies Bt (the operand) and Ct (the product) hold `rows` lines of `cols`, ld = cols.
  const int64_t dim = side == FTBLAS_LEFT ? M : N;
  double* T = nullptr;
  if (ws_alloc(reinterpret_cast<void**>(&T), (size_t)(dim * dim + 2 * rows * cols) * 8, st) != cudaSuccess)
    return FTBLAS_STATUS_ALLOC_FAILED;
  double* Bt = T + dim * dim;
  double* Ct = Bt + rows * cols;
  // op(A)^T in the caller's layout is op(A) in the other one
  int rc = record_cuda(launch_expand(A, lda, !col, dim, 1, uplo == FTBLAS_UPPER, transa != FTBLAS_TRANS,
                                     diag == FTBLAS_UNIT, T, st));
  if (rc == 0) rc = record_cuda(launch_copy2d(B, ldb, 1, Bt, cols, cols, rows, 1.0, st));
  if (rc == 0) {
    const int other = col ? FTBLAS_ROW_MAJOR : FTBLAS_COL_MAJOR;
    rc = side == FTBLAS_LEFT
             ? dgemm_impl(other, FTBLAS_NO_TRANS, FTBLAS_NO_TRANS, M, N, M, alpha, T, dim, Bt, cols, 0.0, Ct, cols,
                          st, report, true, tri, 0)
             : dgemm_impl(other, FTBLAS_NO_TRANS, FTBLAS_NO_TRANS, M, N, N, alpha, Bt, cols, T, dim, 0.0, Ct, cols,
                          st, report, true, 0, tri);
  }
  if (rc == 0) rc = record_cuda(launch_copy2d(Ct, cols, 1, B, ldb, rows, cols, 1.0, st));
  cudaFreeAsync(T, st);
  return rc;
}

int dtrmm_impl(int layout, int side, int uplo, int transa, int diag, int64_t M, int64_t N, double alpha,
               const double* A, int64_t lda, double* B, int64_t ldb, void* stream, ft_report_t* report) {
  if (layout != FTBLAS_ROW_MAJOR && layout != FTBLAS_COL_MAJOR) return -1;
  if (side != FTBLAS_LEFT && side != FTBLAS_RIGHT) return -2;
  if (uplo != FTBLAS_UPPER && uplo != FTBLAS_LOWER) return -3;
  if (transa != FTBLAS_NO_TRANS && transa != FTBLAS_TRANS) return -4;
  if (diag != FTBLAS_NON_UNIT && diag != FTBLAS_UNIT) return -5;
  if (M < 0) return -6;
  if (N < 0) return -7;
  const bool col = layout == FTBLAS_COL_MAJOR;
  const int64_t dim = side == FTBLAS_LEFT ? M : N;
  const bool need = M > 0 && N > 0 && alpha != 0.0;
  if (need && A == nullptr) return -9;
  if (lda < (dim > 1 ? dim : 1)) return -10;
  const int64_t ld_mn = col ? M : N;
  if (M > 0 && N > 0 && B == nullptr) return -11;
  if (ldb < (ld_mn > 1 ? ld_mn : 1)) return -12;
  if (M > kMaxDim || N > kMaxDim) return FTBLAS_STATUS_NOT_SUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!need) {  // alpha = 0 gives B = 0 (B is not read), or an empty B
    const int64_t l1 = ld_mn > 1 ? ld_mn : 1;
    return dgemm_impl(layout, FTBLAS_NO_TRANS, FTBLAS_NO_TRANS, M, N, 0, 0.0, nullptr, l1, nullptr, l1, 0.0, B, ldb,
                      stream, report, true);
  }
  // op(A) is upper when A is upper and not transposed, or lower and transposed
  const bool op_upper = (uplo == FTBLAS_UPPER) == (transa == FTBLAS_NO_TRANS);
  const int tri = op_upper ? 1 : 2;
  const int64_t rows = col ? M : N, cols = col ? N : M;  // storage extent of B
  if (use_other_layout(col, side == FTBLAS_LEFT, tri))
    return dtrmm_other_layout(col, side, uplo, transa, diag, M, N, alpha, A, lda, B, ldb, st, report, tri, rows,
                              cols);
  double *T = nullptr, *B0 = nullptr;
  if (ws_alloc(reinterpret_cast<void**>(&T), (size_t)(dim * dim + rows * cols) * 8, st) != cudaSuccess)
    return FTBLAS_STATUS_ALLOC_FAILED;
  B0 = T + dim * dim;
  int rc = record_cuda(launch_expand(A, lda, !col, dim, 1, uplo == FTBLAS_UPPER, transa == FTBLAS_TRANS,
                                     diag == FTBLAS_UNIT, T, st));
  if (rc == 0) rc = record_cuda(cudaMemcpy2DAsync(B0, rows * 8, B, ldb * 8, rows * 8, cols, cudaMemcpyDeviceToDevice, st));
  if (rc == 0) {
    rc = side == FTBLAS_LEFT
             ? dgemm_impl(layout, FTBLAS_NO_TRANS, FTBLAS_NO_TRANS, M, N, M, alpha, T, dim, B0, rows, 0.0, B, ldb,
                          stream, report, true, tri, 0)
             : dgemm_impl(layout, FTBLAS_NO_TRANS, FTBLAS_NO_TRANS, M, N, N, alpha, B0, rows, T, dim, 0.0, B, ldb,
                          stream, report, true, 0, tri);
  }
  cudaFreeAsync(T, st);
  return rc;
}

// FT-DTRSM: op(A) X = alpha B (left) or X op(A) = alpha B (right), X overwriting B. The
// system is brought to the column-major left form T W = alpha W0 (T = op(A), or op(A)^T for
// the right side; W0 = B or B^T) and solved by recursive blocked substitution: split T into
// halves, solve one, update the other right-hand sides with the protected GEMM
// (W2 -= T21 X1), solve the other; diagonal blocks of kTrsmLeaf rows are solved by the
// checksum-verified leaf kernel. Every internal step writes its own report; they are merged.
struct TrsmCtx {
  const double* T;
  double* W;
  int64_t dim, nrhs;
  bool lower;
  cudaStream_t st;
  ft_report_t* parts;
  std::vector<int64_t> row_off;
  int rc;
};

void trsm_rec(TrsmCtx& c, int64_t i0, int64_t n) {
  if (c.rc != 0 || n == 0) return;
  if (n <= kTrsmLeaf) {
    const size_t p = c.row_off.size();
    c.row_off.push_back(i0);
    CallerPoint pts[kMaxInject];
    const int npts = plan_injections(n, c.nrhs, kTrsmLeaf, 32, pts);
    InjectList inj;
    std::memset(&inj, 0, sizeof(inj));
    for (int q = 0; q < npts; ++q) {
      if (pts[q].site == FT_SITE_STALL) continue;  // FP64 GEMM kernels only
      InjectPoint& ip = inj.p[inj.n++];
      ip.i = (int32_t)pts[q].i; ip.j = (int32_t)pts[q].j; ip.site = pts[q].site; ip.mode = pts[q].mode;
      ip.bit = pts[q].bit; ip.rel_log2 = pts[q].rel_log2; ip.sign = pts[q].sign; ip.kt = 0;
    }
    c.rc = record_cuda(cudaMemsetAsync(c.parts + p, 0, sizeof(ft_report_t), c.st));
    if (c.rc == 0)
      c.rc = record_cuda(launch_trsm_leaf(c.T + i0 + i0 * c.dim, c.dim, c.W + i0, c.dim, (int)n, c.nrhs, c.lower,
                                          c.parts + p, inj, c.st));
    return;
  }
  const int64_t n1 = ((n / 2 + kTrsmLeaf - 1) / kTrsmLeaf) * kTrsmLeaf, n2 = n - n1;
  auto update = [&](int64_t r_dst, int64_t m, int64_t r_src, int64_t k) {
    // W[r_dst : r_dst + m) -= T[r_dst : r_dst + m, r_src : r_src + k) W[r_src : r_src + k)
    const size_t p = c.row_off.size();
    c.row_off.push_back(r_dst);
    if (c.rc == 0)
      c.rc = dgemm_impl(FTBLAS_COL_MAJOR, FTBLAS_NO_TRANS, FTBLAS_NO_TRANS, m, c.nrhs, k, -1.0,
                        c.T + r_dst + r_src * c.dim, c.dim, c.W + r_src, c.dim, 1.0, c.W + r_dst, c.dim, c.st,
                        c.parts + p, true);
  };
  if (c.lower) {
    trsm_rec(c, i0, n1);
    update(i0 + n1, n2, i0, n1);
    trsm_rec(c, i0 + n1, n2);
  } else {
    trsm_rec(c, i0 + n1, n2);
    update(i0, n1, i0 + n1, n2);
    trsm_rec(c, i0, n1);
  }
}

int dtrsm_impl(int layout, int side, int uplo, int transa, int diag, int64_t M, int64_t N, double alpha,
               const double* A, int64_t lda, double* B, int64_t ldb, void* stream, ft_report_t* report) {
  if (layout != FTBLAS_ROW_MAJOR && layout != FTBLAS_COL_MAJOR) return -1;
  if (side != FTBLAS_LEFT && side != FTBLAS_RIGHT) return -2;
  if (uplo != FTBLAS_UPPER && uplo != FTBLAS_LOWER) return -3;
  if (transa != FTBLAS_NO_TRANS && transa != FTBLAS_TRANS) return -4;
  if (diag != FTBLAS_NON_UNIT && diag != FTBLAS_UNIT) return -5;
  if (M < 0) return -6;
  if (N < 0) return -7;
  const bool col = layout == FTBLAS_COL_MAJOR;
  const int64_t dim = side == FTBLAS_LEFT ? M : N, nrhs = side == FTBLAS_LEFT ? N : M;
  const bool need = M > 0 && N > 0 && alpha != 0.0;
  if (need && A == nullptr) return -9;
  if (lda < (dim > 1 ? dim : 1)) return -10;
  const int64_t ld_mn = col ? M : N;
  if (M > 0 && N > 0 && B == nullptr) return -11;
  if (ldb < (ld_mn > 1 ? ld_mn : 1)) return -12;
  if (M > kMaxDim || N > kMaxDim) return FTBLAS_STATUS_NOT_SUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!need) {  // alpha = 0 gives X = 0 (B is not read), or an empty B
    const int64_t l1 = ld_mn > 1 ? ld_mn : 1;
    return dgemm_impl(layout, FTBLAS_NO_TRANS, FTBLAS_NO_TRANS, M, N, 0, 0.0, nullptr, l1, nullptr, l1, 0.0, B, ldb,
                      stream, report, true);
  }
  // T = op(A) (left) or op(A)^T (right), written column-major: the expansion writes in the
  // caller's layout, and a row-major copy of X is the column-major copy of X^T.
  const bool trans_solve = (side == FTBLAS_LEFT) == (transa == FTBLAS_TRANS);
  const bool trans_expand = trans_solve != !col;
  const bool upper = (uplo == FTBLAS_UPPER) == !trans_solve;
  // B's storage read column-major is D (M x N when column-major, else N x M); W = B
  // (left) or B^T (right) is D itself or D^T.
  const bool w_is_d = (side == FTBLAS_LEFT) == col;
  const int64_t d_rows = col ? M : N, d_cols = col ? N : M;
  const int nparts = (int)(2 * ((dim + kTrsmLeaf - 1) / kTrsmLeaf) + 1);
  double* T = nullptr;
  const size_t bytes = (size_t)(dim * dim + dim * nrhs) * 8 + (size_t)nparts * (sizeof(ft_report_t) + 8) + 256;
  if (ws_alloc(reinterpret_cast<void**>(&T), bytes, st) != cudaSuccess) return FTBLAS_STATUS_ALLOC_FAILED;
  double* W = T + dim * dim;
  char* tail = reinterpret_cast<char*>(W + dim * nrhs);
  tail += (256 - reinterpret_cast<uintptr_t>(tail) % 256) % 256;
  ft_report_t* parts = reinterpret_cast<ft_report_t*>(tail);
  int64_t* row_off_dev = reinterpret_cast<int64_t*>(parts + nparts);
  int rc = record_cuda(launch_expand(A, lda, !col, dim, 1, uplo == FTBLAS_UPPER, trans_expand, diag == FTBLAS_UNIT, T,
                                     st));
  if (rc == 0)
    rc = record_cuda(launch_copy2d(B, w_is_d ? 1 : ldb, w_is_d ? ldb : 1, W, dim, dim, nrhs, alpha, st));
  TrsmCtx c{T, W, dim, nrhs, !upper, st, parts, {}, rc};
  trsm_rec(c, 0, dim);
  rc = c.rc;
  if (rc == 0)
    rc = record_cuda(launch_copy2d(W, w_is_d ? 1 : dim, w_is_d ? dim : 1, B, ldb, d_rows, d_cols, 1.0, st));
  if (rc == 0 && report != nullptr) {
    rc = record_cuda(cudaMemsetAsync(report, 0, sizeof(ft_report_t), st));
    if (rc == 0)
      rc = record_cuda(cudaMemcpyAsync(row_off_dev, c.row_off.data(), c.row_off.size() * 8, cudaMemcpyHostToDevice, st));
    if (rc == 0)
      rc = record_cuda(launch_report_merge(parts, row_off_dev, (int)c.row_off.size(), report, side == FTBLAS_RIGHT, st));
  }
  cudaFreeAsync(T, st);
  return rc;
}

// ------------------------------------------------------------------ unfused comparator
int dgemm_unfused_impl(int layout, int ta, int tb, int64_t M, int64_t N, int64_t K, double alpha, const double* A,
                       int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc, void* stream,
                       ft_report_t* report) {
  const bool need_ab = (K > 0 && alpha != 0.0 && M > 0 && N > 0);
  int v = validate(layout, ta, tb, M, N, K, A, lda, B, ldb, C, ldc, need_ab);
  if (v != 0) return v;
  if (M > kMaxDim || N > kMaxDim || K > kMaxDim) return FTBLAS_STATUS_NOT_SUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (report != nullptr) {
    if (int e = record_cuda(cudaMemsetAsync(report, 0, sizeof(ft_report_t), st))) return e;
  }
  if (M == 0 || N == 0) return 0;
  const Frame f = map_frame(layout, ta, tb, M, N, A, lda, B, ldb);
  CallerPoint pts[kMaxInject];
  const int64_t tile_rows = f.swap ? kDBN : kDBM, tile_cols = f.swap ? kDBM : kDBN;
  const int npts = plan_injections(M, N, tile_rows, tile_cols, pts);
  if (K == 0 || alpha == 0.0) return record_cuda(launch_scale(C, ldc, (int32_t)f.M, (int32_t)f.N, beta, st));
  UnfusedParams p;
  std::memset(&p, 0, sizeof(p));
  p.M = (int32_t)f.M; p.N = (int32_t)f.N; p.K = (int32_t)K;
  p.a_kmajor = f.a_kmajor; p.b_kmajor = f.b_kmajor;
  p.swap_report = f.swap;
  p.alpha = alpha; p.beta = beta;
  p.A = static_cast<const double*>(f.A); p.lda = f.lda;
  p.B = static_cast<const double*>(f.B); p.ldb = f.ldb;
  p.C = C; p.ldc = ldc;
  p.report = report;
  for (int q = 0; q < npts; ++q) {
    const CallerPoint& c = pts[q];
    if (c.site == FT_SITE_STALL) continue;  // FP64 GEMM kernels only
    InjectPoint& ip = p.inj.p[p.inj.n++];
    ip.i = (int32_t)(f.swap ? c.j : c.i);
    ip.j = (int32_t)(f.swap ? c.i : c.j);
    ip.site = c.site == FT_SITE_CHECKSUM ? kSiteChecksumRow : c.site;
    ip.mode = c.mode; ip.bit = c.bit; ip.rel_log2 = c.rel_log2; ip.sign = c.sign; ip.kt = c.kt;
  }
  cudaError_t ce = cudaSuccess;
  const int rc = unfused_dgemm(p, st, &ce);
  if (ce != cudaSuccess) return record_cuda(ce);
  return rc;
}

// ------------------------------------------------------------------ mixed precision
// The tensor-core path (A, B BF16 or FP8 E4M3; C and compute FP32) behind ftblas_gemm_ex,
// ftblas_gemm_ex_noabft and ftblas_gemm_ex_noalloc. Workspace: from the stream-ordered
// allocator when ws is null, else the caller's ws_bytes bytes (checked before any device
// work). Argument checks follow ftblas_gemm_ex's positions.
int tc_gemm_impl(int layout, int ta, int tb, int64_t M, int64_t N, int64_t K, const void* alpha, const void* A,
                 int Atype, int64_t lda, const void* B, int Btype, int64_t ldb, const void* beta, void* C, int Ctype,
                 int64_t ldc, int ctype, const float* a_scale, const float* b_scale, void* stream, ft_report_t* report,
                 bool ft, ScratchResolver resolve, size_t ws_bytes, bool allow_fp8) {
  if (layout != FTBLAS_ROW_MAJOR && layout != FTBLAS_COL_MAJOR) return -1;
  if (ta != FTBLAS_NO_TRANS && ta != FTBLAS_TRANS) return -2;
  if (tb != FTBLAS_NO_TRANS && tb != FTBLAS_TRANS) return -3;
  if (M < 0) return -4;
  if (N < 0) return -5;
  if (K < 0) return -6;
  if (alpha == nullptr) return -7;
  if (beta == nullptr) return -14;
  // C in FP32, or in bfloat16: the product is verified, located and corrected in FP32 and
  // rounded to bfloat16 once (by the CTA-pair kernel's epilogue and the resolve pass, or, for
  // the one-CTA kernel, by a pass over an FP32 buffer at the end)
  const bool c_bf16 = Ctype == FTBLAS_R_16BF && resolve == nullptr;
  const bool c32 = (Ctype == FTBLAS_R_32F || c_bf16) && ctype == FTBLAS_R_32F;
  const bool bf16 = c32 && Atype == FTBLAS_R_16BF && Btype == FTBLAS_R_16BF;
  const bool fp8 = c32 && allow_fp8 && Atype == FTBLAS_R_8F_E4M3 && Btype == FTBLAS_R_8F_E4M3;
  if (!bf16 && !fp8) return FTBLAS_STATUS_NOT_SUPPORTED;
  if (bf16 && a_scale != nullptr) return -19;
  if (bf16 && b_scale != nullptr) return -20;
  const int kind = fp8 ? 1 : 0;
  const float al = *static_cast<const float*>(alpha), be = *static_cast<const float*>(beta);
  const bool need_ab = (K > 0 && al != 0.0f && M > 0 && N > 0);
  int v = validate(layout, ta, tb, M, N, K, A, lda, B, ldb, C, ldc, need_ab);
  if (v != 0) {
    static const int pos[15] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 10, 11, 13, 14, 15, 17};
    return -pos[-v];
  }
  if (M > kMaxDim || N > kMaxDim || K > kMaxDim) return FTBLAS_STATUS_NOT_SUPPORTED;
  Frame f = map_frame(layout, ta, tb, M, N, A, lda, B, ldb);
  const int eb = (Atype == FTBLAS_R_8F_E4M3) ? 1 : 2;
  // K-major operands the tensor maps cannot address (base or pitch not 16-byte aligned) are
  // copied too, into aligned rows
  auto aligned = [&](const void* x, int64_t ld) {
    return (reinterpret_cast<uintptr_t>(x) & 15u) == 0 && ((ld * eb) & 15) == 0;
  };
  const bool copy_a = need_ab && (!f.a_kmajor || !aligned(f.A, f.lda));
  const bool copy_b = need_ab && (!f.b_kmajor || !aligned(f.B, f.ldb));
  // such operands are copied into workspace below; the entry point without allocation has
  // no room for copies
  if (resolve != nullptr && (copy_a || copy_b)) return FTBLAS_STATUS_NOT_SUPPORTED;
  const size_t wsb = (ft && need_ab) ? tc_workspace_bytes((int32_t)f.M, (int32_t)f.N, (int32_t)K, kind) : 0;
  if (resolve != nullptr && wsb > ws_bytes) return FTBLAS_STATUS_WORKSPACE_LIMIT;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (ft && report != nullptr) {
    if (int e = record_cuda(cudaMemsetAsync(report, 0, sizeof(ft_report_t), st))) return e;
  }
  if (M == 0 || N == 0) return 0;
  if (!need_ab) {  // C = beta C
    if (c_bf16) return record_cuda(launch_scale_bf16(static_cast<uint16_t*>(C), ldc, f.M, f.N, be, st));
    return record_cuda(launch_scale_f32(static_cast<float*>(C), ldc, f.M, f.N, be, st));
  }
  CallerPoint pts[kMaxInject];
  int npts = 0;
  const int64_t bnp = tc_bn_prot(kind), chk_rows = tc_chk_rows(kind);  // protected tile width, checksum rows
  if (ft) {
    const int64_t tile_rows = f.swap ? bnp : kTcBM, tile_cols = f.swap ? kTcBM : bnp;
    npts = plan_injections(M, N, tile_rows, tile_cols, pts);
  }
  TcParams p;
  std::memset(&p, 0, sizeof(p));
  p.M = (int32_t)f.M; p.N = (int32_t)f.N; p.K = (int32_t)K;
  // accumulation unit: kind::f16 truncates to binary32 (2^-23); kind::f8f6f4 also aligns each
  // group of 32 products to its largest term and truncates every product, taken as 2^-22
  p.alpha = al; p.beta = be; p.u_acc = fp8 ? 0x1p-22f : 0x1p-23f;
  p.kind = kind;
  p.a_scale = fp8 ? (f.swap ? b_scale : a_scale) : nullptr;
  p.b_scale = fp8 ? (f.swap ? a_scale : b_scale) : nullptr;
  // one CTA per 128-row tile, or a CTA pair per 256 rows (B staged half in each CTA); by
  // default the pairs, the faster form measured for protected and unprotected calls alike
  const int cg_set = g_tc_cta_group.load();
  const int cg = cg_set != 0 ? cg_set : 2;
  // a bfloat16 C written by the pair kernel itself (the one-CTA kernel writes FP32 only)
  const bool cb_direct = c_bf16 && cg == 2;
  // K-major, aligned copies of MN-major or misaligned operands (stream-ordered workspace,
  // released at the end)
  void* tws = nullptr;
  // FP32 product buffer of a bfloat16 C (kernel frame, column-major, leading dimension M):
  // the verified copy the resolve pass reads and corrects; none for an unprotected call
  // that writes the bfloat16 C directly
  const bool need_cf = c_bf16 && (ft || !cb_direct);
  const size_t cbytes = need_cf ? (size_t(f.M) * size_t(f.N) * 4 + 255) & ~size_t(255) : 0;
  float* cf = nullptr;
  if (copy_a || copy_b || need_cf) {
    const int64_t pitch = tc_kmajor_pitch(K, eb);
    const size_t abytes = copy_a ? (size_t(f.M * pitch * eb) + 255) & ~size_t(255) : 0;
    const size_t bbytes = copy_b ? (size_t(f.N * pitch * eb) + 255) & ~size_t(255) : 0;
    if (ws_alloc(&tws, abytes + bbytes + cbytes, st) != cudaSuccess) return FTBLAS_STATUS_ALLOC_FAILED;
    if (need_cf) cf = reinterpret_cast<float*>(static_cast<uint8_t*>(tws) + abytes + bbytes);
    uint8_t* base = static_cast<uint8_t*>(tws);
    auto copy = [&](const void* src, int64_t rows, int64_t ld, bool kmajor, uint8_t* dst) {
      if (kmajor)  // rows of K already contiguous: a pitched copy
        return cudaMemcpy2DAsync(dst, size_t(pitch * eb), src, size_t(ld * eb), size_t(K * eb), size_t(rows),
                                 cudaMemcpyDeviceToDevice, st);
      return launch_kmajor_copy(src, rows, K, ld, eb, dst, pitch, st);
    };
    cudaError_t ce = cudaSuccess;
    if (copy_a) {
      ce = copy(f.A, f.M, f.lda, f.a_kmajor, base);
      f.A = base; f.lda = pitch; f.a_kmajor = true;
    }
    if (ce == cudaSuccess && copy_b) {
      ce = copy(f.B, f.N, f.ldb, f.b_kmajor, base + abytes);
      f.B = base + abytes; f.ldb = pitch; f.b_kmajor = true;
    }
    if (ce != cudaSuccess) {
      cudaFreeAsync(tws, st);
      return record_cuda(ce);
    }
  }
  auto release = [&](int rc) {
    if (tws != nullptr) cudaFreeAsync(tws, st);
    return rc;
  };
  p.A = f.A; p.lda = f.lda; p.B = f.B; p.ldb = f.ldb;
  if (cb_direct) {
    // the kernel reads C_in from the bfloat16 C and writes it there (and the FP32 copy into
    // cf when protected)
    p.C = cf; p.ldc = f.M;
    p.Cb = static_cast<uint16_t*>(C); p.ldcb = ldc;
  } else if (c_bf16) {
    p.C = cf; p.ldc = f.M;
    if (be != 0.0f) {
      if (int e = record_cuda(launch_bf16_to_f32(static_cast<const uint16_t*>(C), ldc, cf, f.M, f.M, f.N, st)))
        return release(e);
    }
  } else {
    p.C = static_cast<float*>(C); p.ldc = ldc;
  }
  // the bfloat16 C rounded from the FP32 buffer once every pass over it has finished
  auto finish = [&](int rc) {
    if (rc == 0 && c_bf16 && !cb_direct)
      rc = record_cuda(launch_f32_to_bf16(cf, f.M, static_cast<uint16_t*>(C), ldc, f.M, f.N, st));
    return release(rc);
  };
  p.report = ft ? report : nullptr;
  p.swap_report = f.swap;
  bool stall = false;
  for (int q = 0; q < npts; ++q) {
    const CallerPoint& c = pts[q];
    InjectPoint& ip = p.inj.p[p.inj.n++];
    ip.i = (int32_t)(f.swap ? c.j : c.i);
    ip.j = (int32_t)(f.swap ? c.i : c.j);
    ip.site = c.site == FT_SITE_CHECKSUM ? kSiteChecksumRow : c.site == FT_SITE_STALL ? kSiteStall : c.site;
    ip.mode = c.mode; ip.bit = c.bit; ip.rel_log2 = c.rel_log2; ip.sign = c.sign; ip.kt = c.kt;
    stall |= c.site == FT_SITE_STALL;
  }
  // 2 s per bounded wait (a whole tile takes about 0.1 ms); 20 ms with a stall point planned
  p.wait_limit_ns = stall ? 20000000ull : 2000000000ull;
  TcMaps maps;
  std::memset(&maps, 0, sizeof(maps));
  const uint32_t b_rows = cg == 2 ? kTcBN / 2 : (ft ? (uint32_t)bnp : kTcBN);
  if (!make_map_sw128(&maps.a, eb, f.A, K, f.M, f.lda, kTcBM)) return release(FTBLAS_STATUS_NOT_SUPPORTED);
  if (!make_map_sw128(&maps.b, eb, f.B, K, f.N, f.ldb, b_rows)) return release(FTBLAS_STATUS_NOT_SUPPORTED);
  maps.b2 = maps.b;
  if (cg == 2 && ft && !make_map_sw128(&maps.b2, eb, f.B, K, f.N, f.ldb, (uint32_t)(bnp - kTcBN / 2)))
    return release(FTBLAS_STATUS_NOT_SUPPORTED);
  maps.chk = maps.a;
  g_last_used_tma = 1;
  if (!ft) return finish(record_cuda(launch_tc_gemm(p, maps, false, cg, st)));
  const bool own = resolve == nullptr;
  void* ws = nullptr;
  if (own) {
    if (ws_alloc(&ws, wsb, st) != cudaSuccess) return release(FTBLAS_STATUS_ALLOC_FAILED);
  } else {
    cudaError_t ce = cudaSuccess;
    ws = resolve(&ce);
    if (ws == nullptr) return release(record_cuda(ce != cudaSuccess ? ce : cudaErrorInvalidDevicePointer));
  }
  TcWorkspace w = tc_workspace_carve(ws, p.M, p.N, p.K, kind);
  p.rowAbsA = w.rowAbsA; p.maxAbsBe = w.maxAbsBe; p.sA = w.sA; p.absSA = w.absSA;
  p.sa_pitch = w.kpitch; p.pend = w.pend;
  const int64_t nNb = (f.N + bnp - 1) / bnp;
  int rc = make_map_sw128(&maps.chk, eb, w.chk, K, nNb * chk_rows, w.kpitch, (uint32_t)chk_rows) ? 0
                                                                                              : FTBLAS_STATUS_NOT_SUPPORTED;
  if (rc == 0) rc = record_cuda(launch_tc_encode(p, w, st));  // writes every workspace entry the GEMM reads
  if (rc == 0) rc = record_cuda(launch_tc_gemm(p, maps, true, cg, st));
  if (own) cudaFreeAsync(ws, st);
  return finish(rc);
}

// ------------------------------------------------------------------ emulated FP64
// The binary64 GEMM formed from E4M3 integer slices on the tensor cores (ft_emu.cu).
// Workspace from the stream-ordered allocator, released on the same stream.
int emu_impl(int layout, int ta, int tb, int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t lda,
             const double* B, int64_t ldb, double beta, double* C, int64_t ldc, void* stream, ft_report_t* report,
             bool ft) {
  const bool need_ab = (K > 0 && alpha != 0.0 && M > 0 && N > 0);
  int v = validate(layout, ta, tb, M, N, K, A, lda, B, ldb, C, ldc, need_ab);
  if (v != 0) return v;
  const int s = g_emu_slices.load();
  if (K > emu_max_k(s) || M > (int64_t(1) << 26) || N > (int64_t(1) << 26)) return FTBLAS_STATUS_NOT_SUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (ft && report != nullptr) {
    if (int e = record_cuda(cudaMemsetAsync(report, 0, sizeof(ft_report_t), st))) return e;
  }
  if (M == 0 || N == 0) return 0;
  const Frame f = map_frame(layout, ta, tb, M, N, A, lda, B, ldb);
  const int bn = ft ? kEmuBNProt : kEmuBNPlain;
  CallerPoint pts[kMaxInject];
  int npts = 0;
  if (ft) {
    const int64_t tile_rows = f.swap ? bn : kEmuBM, tile_cols = f.swap ? kEmuBM : bn;
    npts = plan_injections(M, N, tile_rows, tile_cols, pts);
  }
  if (K == 0 || alpha == 0.0) return record_cuda(launch_scale(C, ldc, (int32_t)f.M, (int32_t)f.N, beta, st));
  EmuParams p;
  std::memset(&p, 0, sizeof(p));
  p.M = (int32_t)f.M; p.N = (int32_t)f.N; p.K = (int32_t)K;
  p.s = s;
  p.bn = bn;
  p.nMb = (int32_t)((f.M + kEmuBM - 1) / kEmuBM);
  p.nNb = (int32_t)((f.N + bn - 1) / bn);
  p.m_pad = (int64_t)p.nMb * kEmuBM;
  p.n_pad = (int64_t)p.nNb * bn;
  p.kpitch = (K + 15) / 16 * 16;
  p.swap_report = f.swap;
  p.alpha = alpha; p.beta = beta;
  p.C = C; p.ldc = ldc;
  p.report = ft ? report : nullptr;
  bool stall = false;
  for (int q = 0; q < npts; ++q) {
    const CallerPoint& c = pts[q];
    InjectPoint& ip = p.inj.p[p.inj.n++];
    ip.i = (int32_t)(f.swap ? c.j : c.i);
    ip.j = (int32_t)(f.swap ? c.i : c.j);
    ip.site = c.site == FT_SITE_CHECKSUM ? kSiteChecksumRow : c.site == FT_SITE_STALL ? kSiteStall : c.site;
    ip.mode = c.mode; ip.bit = c.bit; ip.rel_log2 = c.rel_log2; ip.sign = c.sign; ip.kt = c.kt;
    stall |= c.site == FT_SITE_STALL;
  }
  p.wait_limit_ns = stall ? 20000000ull : 2000000000ull;
  // sources of the split: line i of op(A) and line j of op(B)^T in the kernel frame
  const EmuSource sa{static_cast<const double*>(f.A), f.a_kmajor ? f.lda : 1, f.a_kmajor ? 1 : f.lda, f.M};
  const EmuSource sb{static_cast<const double*>(f.B), f.b_kmajor ? f.ldb : 1, f.b_kmajor ? 1 : f.ldb, f.N};
  const int64_t tiles = (int64_t)p.nMb * p.nNb;
  const int sms = current_sm_count();
  const int grid = (int)(tiles < sms ? tiles : sms);
  void* ws = nullptr;
  if (ws_alloc(&ws, emu_workspace_bytes(p, grid), st) != cudaSuccess) return FTBLAS_STATUS_ALLOC_FAILED;
  uint8_t* chk = nullptr;
  emu_workspace_carve(p, ws, grid, &chk);
  CUtensorMap tmA, tmB, tmC;
  std::memset(&tmA, 0, sizeof(tmA)); std::memset(&tmB, 0, sizeof(tmB)); std::memset(&tmC, 0, sizeof(tmC));
  int rc = 0;
  if (!make_map_sw128(&tmA, 1, p.aslices, K, (int64_t)s * p.m_pad, p.kpitch, kEmuBM) ||
      !make_map_sw128(&tmB, 1, p.bslices, K, (int64_t)s * p.n_pad, p.kpitch, (uint32_t)bn) ||
      (ft && !make_map_sw128(&tmC, 1, chk, K, (int64_t)s * p.nNb * kEmuChkRows, p.kpitch, kEmuChkRows)))
    rc = FTBLAS_STATUS_NOT_SUPPORTED;
  if (rc == 0) rc = record_cuda(launch_emu_split(p, sa, sb, chk, ft, st));
  if (rc == 0) rc = record_cuda(launch_emu_gemm(p, &tmA, &tmB, &tmC, ft, grid, st));
  g_last_used_tma = 1;
  cudaFreeAsync(ws, st);
  return rc;
}

int gemm_ex_impl(int layout, int ta, int tb, int64_t M, int64_t N, int64_t K, const void* alpha, const void* A,
                 int Atype, int64_t lda, const void* B, int Btype, int64_t ldb, const void* beta, void* C, int Ctype,
                 int64_t ldc, int ctype, const float* a_scale, const float* b_scale, void* stream,
                 ft_report_t* report, bool ft) {
  // argument positions of ftblas_gemm_ex (1-based)
  if (layout != FTBLAS_ROW_MAJOR && layout != FTBLAS_COL_MAJOR) return -1;
  if (ta != FTBLAS_NO_TRANS && ta != FTBLAS_TRANS) return -2;
  if (tb != FTBLAS_NO_TRANS && tb != FTBLAS_TRANS) return -3;
  if (M < 0) return -4;
  if (N < 0) return -5;
  if (K < 0) return -6;
  if (alpha == nullptr) return -7;
  if (beta == nullptr) return -14;
  const bool all64 = Atype == FTBLAS_R_64F && Btype == FTBLAS_R_64F && Ctype == FTBLAS_R_64F && ctype == FTBLAS_R_64F;
  if (all64) {
    if (a_scale != nullptr) return -19;
    if (b_scale != nullptr) return -20;
    const double al = *static_cast<const double*>(alpha), be = *static_cast<const double*>(beta);
    int v = dgemm_impl(layout, ta, tb, M, N, K, al, static_cast<const double*>(A), lda,
                       static_cast<const double*>(B), ldb, be, static_cast<double*>(C), ldc, stream, report, ft);
    // map dgemm argument positions onto gemm_ex positions
    static const int pos[17] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 10, 11, 13, 14, 15, 17, 21, 22};
    return (v < 0 && -v <= 16) ? -pos[-v] : v;
  }
  return tc_gemm_impl(layout, ta, tb, M, N, K, alpha, A, Atype, lda, B, Btype, ldb, beta, C, Ctype, ldc, ctype, a_scale,
                      b_scale, stream, report, ft, nullptr, 0, true);
}

// ------------------------------------------------------------------ host-buffer workspace
// Copy `cnt` runs of `run` doubles from pitch `spitch` to pitch `dpitch` (elements): one
// linear copy when the pitches agree (the 2-D engine path is far slower) and, for copies
// into the caller's buffer, there is no padding to preserve between runs; else 2-D.
cudaError_t copy_runs(double* dst, int64_t dpitch, const double* src, int64_t spitch, int64_t run, int64_t cnt,
                      cudaMemcpyKind kind, cudaStream_t st) {
  if (run == 0 || cnt == 0) return cudaSuccess;
  const bool linear = dpitch == spitch && (kind == cudaMemcpyHostToDevice || run == dpitch);
  if (linear) return cudaMemcpyAsync(dst, src, size_t((cnt - 1) * spitch + run) * 8, kind, st);
  return cudaMemcpy2DAsync(dst, dpitch * 8, src, spitch * 8, run * 8, cnt, kind, st);
}

// product-kernel timing (ftblas_kernel_timing_begin / _end)
std::mutex g_timer_mu;
bool g_timer_on = false;
bool g_timer_failed = false;
std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_timer_pairs;
thread_local cudaEvent_t g_timer_open = nullptr;

void release_timer_pairs() {
  for (auto& pr : g_timer_pairs) {
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  g_timer_pairs.clear();
}

std::mutex g_ws_mu;
void* g_ws = nullptr;
size_t g_ws_bytes = 0;
int g_ws_device = -1;

}  // namespace

namespace ftk {

cudaError_t ws_alloc(void** ptr, size_t bytes, cudaStream_t st) {
  constexpr int kMaxPoolDevices = 64;
  static std::mutex mu;
  static cudaMemPool_t pools[kMaxPoolDevices] = {};
  static bool tried[kMaxPoolDevices] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxPoolDevices) {
    (void)cudaGetLastError();
    return cudaMallocAsync(ptr, bytes, st);
  }
  cudaMemPool_t pool = nullptr;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!tried[dev]) {
      tried[dev] = true;
      cudaMemPoolProps props;
      std::memset(&props, 0, sizeof(props));
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      if (cudaMemPoolCreate(&pools[dev], &props) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        (void)cudaMemPoolSetAttribute(pools[dev], cudaMemPoolAttrReleaseThreshold, &keep);
      } else {
        pools[dev] = nullptr;
        (void)cudaGetLastError();
      }
    }
    pool = pools[dev];
  }
  if (pool == nullptr) return cudaMallocAsync(ptr, bytes, st);
  return cudaMallocFromPoolAsync(ptr, bytes, pool, st);
}

void kernel_timer_start(cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_timer_mu);
  if (!g_timer_on) return;
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess || cudaEventRecord(e, st) != cudaSuccess) {
    if (e) cudaEventDestroy(e);
    g_timer_failed = true;
    return;
  }
  g_timer_open = e;
}

void kernel_timer_stop(cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_timer_mu);
  if (!g_timer_on || g_timer_open == nullptr) return;
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess || cudaEventRecord(e, st) != cudaSuccess) {
    if (e) cudaEventDestroy(e);
    cudaEventDestroy(g_timer_open);
    g_timer_open = nullptr;
    g_timer_failed = true;
    return;
  }
  g_timer_pairs.emplace_back(g_timer_open, e);
  g_timer_open = nullptr;
}

// The protected BF16 GEMM of ftblas_gemm_ex with the encode workspace in a fixed scratch
// area (no allocation of any kind).
int gemm_bf16_ft_with_scratch(int layout, int ta, int tb, int64_t M, int64_t N, int64_t K, const void* alpha,
                              const void* A, int Atype, int64_t lda, const void* B, int Btype, int64_t ldb,
                              const void* beta, void* C, int Ctype, int64_t ldc, int ctype, const float* a_scale,
                              const float* b_scale, void* stream, ft_report_t* report, ScratchResolver resolve,
                              size_t scratch_bytes) {
  if (resolve == nullptr) return FTBLAS_STATUS_WORKSPACE_LIMIT;
  return tc_gemm_impl(layout, ta, tb, M, N, K, alpha, A, Atype, lda, B, Btype, ldb, beta, C, Ctype, ldc, ctype, a_scale,
                      b_scale, stream, report, true, resolve, scratch_bytes, false);
}

}  // namespace ftk

extern "C" {

int ftblas_set_injection(const ft_inject_t* cfg) {
  std::lock_guard<std::mutex> lk(g_inj_mu);
  g_launch = 0;
  if (cfg == nullptr) {
    g_inj_on = false;
    return 0;
  }
  if (cfg->n_fixed < 0 || cfg->n_fixed > FTBLAS_MAX_FIXED_INJECTIONS) return -1;
  if (cfg->n_fixed == 0) {
    if (cfg->every_n_launches < 0 || cfg->errors_per_launch < 0 ||
        cfg->errors_per_launch > FTBLAS_MAX_INJECTIONS_PER_LAUNCH)
      return -1;
    if (cfg->bit_lo < 0 || cfg->bit_hi > 63 || cfg->bit_lo > cfg->bit_hi) return -1;
    if (cfg->log2_lo > cfg->log2_hi) return -1;
    if (cfg->site < FT_SITE_ACCUM || cfg->site > FT_SITE_CHECKSUM) return -1;
    if (cfg->mode != FT_MODE_BITFLIP && cfg->mode != FT_MODE_ADD_REL) return -1;
  }
  for (int q = 0; q < cfg->n_fixed; ++q) {
    const ft_inject_point_t& f = cfg->fixed[q];
    if (f.site < FT_SITE_ACCUM || f.site > FT_SITE_STALL) return -1;
    if (f.mode != FT_MODE_BITFLIP && f.mode != FT_MODE_ADD_REL) return -1;
    if (f.mode == FT_MODE_BITFLIP && (f.bit < 0 || f.bit > 63)) return -1;
  }
  g_inj = *cfg;
  g_inj_on = true;
  return 0;
}

uint64_t ftblas_injection_launch_count(void) {
  std::lock_guard<std::mutex> lk(g_inj_mu);
  return g_launch;
}

int ftblas_dgemm(ftblas_layout_t layout, ftblas_trans_t transa, ftblas_trans_t transb, int64_t M, int64_t N,
                 int64_t K, double alpha, const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                 double* C, int64_t ldc, void* stream, ft_report_t* report) {
  return dgemm_impl(layout, transa, transb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, stream, report, true);
}

int ftblas_dgemm_noabft(ftblas_layout_t layout, ftblas_trans_t transa, ftblas_trans_t transb, int64_t M, int64_t N,
                        int64_t K, double alpha, const double* A, int64_t lda, const double* B, int64_t ldb,
                        double beta, double* C, int64_t ldc, void* stream) {
  return dgemm_impl(layout, transa, transb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, stream, nullptr, false);
}

int ftblas_dgemm_host(ftblas_layout_t layout, ftblas_trans_t transa, ftblas_trans_t transb, int64_t M, int64_t N,
                      int64_t K, double alpha, const double* A, int64_t lda, const double* B, int64_t ldb,
                      double beta, double* C, int64_t ldc, void* stream, ft_report_t* report) {
  const bool need_ab = (K > 0 && alpha != 0.0 && M > 0 && N > 0);
  int v = validate(layout, transa, transb, M, N, K, A, lda, B, ldb, C, ldc, need_ab);
  if (v != 0) return v;
  const bool col = layout == FTBLAS_COL_MAJOR;
  // Stored extents (contiguous run length x number of runs) of A, B, C.
  const int64_t a_rows = (transa == FTBLAS_NO_TRANS) ? M : K, a_cols = (transa == FTBLAS_NO_TRANS) ? K : M;
  const int64_t b_rows = (transb == FTBLAS_NO_TRANS) ? K : N, b_cols = (transb == FTBLAS_NO_TRANS) ? N : K;
  const int64_t a_run = col ? a_rows : a_cols, a_cnt = col ? a_cols : a_rows;
  const int64_t b_run = col ? b_rows : b_cols, b_cnt = col ? b_cols : b_rows;
  const int64_t c_run = col ? M : N, c_cnt = col ? N : M;
  auto even = [](int64_t x) { return x < 2 ? int64_t(2) : (x + 1) & ~int64_t(1); };
  const int64_t dlda = even(a_run), dldb = even(b_run), dldc = even(c_run);
  const size_t bytesA = need_ab ? size_t(dlda) * a_cnt * 8 : 0, bytesB = need_ab ? size_t(dldb) * b_cnt * 8 : 0;
  const size_t bytesC = size_t(dldc) * c_cnt * 8;
  auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t total = up(bytesA) + up(bytesB) + up(bytesC) + up(sizeof(ft_report_t));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lk(g_ws_mu);
  int dev = 0;
  if (int e = record_cuda(cudaGetDevice(&dev))) return e;
  if (g_ws == nullptr || g_ws_bytes < total || g_ws_device != dev) {
    if (g_ws) {
      cudaStreamSynchronize(st);
      int cur = dev;
      if (g_ws_device >= 0 && g_ws_device != dev) cudaSetDevice(g_ws_device);
      cudaFree(g_ws);
      if (cur != g_ws_device) cudaSetDevice(cur);
      g_ws = nullptr;
    }
    if (cudaMalloc(&g_ws, total) != cudaSuccess) {
      g_ws = nullptr; g_ws_bytes = 0;
      return FTBLAS_STATUS_ALLOC_FAILED;
    }
    g_ws_bytes = total;
    g_ws_device = dev;
  }
  char* base = static_cast<char*>(g_ws);
  double* dA = reinterpret_cast<double*>(base);
  double* dB = reinterpret_cast<double*>(base + up(bytesA));
  double* dC = reinterpret_cast<double*>(base + up(bytesA) + up(bytesB));
  ft_report_t* dR = reinterpret_cast<ft_report_t*>(base + up(bytesA) + up(bytesB) + up(bytesC));
  // Every return below waits for the stream first, failures included: copies already
  // enqueued read or write the caller's host buffers, which are the caller's again on return.
  auto done = [&](int rc) {
    const cudaError_t e = cudaStreamSynchronize(st);
    return rc != 0 ? rc : record_cuda(e);
  };
  if (need_ab) {
    if (int e = record_cuda(copy_runs(dA, dlda, A, lda, a_run, a_cnt, cudaMemcpyHostToDevice, st))) return done(e);
    if (int e = record_cuda(copy_runs(dB, dldb, B, ldb, b_run, b_cnt, cudaMemcpyHostToDevice, st))) return done(e);
  }
  if (beta != 0.0 && M > 0 && N > 0) {
    if (int e = record_cuda(copy_runs(dC, dldc, C, ldc, c_run, c_cnt, cudaMemcpyHostToDevice, st))) return done(e);
  }
  int rc = dgemm_impl(layout, transa, transb, M, N, K, alpha, dA, dlda, dB, dldb, beta, dC, dldc, stream,
                      report ? dR : nullptr, true);
  if (rc != 0) return done(rc);
  if (M > 0 && N > 0) {
    if (int e = record_cuda(copy_runs(C, ldc, dC, dldc, c_run, c_cnt, cudaMemcpyDeviceToHost, st))) return done(e);
  }
  if (report) {
    if (int e = record_cuda(cudaMemcpyAsync(report, dR, sizeof(ft_report_t), cudaMemcpyDeviceToHost, st)))
      return done(e);
  }
  return done(0);
}

int ftblas_gemm_ex(ftblas_layout_t layout, ftblas_trans_t transa, ftblas_trans_t transb, int64_t M, int64_t N, int64_t K,
                   const void* alpha, const void* A, ftblas_dtype_t Atype, int64_t lda, const void* B,
                   ftblas_dtype_t Btype, int64_t ldb, const void* beta, void* C, ftblas_dtype_t Ctype, int64_t ldc,
                   ftblas_dtype_t compute_type, const float* a_scale, const float* b_scale, void* stream,
                   ft_report_t* report) {
  return gemm_ex_impl(layout, transa, transb, M, N, K, alpha, A, Atype, lda, B, Btype, ldb, beta, C, Ctype, ldc,
                      compute_type, a_scale, b_scale, stream, report, true);
}

int ftblas_gemm_ex_noabft(ftblas_layout_t layout, ftblas_trans_t transa, ftblas_trans_t transb, int64_t M, int64_t N,
                          int64_t K, const void* alpha, const void* A, ftblas_dtype_t Atype, int64_t lda,
                          const void* B, ftblas_dtype_t Btype, int64_t ldb, const void* beta, void* C,
                          ftblas_dtype_t Ctype, int64_t ldc, ftblas_dtype_t compute_type, const float* a_scale,
                          const float* b_scale, void* stream) {
  return gemm_ex_impl(layout, transa, transb, M, N, K, alpha, A, Atype, lda, B, Btype, ldb, beta, C, Ctype, ldc,
                      compute_type, a_scale, b_scale, stream, nullptr, false);
}

int ftblas_verification_tile(ftblas_layout_t layout, ftblas_dtype_t compute_type, int64_t M, int64_t N, int64_t K,
                             int64_t* tile_rows, int64_t* tile_cols, int64_t* k_tile) {
  if (layout != FTBLAS_ROW_MAJOR && layout != FTBLAS_COL_MAJOR) return -1;
  if (compute_type != FTBLAS_R_64F && compute_type != FTBLAS_R_32F && compute_type != FTBLAS_R_16BF &&
      compute_type != FTBLAS_R_8F_E4M3)
    return -2;
  if (M < 0) return -3;
  if (N < 0) return -4;
  if (K < 0) return -5;
  if (!tile_rows) return -6;
  if (!tile_cols) return -7;
  if (!k_tile) return -8;
  const bool swap = layout == FTBLAS_ROW_MAJOR;
  const int tc_kind = compute_type == FTBLAS_R_8F_E4M3 ? 1 : 0;  // R_32F and R_16BF: the BF16 form
  int64_t bm = kTcBM, bn = tc_bn_prot(tc_kind), kt = tc_kind == 1 ? 128 : 64;  // k-tile: 128 bytes
  if (compute_type == FTBLAS_R_64F) {
    // square tiles: the kernel frame's transpose of a row-major call does not change them
    bm = bn = chosen_fp64_edge(M, N, g_fp64_engine.load());
    kt = kDBK;
  }
  *tile_rows = swap ? bn : bm;
  *tile_cols = swap ? bm : bn;
  *k_tile = kt;
  return 0;
}

int ftblas_dgemm_emulated(ftblas_layout_t layout, ftblas_trans_t transa, ftblas_trans_t transb, int64_t M, int64_t N,
                          int64_t K, double alpha, const double* A, int64_t lda, const double* B, int64_t ldb,
                          double beta, double* C, int64_t ldc, void* stream, ft_report_t* report) {
  return emu_impl(layout, transa, transb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, stream, report, true);
}

int ftblas_dgemm_emulated_noabft(ftblas_layout_t layout, ftblas_trans_t transa, ftblas_trans_t transb, int64_t M,
                                 int64_t N, int64_t K, double alpha, const double* A, int64_t lda, const double* B,
                                 int64_t ldb, double beta, double* C, int64_t ldc, void* stream) {
  return emu_impl(layout, transa, transb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, stream, nullptr, false);
}

int ftblas_set_emulation_slices(int slices) {
  if (slices < 2 || slices > kEmuSlicesMax) return -1;
  return g_emu_slices.exchange(slices);
}

int64_t ftblas_emulation_max_k(int slices) {
  if (slices < 2 || slices > kEmuSlicesMax) return -1;
  return emu_max_k(slices);
}

int ftblas_emu_convert_i128(const int64_t* words, double* out, int64_t n, void* stream) {
  if (n < 0) return -3;
  if (n > 0 && words == nullptr) return -1;
  if (n > 0 && out == nullptr) return -2;
  return record_cuda(launch_emu_convert(words, out, n, static_cast<cudaStream_t>(stream)));
}

int64_t ftblas_set_verification_interval(int64_t k_interval) {
  if (k_interval < 0) return -1;
  return g_kc_interval.exchange(k_interval);
}

int ftblas_set_tc_cta_group(int cta_group) {
  if (cta_group < 0 || cta_group > 2) return -1;
  return g_tc_cta_group.exchange(cta_group);
}

int ftblas_set_fp64_engine(int engine) {
  if (engine != kEngineDFMA && engine != kEngineDMMA) return -1;
  return g_fp64_engine.exchange(engine);
}

int ftblas_set_fp64_tile(int edge) {
  if (edge != 0 && edge != kDBM && edge != kDBSmall) return -1;
  return g_fp64_tile.exchange(edge);
}

const char* ftblas_status_string(int code) {
  if (code == 0) return "success";
  if (code < 0) return "invalid argument (the negated code is its 1-based position)";
  switch (code) {
    case FTBLAS_STATUS_NOT_SUPPORTED: return "not supported (type, shape or alignment)";
    case FTBLAS_STATUS_CUDA_ERROR: return "CUDA runtime error (see ftblas_last_cuda_error)";
    case FTBLAS_STATUS_ALLOC_FAILED: return "workspace allocation failed";
    case FTBLAS_STATUS_WORKSPACE_LIMIT:
      return "problem needs more scratch than the static workspace of ftblas_gemm_ex_noalloc (16 MiB)";
    default: return "unknown status";
  }
}

int ftblas_last_cuda_error(void) { return g_last_cuda_error; }

int ftblas_last_launch_used_tma(void) { return g_last_used_tma; }

const char* ftblas_version(void) { return "0.1.0"; }

int ftblas_decode_e4m3(const void* codes, float* out, int64_t n, void* stream) {
  if (n > 0 && (codes == nullptr || reinterpret_cast<uintptr_t>(codes) % 8 != 0)) return -1;
  if (n > 0 && out == nullptr) return -2;
  if (n < 0) return -3;
  return record_cuda(launch_decode_e4m3(static_cast<const uint8_t*>(codes), out, n, static_cast<cudaStream_t>(stream)));
}

int ftblas_dgemm_unfused(ftblas_layout_t layout, ftblas_trans_t transa, ftblas_trans_t transb, int64_t M, int64_t N,
                         int64_t K, double alpha, const double* A, int64_t lda, const double* B, int64_t ldb,
                         double beta, double* C, int64_t ldc, void* stream, ft_report_t* report) {
  return dgemm_unfused_impl(layout, transa, transb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, stream, report);
}

int ftblas_dsymm(ftblas_layout_t layout, ftblas_side_t side, ftblas_uplo_t uplo, int64_t M, int64_t N, double alpha,
                 const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
                 void* stream, ft_report_t* report) {
  return dsymm_impl(layout, side, uplo, M, N, alpha, A, lda, B, ldb, beta, C, ldc, stream, report);
}

int ftblas_dtrmm(ftblas_layout_t layout, ftblas_side_t side, ftblas_uplo_t uplo, ftblas_trans_t transa,
                 ftblas_diag_t diag, int64_t M, int64_t N, double alpha, const double* A, int64_t lda, double* B,
                 int64_t ldb, void* stream, ft_report_t* report) {
  return dtrmm_impl(layout, side, uplo, transa, diag, M, N, alpha, A, lda, B, ldb, stream, report);
}

int ftblas_dtrsm(ftblas_layout_t layout, ftblas_side_t side, ftblas_uplo_t uplo, ftblas_trans_t transa,
                 ftblas_diag_t diag, int64_t M, int64_t N, double alpha, const double* A, int64_t lda, double* B,
                 int64_t ldb, void* stream, ft_report_t* report) {
  return dtrsm_impl(layout, side, uplo, transa, diag, M, N, alpha, A, lda, B, ldb, stream, report);
}

int ftblas_kernel_timing_begin(void) {
  std::lock_guard<std::mutex> lk(g_timer_mu);
  release_timer_pairs();
  g_timer_failed = false;
  g_timer_on = true;
  return 0;
}

int ftblas_kernel_timing_end(double* total_ms, int64_t* launches) {
  std::lock_guard<std::mutex> lk(g_timer_mu);
  g_timer_on = false;
  double t = 0.0;
  int64_t n = 0;
  bool failed = g_timer_failed;
  for (auto& pr : g_timer_pairs) {
    float ms = 0.0f;
    if (cudaEventSynchronize(pr.second) == cudaSuccess && cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) {
      t += ms;
      ++n;
    } else {
      failed = true;
    }
  }
  release_timer_pairs();
  if (total_ms) *total_ms = t;
  if (launches) *launches = n;
  return failed ? FTBLAS_STATUS_CUDA_ERROR : 0;
}

}  // extern "C"
