// Internal declarations shared by the host API (ftblas_api.cu) and the kernel translation
// units. Everything here is in the KERNEL frame: a column-major problem C = alpha *
// op(A) op(B) + beta C. A row-major call is mapped to it by computing C^T = op(B)^T op(A)^T,
// so kernel "rows" are caller columns; `swap_report` tells the kernels to write report
// records back in the caller's frame.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/ftblas.h"

namespace ftk {

// Injection sites in the kernel frame (the caller's FT_SITE_CHECKSUM maps to a row or a
// column checksum depending on the layout).
enum : int32_t { kSiteAccum = 1, kSiteOutput = 2, kSiteChecksumRow = 3, kSiteChecksumCol = 4, kSiteStall = 5 };

struct InjectPoint {
  int32_t i, j;          // kernel-frame element
  int32_t site, mode;    // kSite*, FT_MODE_*
  int32_t bit, rel_log2, sign;
  int32_t kt;            // FP64 accumulator and stall sites: k-tile of the point (0: floor(nk/2))
};

constexpr int kMaxInject = FTBLAS_MAX_INJECTIONS_PER_LAUNCH;

struct InjectList {
  int32_t n;
  int32_t pad;
  InjectPoint p[kMaxInject];
};

// Parameters of one FP64 launch (passed by value as a __grid_constant__ struct).
struct DgemmParams {
  int32_t M, N, K;               // kernel frame
  int32_t use_tma;               // 1: operands staged by TMA; 0: by cooperative loads
  double alpha, beta;
  const double* A; int64_t lda;  // kernel-frame op(A) source (recompute, fallback loads)
  const double* B; int64_t ldb;
  double* C; int64_t ldc;
  int32_t a_kmajor, b_kmajor;    // storage: A k-contiguous?  B k-contiguous?
  ft_report_t* report;           // may be null
  int32_t swap_report;           // 1: records in the transposed (caller row-major) frame
  int32_t kc_tiles;              // online verification every kc_tiles k-tiles (0: finished tile only)
  int32_t tri_a, tri_b;          // op(A) / op(B) triangular in the kernel frame: 0 no, 1 upper, 2 lower
                                 // (each tile then runs only the k-tiles the nonzero triangle reaches)
  uint64_t wait_limit_ns;        // limit of every bounded wait (short when a stall point is planned)
  InjectList inj;
};

// FP64 tile geometry. Tiles are square, kDBM x kDBN, or kDBSmall x kDBSmall (DFMA engine
// only) when the larger tiles would leave many SMs idle (fp64_tile_edge).
constexpr int kDBM = 128;      // tile rows (kernel frame)
constexpr int kDBN = 128;      // tile columns
constexpr int kDBSmall = 64;   // edge of the small tile
constexpr int kDBK = 32;       // k-tile depth
constexpr int kDStages = 3;    // smem ring depth
constexpr int kDThreads = 256; // 8 warps, all compute

enum Fp64Engine : int { kEngineDFMA = 0, kEngineDMMA = 1 };

// Tile edge (kDBM or kDBSmall) of the FP64 kernels for a kernel-frame M x N output on
// `engine`, given the GPU's SM count: the tile whose waves of CTAs, weighted by the checksum
// work per product operation (about 4 / edge), keep the most SMs busy; kDBSmall only when
// that gain is at least 3 %. DMMA: kDBM always.
int fp64_tile_edge(int64_t M, int64_t N, int engine, int sm_count);

// Launch the FP64 kernel family. `ft` selects protection; tile_edge must be
// fp64_tile_edge's answer for p.M, p.N (the TMA boxes are cut to it). Returns a cudaError_t.
cudaError_t launch_dgemm(const DgemmParams& p, const CUtensorMap* tmA, const CUtensorMap* tmB,
                         bool ft, int engine, int tile_edge, cudaStream_t stream);

// Unfused comparator (ftblas_dgemm_unfused): checksum passes around a library DGEMM.
struct UnfusedParams {
  int32_t M, N, K;               // kernel frame
  int32_t a_kmajor, b_kmajor;    // storage: op(A) k-contiguous (stored K x M)?  op(B) k-contiguous (K x N)?
  int32_t swap_report;
  double alpha, beta;
  const double* A; int64_t lda;
  const double* B; int64_t ldb;
  double* C; int64_t ldc;
  ft_report_t* report;           // may be null
  InjectList inj;                // output and checksum sites (accumulator points act on the output)
};
// Returns 0 or an FTBLAS_STATUS_* code; on a CUDA failure *cuda_err holds the error.
int unfused_dgemm(const UnfusedParams& p, cudaStream_t stream, cudaError_t* cuda_err);

// Stream-ordered workspace (released with cudaFreeAsync on the same stream) from a memory
// pool the library owns for the current device, which keeps what it has reserved between
// calls instead of returning it to the driver at every synchronisation.
cudaError_t ws_alloc(void** ptr, size_t bytes, cudaStream_t stream);

// Product-kernel timing (ftblas_kernel_timing_begin / _end): event records on `stream`
// immediately before and after a product kernel launch; no-ops unless timing is on.
void kernel_timer_start(cudaStream_t stream);
void kernel_timer_stop(cudaStream_t stream);

// Full copy of a symmetric (mode 0) or triangular (mode 1, op(X) with zeros and an optional
// unit diagonal) n x n matrix stored in one triangle of X, in X's layout with ld = n.
cudaError_t launch_expand(const double* X, int64_t ldx, bool row_major, int64_t n, int mode, bool upper, bool trans,
                          bool unit_diag, double* T, cudaStream_t stream);

// FT-DTRSM blocks (ft_trsm.cu).
constexpr int kTrsmLeaf = 128;  // diagonal block edge of the blocked substitution
// dst(r, c) = scale * src[r * rs + c * cs] into a column-major dst (leading dimension ld)
cudaError_t launch_copy2d(const double* src, int64_t rs, int64_t cs, double* dst, int64_t ld, int64_t rows,
                          int64_t cols, double scale, cudaStream_t stream);
// Solve the n x n (n <= kTrsmLeaf) lower / upper triangular block T X = W in place for
// nrhs columns of W, each column verified by its checksum and solved again on a mismatch.
cudaError_t launch_trsm_leaf(const double* T, int64_t ldt, double* W, int64_t ldw, int n, int64_t nrhs, bool lower,
                             ft_report_t* report, const InjectList& inj, cudaStream_t stream);
// Sum nparts step reports into out (records moved by row_off[p] rows, then transposed when swap).
cudaError_t launch_report_merge(const ft_report_t* parts, const int64_t* row_off, int nparts, ft_report_t* out,
                                bool swap, cudaStream_t stream);

// C = beta * C over an M x N column-major kernel-frame matrix (quick-return path).
cudaError_t launch_scale(double* C, int64_t ldc, int32_t M, int32_t N, double beta, cudaStream_t stream);

}  // namespace ftk
