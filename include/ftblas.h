/*
 * ftblas.h - C ABI of the GB300 (sm_103a) ABFT-protected GEMM.
 *
 * Operation (FT-BLAS, Zhai et al., ICS '21, Section II.A with Section V): the BLAS GEMM
 *     C = alpha * op(A) * op(B) + beta * C,   op(X) = X or X^T,
 * where op(A) is M x K, op(B) is K x N and C is M x N, protected by Huang-Abraham
 * checksums (Section II.A): column sums e^T A and row sums B e are encoded while the
 * operand tiles are staged, the row and column checksums of every output tile are
 * verified after the product (C = beta*C folded in, Section V.B), and a single corrupted
 * element per tile is located at the crossing of the mismatching row and column
 * (Section V.A) and corrected (Section VI.C). One verification interval is one output
 * tile over all of K in one call; ftblas_verification_tile() reports its shape.
 *
 * Workspace: the calls that need workspace take it stream-ordered from a memory pool the
 * library creates per device, and release it on the same stream; the pool keeps the memory
 * it has reserved (up to the largest call's need) until the process exits, so that calls do
 * not map and unmap device memory each time.
 *
 * Storage follows BLAS/CBLAS: column-major (element (r, c) of X at X[r + c*ld], ld >=
 * max(1, rows)) or row-major (X[r*ld + c], ld >= max(1, cols)), selected per call.
 *
 * Ownership and asynchrony: A, B, C are caller-owned DEVICE pointers; the library never
 * frees them. A call validates its arguments on the host, enqueues its kernels on
 * `stream` (a cudaStream_t; NULL = the legacy default stream) and returns without
 * synchronising. The report, when given, must be device-accessible memory (device,
 * pinned-mapped or managed); the call resets it on the stream and the kernels fill it, so
 * it is valid after the stream has been synchronised. C and the report must not be used
 * by other work on other streams while the call is in flight.
 *
 * Return values (all entry points): 0 on success; -p when argument p (1-based, in the
 * order of the signature) is invalid, BLAS xerbla style; a positive FTBLAS_STATUS_* code
 * otherwise. Detection results never change the return value (the call is asynchronous):
 * they are in the report.
 */
#ifndef FTBLAS_H_
#define FTBLAS_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { FTBLAS_ROW_MAJOR = 101, FTBLAS_COL_MAJOR = 102 } ftblas_layout_t;   /* CBLAS values */
typedef enum { FTBLAS_NO_TRANS = 111, FTBLAS_TRANS = 112 } ftblas_trans_t;
typedef enum { FTBLAS_UPPER = 121, FTBLAS_LOWER = 122 } ftblas_uplo_t;
typedef enum { FTBLAS_NON_UNIT = 131, FTBLAS_UNIT = 132 } ftblas_diag_t;
typedef enum { FTBLAS_LEFT = 141, FTBLAS_RIGHT = 142 } ftblas_side_t;

/* Element types of ftblas_gemm_ex. */
typedef enum {
  FTBLAS_R_64F = 0,      /* binary64 */
  FTBLAS_R_32F = 1,      /* binary32 */
  FTBLAS_R_16BF = 2,     /* bfloat16 */
  FTBLAS_R_8F_E4M3 = 3   /* OCP FP8 E4M3 (finite-only, max 448) */
} ftblas_dtype_t;

/* Positive status codes. */
#define FTBLAS_STATUS_NOT_SUPPORTED 2   /* dtype / shape / alignment combination not provided */
#define FTBLAS_STATUS_CUDA_ERROR 3      /* a CUDA runtime call failed (see ftblas_last_cuda_error) */
#define FTBLAS_STATUS_ALLOC_FAILED 4    /* the library could not obtain workspace */
#define FTBLAS_STATUS_WORKSPACE_LIMIT 5 /* ftblas_gemm_ex_noalloc: problem exceeds its static scratch */

/* Report status bits (ft_report_t.status). */
#define FT_STATUS_TIMEOUT 1u            /* a bounded device wait gave up; affected tiles were not stored */
#define FT_STATUS_RECORDS_TRUNCATED 2u  /* more than FTBLAS_MAX_RECORDS records were produced */

/* Record kinds (ft_error_record_t.kind). */
#define FT_KIND_CORRECTED 1       /* one row and one column mismatched: element located and recomputed */
#define FT_KIND_CHECKSUM_ONLY 2   /* mismatch on one side only: fault in the checksum path; C kept */
#define FT_KIND_UNCORRECTABLE 3   /* several rows and/or columns mismatched; C left as computed */
#define FT_KIND_INPUT_NONFINITE 4 /* an encoded checksum of A, B or C_in is not finite; not checked */

#define FTBLAS_MAX_RECORDS 64

/* One detection event, in the caller's coordinates of C (row-major calls included). */
typedef struct {
  int64_t tile_row, tile_col;   /* verification tile: rows [tile_row*tile_rows, ...), columns likewise */
  int64_t i, j;                 /* located element, or the first flagged row / column (-1: none) */
  double delta_row;             /* C^r_ref(i) - C^r(i): reference minus predicted row checksum */
  double delta_col;             /* C^c_ref(j) - C^c(j) */
  double tau_row, tau_col;      /* round-off thresholds the deltas were compared with */
  double value_before;          /* C(i, j) as computed, error included (FT_KIND_CORRECTED) */
  double value_after;           /* C(i, j) as stored after recomputation */
  int32_t kind;                 /* FT_KIND_* */
  int32_t rows_flagged, cols_flagged;
  int32_t reserved;
} ft_error_record_t;

/* Per-call detection report (Section VI.C: located element, magnitude, correction). */
typedef struct {
  uint64_t tiles_checked;     /* verification intervals (tiles) checked */
  uint64_t detected;          /* tiles with any mismatch */
  uint64_t corrected;         /* tiles with one located and corrected element */
  uint64_t uncorrectable;     /* tiles left as computed: several mismatching rows/columns */
  uint64_t checksum_only;     /* tiles with a mismatch on one side only */
  uint64_t input_nonfinite;   /* tiles whose encoded input checksums were not finite */
  uint32_t status;            /* FT_STATUS_* bits */
  uint32_t n_records;         /* records produced (may exceed FTBLAS_MAX_RECORDS; see status) */
  ft_error_record_t rec[FTBLAS_MAX_RECORDS];
} ft_report_t;

/* ---------------------------------------------------------------------------------- */
/* Fault injection (Section VI.C: errors injected into C at chosen points, then        */
/* detected, located and corrected). Test and benchmark facility; off by default.     */
/* ---------------------------------------------------------------------------------- */

#define FT_SITE_ACCUM 1     /* flip a bit of the running sum of C(i,j) after bk*floor(nk/2) products */
#define FT_SITE_OUTPUT 2    /* perturb C(i,j) after alpha/beta, before verification */
#define FT_SITE_CHECKSUM 3  /* perturb the predicted row checksum C^r(i) of the tile holding (i,j) */
#define FT_SITE_STALL 4     /* fixed points only (a test of the bounded waits), FP64 GEMM kernels
                               staged by TMA and the tensor-core product kernel: the staging barrier of
                               k-tile k_tile (0: the middle one) of the tile holding (i,j) expects 16
                               bytes more than arrive, so it never completes; the call's waits give up
                               after 20 ms instead of 4 s (2 s), the tile is not stored (the persistent
                               tensor-core CTA also abandons its later tiles) and the report's status
                               gets FT_STATUS_TIMEOUT. Other kernels ignore the point. */
#define FT_MODE_BITFLIP 0   /* XOR bit `bit` (0 = lsb of the IEEE pattern of the accumulator type) */
#define FT_MODE_ADD_REL 1   /* add sign * 2^rel_log2 * |value| */

#define FTBLAS_MAX_FIXED_INJECTIONS 16
#define FTBLAS_MAX_INJECTIONS_PER_LAUNCH 64

typedef struct {
  int64_t i, j;               /* element of C, caller's coordinates */
  int32_t site, mode, bit, rel_log2, sign;
  int32_t k_tile;             /* FP64 accumulator site: flip after k_tile k-tiles of products
                                 (0: after floor(nk/2)); the tensor-core paths flip after all K.
                                 The injection model holds one FP64 accumulator point per element
                                 and launch: the oracle applies only the first point at an element,
                                 so a plan with two there has no reference (the seeded draw never
                                 makes one: its points fall in distinct tiles) */
} ft_inject_point_t;

typedef struct {
  uint64_t seed;              /* seeded draw: SplitMix64 stream seed ^ (launch * 0xD1B54A32D192ED03) */
  int32_t site, mode;         /* FT_SITE_*, FT_MODE_* of drawn points */
  int32_t bit_lo, bit_hi;     /* drawn bit range (inclusive) */
  int32_t log2_lo, log2_hi;   /* drawn rel_log2 range (inclusive) */
  int32_t every_n_launches;   /* launch n injects when n % every == seed % every; 0 = no draw */
  int32_t errors_per_launch;  /* distinct tiles per injecting launch (<= FTBLAS_MAX_INJECTIONS_PER_LAUNCH) */
  int32_t n_fixed;            /* > 0: inject exactly fixed[0..n_fixed-1] on every launch instead */
  int32_t reserved;
  ft_inject_point_t fixed[FTBLAS_MAX_FIXED_INJECTIONS];
} ft_inject_t;

/* Fault injection of Section VI.C's experiment. Install (cfg != NULL) or remove (cfg == NULL)
 * the process-wide injection plan and reset the launch counter to 0. Every protected call with
 * M, N > 0 that passes validation counts as one launch. For launch n the seeded draw takes,
 * per injection, six SplitMix64 outputs in the order tile, row offset, column offset, bit,
 * rel_log2, sign; tiles are numbered t = tile_row + tile_col * n_tile_rows in the caller's
 * coordinates and drawn without replacement. Returns 0, or -1 when cfg is malformed (ranges,
 * counts). */
int ftblas_set_injection(const ft_inject_t* cfg);

/* Protected launches counted since the last ftblas_set_injection. */
uint64_t ftblas_injection_launch_count(void);

/* ---------------------------------------------------------------------------------- */
/* GEMM entry points                                                                  */
/* ---------------------------------------------------------------------------------- */

/* FP64 ABFT-protected GEMM (Sections II.A, V; products and checksums in binary64).
 * Arguments 1-16: layout, transa, transb, M, N, K (>= 0), alpha, A, lda, B, ldb, beta, C,
 * ldc, stream, report (NULL: no report). A and B are read only; C is read when beta != 0
 * and written. M == 0 or N == 0 returns at once; K == 0 or alpha == 0 computes C = beta*C
 * with no checks; beta == 0 never reads C (NaN there does not propagate). */
int ftblas_dgemm(ftblas_layout_t layout, ftblas_trans_t transa, ftblas_trans_t transb,
                 int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t lda,
                 const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
                 void* stream, ft_report_t* report);

/* The same kernel with the protection compiled out (no encode, verify or correction, no
 * injection): the baseline the ABFT overhead is measured against, as Section VI.B compares
 * FT-BLAS with its own implementation without FT capability. Same arguments; no
 * report. */
int ftblas_dgemm_noabft(ftblas_layout_t layout, ftblas_trans_t transa, ftblas_trans_t transb,
                        int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t lda,
                        const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
                        void* stream);

/* FT-DSYMM (the Level-3 routines beside GEMM, Sections III.C and VI.B): C = alpha A B + beta C (side LEFT, A
 * M x M) or C = alpha B A + beta C (side RIGHT, A N x N), A symmetric with only its `uplo`
 * triangle read. A full copy of A is formed on `stream` (workspace from the stream-ordered
 * allocator) and the product runs through ftblas_dgemm's protected kernel: same report,
 * tiles, thresholds, injection plan and online verification. Arguments 1-15 in CBLAS
 * order (layout, side, uplo, M, N, alpha, A, lda, B, ldb, beta, C, ldc, stream, report);
 * returns -p for a bad argument p, or an FTBLAS_STATUS_* code. */
int ftblas_dsymm(ftblas_layout_t layout, ftblas_side_t side, ftblas_uplo_t uplo, int64_t M, int64_t N,
                 double alpha, const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                 double* C, int64_t ldc, void* stream, ft_report_t* report);

/* FT-DTRMM (the Level-3 routines beside GEMM, Sections III.C and VI.B): B = alpha op(A) B
 * (side LEFT, A M x M) or B = alpha B op(A) (side RIGHT, A N x N), A triangular (`uplo`,
 * `diag`: FTBLAS_UNIT takes the diagonal as 1 without reading it), B overwritten. A copy of
 * op(A) with explicit zeros and a copy of B are formed on `stream`, then ftblas_dgemm's
 * protected kernel runs, each tile visiting only the k-tiles the triangle leaves nonzero
 * (about half the work of the full product). When the other storage layout gives a better
 * launch order of these unequal tiles (heaviest first, or no longer heaviest last), the copies
 * and the product are made in that layout and the product is copied back. The values are the
 * same. The workspace is then n^2 + 2 M N doubles instead of n^2 + M N (n = M or N, A's
 * order). Protection as for ftblas_dgemm; an accumulator injection point whose k-tile
 * (explicit, or floor(nk/2)) falls outside its tile's range is not applied. Arguments 1-14 in
 * CBLAS order (layout, side, uplo, transa, diag, M, N, alpha, A, lda, B, ldb, stream, report). */
int ftblas_dtrmm(ftblas_layout_t layout, ftblas_side_t side, ftblas_uplo_t uplo, ftblas_trans_t transa,
                 ftblas_diag_t diag, int64_t M, int64_t N, double alpha, const double* A, int64_t lda,
                 double* B, int64_t ldb, void* stream, ft_report_t* report);

/* FT-DTRSM: op(A) X = alpha B (side LEFT, A M x M) or X op(A) = alpha B (side RIGHT, A N x N),
 * A triangular (`uplo`, `diag`), X overwriting B. Recursive blocked substitution on a
 * column-major copy (workspace from the library's workspace pool): the off-diagonal updates
 * run through ftblas_dgemm's protected kernel, and each 128-row diagonal block is solved by
 * a kernel that verifies every right-hand side by its checksum, e^T (T X) = (e^T T) X
 * against e^T R (Section II.A applied to T X = R), and solves a mismatching column again
 * from its untouched right-hand side (bit-exact). `report` sums all internal steps; records
 * carry B's (i, j) and, for the diagonal solves, the first row where the solved-again
 * column differed. The injection plan applies to every internal step, in that step's own
 * coordinates (a diagonal solve flips bit `bit` of X(i, j) as it is formed). A singular
 * diagonal is not detected (as in BLAS). Arguments 1-14 in CBLAS order. */
int ftblas_dtrsm(ftblas_layout_t layout, ftblas_side_t side, ftblas_uplo_t uplo, ftblas_trans_t transa,
                 ftblas_diag_t diag, int64_t M, int64_t N, double alpha, const double* A, int64_t lda,
                 double* B, int64_t ldb, void* stream, ft_report_t* report);

/* The unfused comparator (no counterpart in the fused design; it reproduces the
 * arrangement Section V improves on: ABFT as separate passes around a BLAS library call).
 * Same arguments, checks, report and injection plan as ftblas_dgemm, and the same
 * 128 x 128 verification tiles. The product is cuBLAS's DGEMM (loaded at run time); the
 * checksums are formed by separate bandwidth-bound passes that read op(A), op(B), C_in
 * (beta != 0) and the output C once each, plus two thin cuBLAS products for the predicted
 * checksums A (B e) and (e^T A) B. The threshold is ftblas_dgemm's with the magnitude
 * products bounded by (sum_k |A(i,k)|)(max_k sum_{j in tile} |B(k,j)|) and its transpose.
 * A located error is corrected from the row checksum as C^r(i) - sum_{j' != j} C(i,j')
 * (within the row threshold of the fault-free value, not bit-exact: the library's
 * summation order is unknown). Accumulator-site injection points act on the output
 * element (the library's accumulator is out of reach). Workspace comes from the
 * library's workspace pool. Returns FTBLAS_STATUS_NOT_SUPPORTED when cuBLAS cannot be
 * loaded or a dimension exceeds its 32-bit interface. */
int ftblas_dgemm_unfused(ftblas_layout_t layout, ftblas_trans_t transa, ftblas_trans_t transb,
                         int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t lda,
                         const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
                         void* stream, ft_report_t* report);

/* ftblas_dgemm (Sections II.A, V) on HOST buffers: copies A, B (and C when beta != 0) to
 * library-owned device workspace on `stream`, runs the protected GEMM, copies C and the report
 * back and synchronises the stream before returning (on failures too, so no copy outlives
 * the call). report (host memory) may be NULL. Pinned
 * host memory gives the fastest copies. Workspace grows to the largest call and is kept. */
int ftblas_dgemm_host(ftblas_layout_t layout, ftblas_trans_t transa, ftblas_trans_t transb,
                      int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t lda,
                      const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
                      void* stream, ft_report_t* report);

/* Mixed-precision ABFT-protected GEMM (Section II.A checksums; FP32 accumulation on the
 * tensor cores, binary64 checksum comparison). Arguments 1-22 in order: layout, transa,
 * transb, M, N, K, alpha, A, Atype, lda, B, Btype, ldb, beta, C, Ctype, ldc, compute_type,
 * a_scale, b_scale, stream, report. alpha and beta point to HOST scalars of the compute
 * type (double for FTBLAS_R_64F, float for FTBLAS_R_32F). Supported combinations:
 *   A, B, C, compute all FTBLAS_R_64F            -> the same path as ftblas_dgemm;
 *   A, B FTBLAS_R_16BF or both FTBLAS_R_8F_E4M3, compute FTBLAS_R_32F, C FTBLAS_R_32F
 *                                                 -> tcgen05 GEMM, C stored in FP32;
 *   the same with C FTBLAS_R_16BF                  -> the product is verified, located and
 *       corrected in FP32 exactly as above, and each element of C is rounded to nearest
 *       bfloat16 once. With the CTA-pair kernel (the default form) the epilogue reads C_in
 *       from the bfloat16 C and stores the rounded value there, and a protected call keeps
 *       the FP32 values in a buffer from the workspace pool for the resolve pass, which
 *       stores a corrected element in both; with one CTA per tile the product runs into
 *       that buffer (filled from C first when beta != 0) and C is rounded in one pass at the
 *       end. Either way C equals the rounding of the FP32 result. The checks cover the FP32
 *       values; the rounding itself is not checked.
 * a_scale / b_scale (device pointers to one float each) scale FP8 operands and must be
 * NULL otherwise. The tensor-core kernel reads both operands K-contiguous in the
 * column-major kernel frame (column-major: A transposed and B not; row-major: A not
 * transposed and B transposed), through tensor maps that need 16-byte aligned base
 * addresses and leading dimensions. Every transpose combination and alignment is accepted:
 * an operand stored the other way, or misaligned, is first copied K-major and aligned into
 * workspace from the library's workspace pool (one read and one write of it). Its threshold
 * assumes the tensor core accumulates in binary32 with unit roundoff 2^-23 (measured on
 * GB300: truncating accumulation). Protected tiles hold 128 x 248 outputs: B^r = [B, Be]
 * (Section II.A) fills the 256-column MMA, the last 8 columns holding the pieces of B e
 * (three bfloat16 or eight e4m3 pieces). Row checksums are verified in every tile and
 * column checksums only in tiles with a row mismatch (Section V.A); when those flag no
 * column (rows of very different scale) and beta == 0, the mismatching row is recomputed
 * and compared element by element; a located error is corrected by subtracting the row mismatch
 * (Section VI.C), evaluated as C^r(i) - sum_{j' != j} C(i,j') so that a huge or
 * non-finite error does not cancel catastrophically. Locating runs after the product, for
 * at most 64 mismatching tiles per call; further mismatching tiles of the same call are
 * reported as FT_KIND_UNCORRECTABLE (detected, C left as computed). Workspace (about
 * 16*K*ceil(N/248) + 8*K*ceil(M/128) + 4*M*ceil(K/256) bytes for BF16, 8*K*ceil(N/248) + ...
 * for FP8) is taken from the library's workspace pool and released on the same stream. */
int ftblas_gemm_ex(ftblas_layout_t layout, ftblas_trans_t transa, ftblas_trans_t transb,
                   int64_t M, int64_t N, int64_t K, const void* alpha,
                   const void* A, ftblas_dtype_t Atype, int64_t lda,
                   const void* B, ftblas_dtype_t Btype, int64_t ldb, const void* beta,
                   void* C, ftblas_dtype_t Ctype, int64_t ldc, ftblas_dtype_t compute_type,
                   const float* a_scale, const float* b_scale, void* stream, ft_report_t* report);

/* ftblas_gemm_ex with the protection compiled out (no encode pre-pass, no checksum MMA, no
 * verification): the baseline for the overhead (Section VI.B's comparison). Same arguments
 * without the report. */
int ftblas_gemm_ex_noabft(ftblas_layout_t layout, ftblas_trans_t transa, ftblas_trans_t transb,
                          int64_t M, int64_t N, int64_t K, const void* alpha,
                          const void* A, ftblas_dtype_t Atype, int64_t lda,
                          const void* B, ftblas_dtype_t Btype, int64_t ldb, const void* beta,
                          void* C, ftblas_dtype_t Ctype, int64_t ldc, ftblas_dtype_t compute_type,
                          const float* a_scale, const float* b_scale, void* stream);

/* ftblas_gemm_ex for callers that must not allocate device memory. The paper has no
 * counterpart: this entry point exists for integrations where the process does not own
 * the device allocator, so cudaMalloc / cudaMallocAsync are unavailable or forbidden
 * while work is being issued. Examples are a runtime whose memory is fully reserved up
 * front by another framework's caching allocator, a real-time or certification setting
 * that forbids allocation after initialisation, and a caller holding a lock under which
 * allocation could block. The protected BF16 GEMM (the argument list of ftblas_gemm_ex,
 * and only its BF16 combination: A, B FTBLAS_R_16BF, C and compute FTBLAS_R_32F; FP64,
 * FP8 E4M3 and a bfloat16 C return FTBLAS_STATUS_NOT_SUPPORTED; both operands K-contiguous in the kernel
 * frame with 16-byte aligned bases and leading dimensions, since this entry point makes no
 * copies: other operands return FTBLAS_STATUS_NOT_SUPPORTED) takes its encode scratch from one static
 * device array of 16 MiB that every GPU loading this library holds until the process
 * exits; nothing else is allocated (no cudaMalloc, cudaFree, stream-ordered or library
 * allocation).
 *   - Size limit: problems whose scratch, about 16*K*ceil(N/248) + 8*K*ceil(M/128) +
 *     4*M*ceil(K/256) bytes, exceeds 16 MiB are rejected with
 *     FTBLAS_STATUS_WORKSPACE_LIMIT before any device work (M = N = K = 8192 fits).
 *   - First call per device: the first call that launches the protected product looks
 *     up the device address of the static array, with the device current (argument,
 *     type and size checks and the quick returns come before and need no lookup); make
 *     that first call before any stream capture. A failed lookup returns
 *     FTBLAS_STATUS_CUDA_ERROR, its code readable with ftblas_last_cuda_error.
 *   - Sharing: every call on a device uses the same array and its encode pass writes
 *     every scratch entry its GEMM reads. Calls whose device work overlaps (different streams, or other
 *     threads) race on it and must be serialised by the caller.
 * Argument errors return -p as ftblas_gemm_ex does. */
int ftblas_gemm_ex_noalloc(ftblas_layout_t layout, ftblas_trans_t transa, ftblas_trans_t transb,
                           int64_t M, int64_t N, int64_t K, const void* alpha,
                           const void* A, ftblas_dtype_t Atype, int64_t lda,
                           const void* B, ftblas_dtype_t Btype, int64_t ldb, const void* beta,
                           void* C, ftblas_dtype_t Ctype, int64_t ldc, ftblas_dtype_t compute_type,
                           const float* a_scale, const float* b_scale, void* stream, ft_report_t* report);

/* Emulated FP64 ABFT-protected GEMM (Section II.A checksums, Section V.A's argument for
 * cheap checksums carried over to the product itself): the binary64 GEMM of ftblas_dgemm
 * (same arguments 1-16, same quick returns) formed on the E4M3 tensor cores from integer
 * slices.
 *   - Scales and slices: row i of op(A) is scaled by 2^-e_i, e_i the binary exponent of
 *     max_k |A(i,k)|, and column j of op(B) likewise; each scaled value x in (-1, 1) is
 *     split into s slices a_p = rint(r_p), r_0 = 16 x, r_{p+1} = 16 (r_p - a_p), integers of
 *     magnitude <= 16 (s = ftblas_set_emulation_slices, 14 by default).
 *   - Product: the groups G_g = sum_{p+q=g} A_p B_q, g < s, are formed exactly on the tensor
 *     cores (every partial sum an integer below 2^24: K <= ftblas_emulation_max_k(s), 16384
 *     for s = 14, else FTBLAS_STATUS_NOT_SUPPORTED), combined exactly in 128-bit integers,
 *     and C = alpha 2^(e_i + f_j - 4(s+1)) S + beta C_in in binary64 (S converted with one
 *     rounding). The error against the exact product is at most |alpha| 2^(e_i + f_j) K
 *     16^-s (s + 3) / 4 plus a few units of the last place of C: with s = 14, at most 3.3e-16
 *     of max|A| max|B| K.
 *   - Checks: in every tile of 128 x 248 outputs (ftblas_verification_tile with
 *     FTBLAS_R_8F_E4M3) each group's row sums are compared exactly with A_p (B_q e), B e
 *     held as four base-16 digits in the MMA's last columns: zero threshold, so every
 *     change of a group value is detected; C's row sums are compared with alpha sum_j v +
 *     beta sum_j C_in within the rounding of the binary64 stage.
 *   - Correction: a flagged row is recomputed exactly from the slices and stored, so C is
 *     the fault-free result bit for bit; records name the elements that differed
 *     (FT_KIND_CORRECTED, delta_row the integer mismatch or the binary64 stage's, tau_row 0
 *     for an integer check), or FT_KIND_CHECKSUM_ONLY when none did. More than 4 flagged
 *     rows in a tile, or more than 64 flagged tiles in a call: FT_KIND_UNCORRECTABLE, C as
 *     computed. A row or column holding a non-finite value gives NaN there, and its tiles
 *     are reported FT_KIND_INPUT_NONFINITE.
 *   - Injection: the accumulator site flips bit (bit & 31) of the binary32 value of G_g(i,j)
 *     with g = the point's k_tile (0: the leading group); the output and checksum sites
 *     act on C(i,j) and on group 0's predicted row checksum (adding sign max(1,
 *     floor(2^rel_log2 |P|))); the stall site as for the tensor-core product kernel.
 * Workspace (about 2 s (M + N) K bytes) from the library's workspace pool, released on the
 * same stream. Row-major calls compute C^T in the column-major frame, whose rows are the
 * caller's columns; the values are identical. */
int ftblas_dgemm_emulated(ftblas_layout_t layout, ftblas_trans_t transa, ftblas_trans_t transb,
                          int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t lda,
                          const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
                          void* stream, ft_report_t* report);

/* ftblas_dgemm_emulated with the protection compiled out (no checksum digits, no checks;
 * 256-column tiles): the baseline of its overhead, as Section VI.B compares FT-BLAS with its
 * own implementation without FT capability. Same arguments without the report. */
int ftblas_dgemm_emulated_noabft(ftblas_layout_t layout, ftblas_trans_t transa, ftblas_trans_t transb,
                                 int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t lda,
                                 const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
                                 void* stream);

/* Library control, no counterpart in the paper: slices per operand of the emulated FP64 GEMM,
 * 2 .. 15 (default 14). Fewer slices run faster with a larger error bound (above).
 * Returns the previous value, or -1 for another value. Process-wide. */
int ftblas_set_emulation_slices(int slices);

/* Library control, no counterpart in the paper: the largest K the emulated FP64 GEMM accepts
 * with `slices` slices, 2^18 / (slices + 2); -1 for slices outside 2 .. 15. */
int64_t ftblas_emulation_max_k(int slices);

/* Test support (no counterpart in the paper): the emulated GEMM's conversion of n 128-bit
 * integers (words[2i] low, words[2i+1] high, two's complement; device memory) to binary64
 * rounded to nearest, ties to even, into out (device memory). Asynchronous on stream.
 * Returns 0, -p for an invalid argument p, or FTBLAS_STATUS_CUDA_ERROR. */
int ftblas_emu_convert_i128(const int64_t* words, double* out, int64_t n, void* stream);

/* The verification interval of Section II.A (one error correctable in each): the shape of the
 * verification tile used for a call, in the caller's coordinates of C, and the k-tile depth
 * that sets the accumulator injection point (bk * floor(ceil(K/bk)/2) products; for the
 * tensor-core forms the k-tile of their staging, 128 bytes). compute_type selects the kernel
 * family: FTBLAS_R_64F (ftblas_dgemm and the Level-3 routines built on it), FTBLAS_R_32F or
 * FTBLAS_R_16BF (BF16 tensor-core path: 128 x 248 tiles, k-tile 64) or FTBLAS_R_8F_E4M3 (FP8
 * tensor-core path: 128 x 248 tiles, k-tile 128). FP64 tiles are square, 128 x 128, or 64 x 64
 * with the DFMA engine when 128-edge tiles would leave many of the current device's SMs idle:
 * the choice depends on M, N, the engine (ftblas_set_fp64_engine) and the SM count (152 when
 * no device answers). The unfused comparator ftblas_dgemm_unfused always verifies 128 x 128
 * tiles. Returns 0, or a negative argument index. */
int ftblas_verification_tile(ftblas_layout_t layout, ftblas_dtype_t compute_type,
                             int64_t M, int64_t N, int64_t K,
                             int64_t* tile_rows, int64_t* tile_cols, int64_t* k_tile);

/* Library control, no counterpart in the paper. FP64 product engine: 0 = DFMA (SIMT fused
 * multiply-add, default; 128 or 64 tile edge), 1 = DMMA (FP64 tensor-core mma.sync m8n8k4; 128
 * tile edge). Both run the same staging, encode and epilogue. Returns the previous engine, or
 * -1 for an unknown value. Process-wide. */
int ftblas_set_fp64_engine(int engine);

/* Library control, no counterpart in the paper. Tensor-core (BF16, FP8) product kernel: 2 =
 * a pair of CTAs on one TPC computes each 256 x 256 product with cta_group::2 MMAs, each CTA
 * staging its own 128 rows of A and half of the B columns; 1 = one CTA per 128 x 256
 * product; 0 = the faster form measured on GB300 (the default: CTA pairs, for protected and
 * unprotected calls). Both verify, locate and correct per
 * 128 x 248 tile (the verification interval of ftblas_verification_tile is the same), so
 * reports do not depend on the form; values agree within the accumulation bound. Returns the
 * previous setting, or -1 for a value other than 0, 1 or 2. Process-wide. */
int ftblas_set_tc_cta_group(int cta_group);

/* Library control, no counterpart in the paper. FP64 tile edge of the DFMA engine: 0 =
 * automatic (the default; the rule described at ftblas_verification_tile), 128 or 64 = that
 * edge for every later call. The DMMA engine always uses 128. Returns the previous setting, or
 * -1 for another value. Process-wide. */
int ftblas_set_fp64_tile(int edge);

/* Online verification (Section V.A): the FP64 protected kernels also check each tile
 * after every k_interval products (rounded up to whole k-tiles of ftblas_verification_tile's
 * depth), on the partial product, with the finished tile's threshold for the k processed so
 * far; exactly one mismatching row and column there are corrected at once by recomputing
 * that accumulator over those k (bit-exact), so one error per interval per tile is
 * correctable. Other patterns at an interval are left to the check of the finished tile.
 * Report counters then count verification events. 0 (the default) checks only the
 * finished tile. Process-wide; returns the previous value, or -1 for a negative argument. */
int64_t ftblas_set_verification_interval(int64_t k_interval);

/* Diagnostics (no counterpart in the paper). Staging path of the calling thread's most recent
 * GEMM launch: 1 = operands staged by TMA (16-byte aligned base addresses and leading
 * dimensions), 0 = cooperative loads (any other alignment), -1 = no kernel launched yet on
 * this thread. For tests and tuning. */
int ftblas_last_launch_used_tma(void);

/* Diagnostics (no counterpart in the paper): human-readable text of a return code. */
const char* ftblas_status_string(int code);

/* Diagnostics (no counterpart in the paper): cudaError_t of the last failing CUDA call made by
 * the library on this thread (0: none). */
int ftblas_last_cuda_error(void);

/* Diagnostics (no counterpart in the paper): library version, e.g. "0.1.0". */
const char* ftblas_version(void);

/* Test support (no counterpart in the paper). Decode n FP8 E4M3 codes (device memory, one byte
 * each, 8-byte aligned) to binary32 (device memory, n floats) with the unpacking that the
 * tensor-core path's encode kernel uses (eight codes per load, two per conversion
 * instruction). A diagnostic, so that tests can compare it code by code with the format's
 * definition (bias 7, subnormals at exponent field 0, S.1111.111 = NaN). Asynchronous on
 * `stream`. Returns 0, -p for an invalid argument p (null or misaligned pointer with n > 0, n
 * < 0), or FTBLAS_STATUS_CUDA_ERROR. */
int ftblas_decode_e4m3(const void* codes, float* out, int64_t n, void* stream);

/* Measurement support, no counterpart in the paper. Device time of the product kernels. After
 * ftblas_kernel_timing_begin, every GEMM call (any entry point, protected or not) records a
 * pair of CUDA events on its stream around its product kernel only: the encode, resolve and
 * scaling kernels and the report clear fall outside the pair. ftblas_kernel_timing_end stops
 * recording, waits for the recorded events, frees them, and returns in *total_ms the summed
 * durations and in *launches the number of timed launches (either pointer may be NULL).
 * Returns 0, or FTBLAS_STATUS_CUDA_ERROR if an event could not be created, recorded or read
 * (those launches are left out). Process-wide; begin discards pairs not yet collected. */
int ftblas_kernel_timing_begin(void);
int ftblas_kernel_timing_end(double* total_ms, int64_t* launches);

#ifdef __cplusplus
}
#endif

#endif /* FTBLAS_H_ */
