// Internal declarations of the reduced-precision (tcgen05) path, kernel frame: C is M x N
// column-major FP32, A is M x K and B is K x N, both K-contiguous.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "ft_internal.h"

namespace ftk {

constexpr int kTcBM = 128;       // tile rows (TMEM lanes)
constexpr int kTcBN = 256;       // data columns per tile, unprotected (= MMA N)
// Protected tiles: B^r = [B, Be] fills the MMA's N = 256 with the tile's data columns followed
// by the rows of the checksum operand that hold the pieces of B e: three bfloat16 pieces or
// eight e4m3 pieces, in 8 rows for both kinds (248 data columns).
constexpr int tc_chk_rows(int /*kind*/) { return 8; }
constexpr int tc_bn_prot(int kind) { return kTcBN - tc_chk_rows(kind); }
constexpr int kTcBNProtMax = 248;  // the larger tc_bn_prot: per-column arrays of a pending tile
static_assert(tc_bn_prot(0) <= kTcBNProtMax && tc_bn_prot(1) <= kTcBNProtMax, "pending-tile arrays too small");

// A tile whose row checksums mismatch, handed from the GEMM's epilogue to the resolve pass
// (lazy column side, row recompute, classification and correction), which runs after
// every tile is stored. Per-column results are written by the resolve pass.
constexpr int kTcPendCap = 64;   // mismatching tiles per call the resolve pass can locate
struct TcPendingEntry {
  int32_t mt, nt, nr, first_row;
  double delta_row, tau_row, pred_row;
  uint32_t done;                 // column groups finished (the last one classifies)
  int32_t pad_;
  double cin_sum[kTcBNProtMax];     // beta != 0: sum_i C_in(i,j) over the tile (C_in is overwritten)
  float cin_abs[kTcBNProtMax];      //            upward sum_i |C_in(i,j)|
  double col_delta[kTcBNProtMax];   // C^c_ref - C^c per column
  double col_tau[kTcBNProtMax];
  uint8_t col_flag[kTcBNProtMax];   // column mismatches
  uint8_t elem_flag[kTcBNProtMax];  // row recompute: element mismatches of the flagged row
};
struct TcPending {
  uint32_t count;                // tiles pushed (may exceed kTcPendCap; the rest are not located)
  uint32_t pad_[63];
  TcPendingEntry e[kTcPendCap];
};

struct TcParams {
  int32_t M, N, K;
  int32_t swap_report;
  float alpha, beta;
  float u_acc;                   // unit roundoff assumed for the tensor-core accumulation
  int32_t kind;                  // 0: BF16 operands, 1: FP8 E4M3 operands
  const float* a_scale;          // FP8 per-tensor scales (device values), or null
  const float* b_scale;
  const void* A; int64_t lda;
  const void* B; int64_t ldb;
  float* C; int64_t ldc;          // FP32 C (protected calls with a bfloat16 C: the verified FP32 copy)
  uint16_t* Cb; int64_t ldcb;     // bfloat16 C (bits): the CTA-pair kernel's epilogue reads C_in from
                                  // it and stores the rounded output there, the resolve pass a corrected
                                  // element; null for an FP32 C
  const float* rowAbsA;          // [M]        upward sum_k |A(i,k)|
  const float* maxAbsBe;         // [nNb]      max_k upward sum_{j in block} |B(k,j)|
  float* sA;                     // [nMb][sa_pitch] e^T A per 128-row block (binary32 sum), formed after
                                 // the GEMM for the row blocks of pending tiles only
  float* absSA;                  // [nMb][sa_pitch] upward sum_{i in block} |A(i,k)|, likewise
  int64_t sa_pitch;              // multiple of 8 (32-byte aligned rows)
  TcPending* pend;
  ft_report_t* report;
  uint64_t wait_limit_ns;        // limit of every bounded wait (short when a stall point is planned)
  InjectList inj;
};

struct TcWorkspace {
  void* chk;  int64_t kpitch;    // checksum operand, [nNb * 16][kpitch] elements of the input kind
  float* sA;
  float* absSA;
  float* rowAbsA;
  float* maxAbsBe;
  float* rowPart;                // [nkc][M] per-k-chunk partial sums of |A(i,k)|
  unsigned* rowdone;             // [nMb] k-chunks of each row block finished (follows maxAbsBe)
  size_t zero_bytes;             // maxAbsBe and rowdone: zeroed before the encode
  TcPending* pend;
  size_t bytes;
};

int64_t tc_kpitch(int32_t K);
size_t tc_workspace_bytes(int32_t M, int32_t N, int32_t K, int kind);
TcWorkspace tc_workspace_carve(void* base, int32_t M, int32_t N, int32_t K, int kind);
cudaError_t launch_scale_f32(float* C, int64_t ldc, int64_t M, int64_t N, float beta, cudaStream_t st);
cudaError_t launch_tc_encode(const TcParams& p, const TcWorkspace& w, cudaStream_t st);
// out[i] = the encode's binary32 value of E4M3 code codes[i], i < n
cudaError_t launch_decode_e4m3(const uint8_t* codes, float* out, int64_t n, cudaStream_t st);
// Tensor maps of one call, all K-major with 128-byte boxes along K: a (128 rows per box),
// b (data rows of B: BN per box for one CTA per tile, 128 for a CTA pair), b2 (a CTA pair's
// odd CTA, protected: 120 rows) and chk (the checksum operand, 8 rows).
struct TcMaps {
  CUtensorMap a, b, b2, chk;
};
// cg: 1 (one CTA per 128-row tile) or 2 (a CTA pair per 256 rows, cta_group::2). A bfloat16 C
// (p.Cb) needs cg 2; the one-CTA kernel writes only the FP32 C.
cudaError_t launch_tc_gemm(const TcParams& p, const TcMaps& m, bool ft, int cg, cudaStream_t st);

// K-major copy of an MN-major operand: dst[r * pitch + k] = src[r + k * ld] for r < R,
// k < K, elem_bytes 1 or 2 (asynchronous on st). pitch: tc_kmajor_pitch(K, elem_bytes), K
// rounded up to 16 bytes.
int64_t tc_kmajor_pitch(int64_t K, int elem_bytes);
cudaError_t launch_kmajor_copy(const void* src, int64_t R, int64_t K, int64_t ld, int elem_bytes, void* dst,
                               int64_t pitch, cudaStream_t st);

// Column-major R x Cc format conversions for bfloat16 outputs (asynchronous on st): with one
// CTA per tile the product runs into an FP32 buffer that the library rounds to bfloat16 at the
// end (and, for beta != 0, fills from the bfloat16 C first); C = beta C directly on a bfloat16
// matrix.
cudaError_t launch_f32_to_bf16(const float* src, int64_t sld, uint16_t* dst, int64_t dld, int64_t R, int64_t Cc,
                               cudaStream_t st);
cudaError_t launch_bf16_to_f32(const uint16_t* src, int64_t sld, float* dst, int64_t dld, int64_t R, int64_t Cc,
                               cudaStream_t st);
cudaError_t launch_scale_bf16(uint16_t* C, int64_t ldc, int64_t R, int64_t Cc, float beta, cudaStream_t st);

// Device address of a fixed scratch area, looked up only when a call needs it; returns null
// and sets *err on failure.
using ScratchResolver = void* (*)(cudaError_t* err);

// The protected BF16 GEMM of ftblas_gemm_ex run on a fixed scratch area of scratch_bytes
// bytes instead of stream-ordered allocations. Arguments are checked first, then the
// problem's scratch size (FTBLAS_STATUS_WORKSPACE_LIMIT before any device work); the
// scratch address is resolved only after that, and only when the call launches the
// protected product (quick returns never resolve it). A failed lookup returns
// FTBLAS_STATUS_CUDA_ERROR with the CUDA error recorded for ftblas_last_cuda_error.
int gemm_bf16_ft_with_scratch(int layout, int ta, int tb, int64_t M, int64_t N, int64_t K, const void* alpha,
                              const void* A, int Atype, int64_t lda, const void* B, int Btype, int64_t ldb,
                              const void* beta, void* C, int Ctype, int64_t ldc, int ctype, const float* a_scale,
                              const float* b_scale, void* stream, ft_report_t* report, ScratchResolver resolve,
                              size_t scratch_bytes);

}  // namespace ftk
