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
constexpr int kTcBNProt = 240;   // data columns per tile, protected: B^r = [B, Be] fills N = 256
constexpr int kTcChkRows = 16;   // rows of the checksum operand per column block (pieces of B e in 0..2)

struct TcParams {
  int32_t M, N, K;
  int32_t swap_report;
  float alpha, beta;
  float u_acc;                   // unit roundoff assumed for the tensor-core accumulation
  int32_t pad_;
  const void* A; int64_t lda;
  const void* B; int64_t ldb;
  float* C; int64_t ldc;
  const float* rowAbsA;          // [M]        upward sum_k |A(i,k)|
  const float* maxAbsBe;         // [nNb]      max_k upward sum_{j in block} |B(k,j)|
  const float2* sA;              // [nMb][K]   e^T A per 128-row block, hi + lo
  const float* absSA;            // [nMb][K]   upward sum_{i in block} |A(i,k)|
  ft_report_t* report;
  InjectList inj;
};

struct TcWorkspace {
  uint16_t* chk;  int64_t kpitch;
  float2* sA;
  float* absSA;
  float* rowAbsA;
  float* maxAbsBe;
  size_t bytes;
};

size_t tc_workspace_bytes(int32_t M, int32_t N, int32_t K);
TcWorkspace tc_workspace_carve(void* base, int32_t M, int32_t N, int32_t K);
cudaError_t launch_tc_encode(const TcParams& p, const TcWorkspace& w, void* ws_base, cudaStream_t st);
cudaError_t launch_tc_gemm(const TcParams& p, const CUtensorMap* tmA, const CUtensorMap* tmB, const CUtensorMap* tmChk,
                           bool ft, cudaStream_t st);

// The protected BF16 GEMM of ftblas_gemm_ex run on caller-supplied device scratch of
// ws_bytes bytes instead of stream-ordered allocations. Returns
// FTBLAS_STATUS_WORKSPACE_LIMIT, before any device work, when the problem needs more.
int gemm_bf16_ft_with_workspace(int layout, int ta, int tb, int64_t M, int64_t N, int64_t K, const void* alpha,
                                const void* A, int Atype, int64_t lda, const void* B, int Btype, int64_t ldb,
                                const void* beta, void* C, int Ctype, int64_t ldc, int ctype, const float* a_scale,
                                const float* b_scale, void* stream, ft_report_t* report, void* ws, size_t ws_bytes);

}  // namespace ftk
