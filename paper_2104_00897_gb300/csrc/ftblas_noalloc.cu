// ftblas_gemm_ex_noalloc: the protected BF16 GEMM on a static device scratch array, for
// callers that cannot allocate device memory (see the declaration in ftblas.h). The
// paper has no counterpart.
#include <mutex>

#include "ft_internal.h"
#include "ft_tc.h"

namespace {

// Scratch of the no-allocation entry point. Every GPU that loads the library holds it
// until the process exits. Host code must not use this name as a device address: the
// address comes from cudaGetSymbolAddress, per device.
constexpr size_t kStaticScratchBytes = size_t(16) << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the static scratch on the current device, looked up once per device
// (with that device current). Returns null on failure with the CUDA error in *err; the
// caller records it for ftblas_last_cuda_error.
void* scratch_for_current_device(cudaError_t* err) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    *err = e != cudaSuccess ? e : cudaErrorInvalidDevice;
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (g_scratch_addr[dev] == nullptr) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess || ptr == nullptr) {
      *err = e != cudaSuccess ? e : cudaErrorInvalidSymbol;
      return nullptr;
    }
    g_scratch_addr[dev] = ptr;
  }
  return g_scratch_addr[dev];
}

}  // namespace

extern "C" int ftblas_gemm_ex_noalloc(ftblas_layout_t layout, ftblas_trans_t transa, ftblas_trans_t transb, int64_t M,
                                      int64_t N, int64_t K, const void* alpha, const void* A, ftblas_dtype_t Atype,
                                      int64_t lda, const void* B, ftblas_dtype_t Btype, int64_t ldb, const void* beta,
                                      void* C, ftblas_dtype_t Ctype, int64_t ldc, ftblas_dtype_t compute_type,
                                      const float* a_scale, const float* b_scale, void* stream, ft_report_t* report) {
  // The address lookup runs inside, after the argument, type and size checks and only when
  // the protected product is launched.
  return ftk::gemm_bf16_ft_with_scratch(layout, transa, transb, M, N, K, alpha, A, Atype, lda, B, Btype, ldb, beta, C,
                                        Ctype, ldc, compute_type, a_scale, b_scale, stream, report,
                                        scratch_for_current_device, kStaticScratchBytes);
}
