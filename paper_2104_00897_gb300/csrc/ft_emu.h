// Internal declarations of the emulated FP64 path: binary64 operands split into E4M3
// integer slices, group products formed exactly by the tcgen05 tensor cores, exact integer
// row checksums per group, and the binary64 output stage. Kernel frame: C is M x N
// column-major, op(A) M x K, op(B) K x N (a row-major call is mapped by the host).
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "ft_internal.h"

namespace ftk {

constexpr int kEmuBM = 128;         // tile rows (TMEM lanes)
constexpr int kEmuBNProt = 248;     // data columns of a protected tile
constexpr int kEmuBNPlain = 256;    // data columns of an unprotected tile
constexpr int kEmuChkRows = 8;      // checksum rows after the data rows (four base-16 digits used)
constexpr int kEmuDigits = 4;
constexpr int kEmuSlicesDefault = 14;
constexpr int kEmuSlicesMax = 15;
constexpr int kEmuPendCap = 64;     // tiles with flagged rows the resolve pass handles per call
constexpr int kEmuPendRows = 4;     // flagged rows per tile the resolve pass recomputes

// Largest K for which every group value (and every partial sum) stays an integer of
// magnitude <= 2^24 with s slices: 64 (s + 2) K <= 2^24.
constexpr int64_t emu_max_k(int s) { return (int64_t(1) << 18) / (s + 2); }

// A flagged row of a tile, handed from the product kernel's epilogue to the resolve pass.
struct EmuPendRow {
  int32_t row;                     // tile-local row
  int32_t pad_;
  double delta, tau;               // first failed check of the row (tau 0: an exact integer check)
  double c_computed[kEmuBNProt];   // C(i, j) as the product kernel formed it
  double c_true[kEmuBNProt];       // C(i, j) recomputed by the resolve pass
  uint8_t differs[kEmuBNProt];
};
struct EmuPendEntry {
  int32_t mt, nt, nrows, first_row;
  uint32_t done;                   // resolve work items finished (the last one classifies)
  int32_t pad_[3];
  EmuPendRow r[kEmuPendRows];
};
struct EmuPending {
  uint32_t count;                  // tiles entered (may exceed kEmuPendCap: the rest are uncorrectable)
  uint32_t pad_[63];
  EmuPendEntry e[kEmuPendCap];
};

struct EmuParams {
  int32_t M, N, K;                 // kernel frame
  int32_t s;                       // slices per operand
  int32_t nMb, nNb;                // tile rows / columns
  int32_t bn;                      // data columns per tile (kEmuBNProt or kEmuBNPlain)
  int32_t swap_report;
  int64_t m_pad, n_pad;            // slice rows per slice: nMb * 128, nNb * bn
  int64_t kpitch;                  // bytes per slice row (K rounded up to 16)
  double alpha, beta;
  double* C; int64_t ldc;
  const int32_t* erow;             // [m_pad] row exponents of op(A)
  const int32_t* fcol;             // [n_pad] column exponents of op(B)
  const uint8_t* row_bad;          // [m_pad] row of op(A) holds a non-finite value
  const uint8_t* col_bad;          // [n_pad]
  const uint8_t* rowblk_bad;       // [nMb]  a row of the tile row block is bad
  const uint8_t* colblk_bad;       // [nNb]
  const uint8_t* aslices;          // [s][m_pad][kpitch] E4M3 integer slices of op(A) rows
  const uint8_t* bslices;          // [s][n_pad][kpitch] E4M3 integer slices of op(B) columns
  int64_t* scratch;                // [grid][2][bn][128] running sums of the two group halves
                                   // (H, L), L replaced by the output values after the last group
  EmuPending* pend;
  ft_report_t* report;
  uint64_t wait_limit_ns;
  InjectList inj;                  // accumulator site: group = point's kt
};

// Strided FP64 source of the split: element (r, k) of a matrix with R rows at
// base[r * rs + k * ks], K columns.
struct EmuSource {
  const double* base;
  int64_t rs, ks;
  int64_t R;
};

size_t emu_workspace_bytes(const EmuParams& p, int grid);
// Carve the workspace into p's arrays (p's sizes set).
void emu_workspace_carve(EmuParams& p, void* ws, int grid, uint8_t** chk_out);
// Exponents, non-finite flags and slices of op(A) rows and op(B) columns, and (protected)
// the checksum digits; all asynchronous on st.
cudaError_t launch_emu_split(const EmuParams& p, const EmuSource& a, const EmuSource& b, uint8_t* chk, bool ft,
                             cudaStream_t st);
// The product kernel (and, protected, the resolve pass).
cudaError_t launch_emu_gemm(const EmuParams& p, const CUtensorMap* tmA, const CUtensorMap* tmB,
                            const CUtensorMap* tmChk, bool ft, int grid, cudaStream_t st);
// Test support: rounded-to-nearest binary64 values of n 128-bit integers (lo, hi words).
cudaError_t launch_emu_convert(const int64_t* words, double* out, int64_t n, cudaStream_t st);

}  // namespace ftk
