// sv_tc.h -- tensor-core (tcgen05 3xTF32) stage GEMM: constants and host helpers.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace svgb {

// Per stage, the operand B' = [B_hi ; B_lo] (64 rows n, 32 columns k, TF32 in
// 32-bit words) in the canonical K-major layout without swizzle: 8 KB.
constexpr uint32_t kTcBImage = 8192;
constexpr uint32_t kTcBKStep = 2048;       // bytes per K step of 8 (64 rows x 32 B)
// TMEM columns per 128-row group: A_hi (32), A_lo (32), D (64: D_left, D_right).
constexpr uint32_t kTcColsPerGroup = 128;

// Byte offset of B'[n][k] (n < 64, k < 32) inside a stage image.
size_t tc_b_offset(int n, int k);
// Split a 32x32 real matrix B[n][k] (double) into the TF32 hi/lo image B'.
void tc_b_image(const double *B, uint8_t *img);
// One 128x32 (A, host) times 32x32 (B[n][k], host) product on the tensor cores.
cudaError_t tc_selftest(const float *A_host, const double *B_host, float *D_host, int *status_host);
// Waits (bounded by limit_ms) on an mbarrier that nothing arrives on; *status_host = 1 on timeout.
cudaError_t wait_nothing(uint32_t limit_ms, int *status_host);

}  // namespace svgb
