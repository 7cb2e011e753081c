// sv_tc.h -- tensor-core (tcgen05 3xTF32) stage GEMM: constants and host helpers.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace svgb {

constexpr uint32_t kTcBImage = 8192;       // B_hi (4 K steps x 1 KB) then B_lo
constexpr uint32_t kTcColsPerGroup = 128;  // TMEM columns per 128-row group: A_hi, A_lo, D0, D1
constexpr uint32_t kTcIssuersPerGroup = 2; // MMA-issuing warps per row group (half the K steps each)

// Byte offset of B[n][k] (n, k < 32) inside one 4 KB half of a stage image.
size_t tc_b_offset(int n, int k);
// Split a 32x32 real matrix B[n][k] (double) into the TF32 hi/lo image.
void tc_b_image(const double *B, uint8_t *img);
// One 128x32 (A, host) times 32x32 (B[n][k], host) product on the tensor cores.
cudaError_t tc_selftest(const float *A_host, const double *B_host, float *D_host, int *status_host);
// Waits (bounded by limit_ms) on an mbarrier that nothing arrives on; *status_host = 1 on timeout.
cudaError_t wait_nothing(uint32_t limit_ms, int *status_host);

}  // namespace svgb
