// sv_tc.h -- tensor-core (tcgen05 3xTF32) stage GEMM: constants and host helpers.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace svgb {

// A stage of R register qubits (R = 4 or 5) holds 2^R amplitudes per row, so its
// real-embedded product has K = 2^(R+1) columns.  Per stage, the operand
// B' = [B_hi ; B_lo] (2K rows n, K columns k, TF32 in 32-bit words) sits in the
// canonical K-major layout without swizzle: 8 KB for R = 4, 32 KB for R = 5.
__host__ __device__ constexpr uint32_t tc_k(int R) { return 2u << R; }
__host__ __device__ constexpr uint32_t tc_b_image_bytes(int R) { return 2u * tc_k(R) * tc_k(R) * 4u; }
// bytes per K step of 8 in the image (2K rows x 32 B)
__host__ __device__ constexpr uint32_t tc_b_kstep(int R) { return 2u * tc_k(R) * 32u; }
// TMEM columns per 128-row group: A_hi (K), A_lo (K), D (2K: D_left, D_right).
__host__ __device__ constexpr uint32_t tc_cols_per_group(int R) { return 4u * tc_k(R); }

// Byte offset of B'[n][k] (n < 2K, k < K) inside a stage image of width R.
size_t tc_b_offset(int R, int n, int k);
// Split a K x K real matrix B[n][k] (double) into the TF32 hi/lo image B'.
void tc_b_image(int R, const double *B, uint8_t *img);
// One 128 x K (A, host) times K x K (B[n][k], host) product on the tensor cores.
cudaError_t tc_selftest(int R, const float *A_host, const double *B_host, float *D_host, int *status_host);
// Waits (bounded by limit_ms) on an mbarrier that nothing arrives on; *status_host = 1 on timeout.
cudaError_t wait_nothing(uint32_t limit_ms, int *status_host);

}  // namespace svgb
