// sv_tc.cu -- tensor-core (tcgen05, 3xTF32) stage product: self-test and host helpers.
//
// A register stage of a pass (see StageRec) holds, in every thread, the 2^R
// amplitudes of one "row" (R = 4 or 5): the values of the stage's R register
// qubits for the thread's fixed values of the other tile qubits.  All dense
// fused blocks of the stage multiply into one 2^R x 2^R complex matrix U (built
// on the host in complex128).  Applying it to the whole tile is the real GEMM
//
//     D[m][n] = sum_k A[m][k] * B[n][k],   m = row (thread), k, n < K = 2^(R+1),
//
// with A[m][2j+c] = component c (re/im) of amplitude j of row m and B the real
// embedding of U: B[2r][2j] = Re U[r][j], B[2r][2j+1] = -Im U[r][j],
// B[2r+1][2j] = Im U[r][j], B[2r+1][2j+1] = Re U[r][j].
//
// Precision: split-TF32 (3xTF32).  x = x_hi + x_lo with x_hi the TF32 part of
// x and x_lo = x - x_hi; the product is taken as A_hi*B_hi + A_hi*B_lo +
// A_lo*B_hi with float32 accumulation, dropping A_lo*B_lo -- the split-precision
// tensor-core scheme of Ootomo & Yokota (2022), after Markidis et al. (2018).
// B is split on the host (x_hi = x rounded to the nearest TF32 value), A on the
// device (Veltkamp splitting, also round to nearest); x_lo takes either sign,
// so the tensor core's truncation of x_lo to TF32 has no systematic direction.
//
// Mapping to tcgen05 (per 128-row group):
//   * A_hi, A_lo live in tensor memory (lane = row % 128, K columns each),
//     written by the threads with tcgen05.st;
//   * B' = [B_hi ; B_lo] (per stage, 2K x K: 8 KB for R = 4, 32 KB for R = 5)
//     sits in shared memory in the canonical K-major layout without swizzle
//     (8-row x 16-byte core matrices);
//   * one thread issues the stage's K/4 MMAs (issue_stage_mma): A_hi times B'
//     (N = 2K) gives A_hi B_hi in D_left and A_hi B_lo in D_right, then A_lo
//     times B_hi (N = K) accumulates into D_left; the threads add D_left and
//     D_right (round to nearest) after tcgen05.ld;
//   * every mbarrier wait is bounded by %globaltimer and reported, never trapped.
#include <cstdint>
#include <cstring>
#include <vector>

#include "sv_internal.h"
#include "sv_tc.h"
#include "sv_tc_ptx.cuh"

namespace svgb {

// ---- self-test: one 128 x 32 x 32 product -----------------------------------------

template <int R>
__global__ void __launch_bounds__(128) k_tc_selftest(const float *__restrict__ A, const uint8_t *__restrict__ bimg,
                                                     float *__restrict__ D, int *__restrict__ status) {
  constexpr uint32_t K = tc_k(R), IMG = tc_b_image_bytes(R), COLS = tc_cols_per_group(R);
  extern __shared__ __align__(1024) uint8_t bsm[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tbase_s;
  const uint32_t tid = threadIdx.x, warp = tid >> 5;
  for (uint32_t i = tid; i < IMG / 16; i += blockDim.x)
    reinterpret_cast<uint4 *>(bsm)[i] = reinterpret_cast<const uint4 *>(bimg)[i];
  fence_proxy_async_smem();
  if (warp == 0) {
    tmem_alloc(&tbase_s, COLS);
    tmem_relinquish();
  }
  if (tid == 0) mbar_init(&bar, 1);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tbase_s;
  const uint32_t tq = tbase + ((warp * 32u) << 16);
  float2 v[1 << R];
  for (uint32_t j = 0; j < K / 2; j++) v[j] = make_float2(A[tid * K + 2 * j], A[tid * K + 2 * j + 1]);
  store_row_split<R>(tq, v);
  tmem_wait_st();
  tc_fence_before();
  __syncthreads();
  if (tid == 0) {
    tc_fence_after();
    issue_stage_mma<R>(tbase, smem_u32(bsm));
    mma_commit(&bar);
  }
  const bool ok = mbar_wait_bounded(&bar, 0);
  tc_fence_after();
  if (__syncthreads_and(ok)) {
    load_row_sum<R>(tq, v);
    for (uint32_t j = 0; j < K / 2; j++) {
      D[tid * K + 2 * j] = v[j].x;
      D[tid * K + 2 * j + 1] = v[j].y;
    }
    if (tid == 0) *status = 0;
  } else if (tid == 0) {
    *status = 1;
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tbase, COLS);
}

// ---- bounded-wait check: an mbarrier that nothing arrives on -------------------------

__global__ void k_wait_nothing(uint32_t limit_ns, int *status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  bool done = mbar_try_wait(&bar, 0);
  const uint64_t t0 = global_ns();
  while (!done && global_ns() - t0 < limit_ns) done = mbar_try_wait(&bar, 0);
  __syncthreads();
  if (threadIdx.x == 0) *status = done ? 0 : 1;
}

cudaError_t wait_nothing(uint32_t limit_ms, int *status_host) {
  int *d = nullptr;
  cudaError_t e = cudaMalloc(&d, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(d, 0xff, sizeof(int));
  if (e == cudaSuccess) {
    k_wait_nothing<<<1, 32>>>(limit_ms * 1000000u, d);
    count_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(status_host, d, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d);
  return e;
}

// ---- host helpers ------------------------------------------------------------------

static inline float tf32_rn(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u = (u + 0x1000u) & 0xFFFFE000u;
  float r;
  std::memcpy(&r, &u, 4);
  return r;
}

size_t tc_b_offset(int R, int n, int k) {
  const int ks = k >> 3, kk = k & 7;
  return size_t(ks) * tc_b_kstep(R) + size_t(n >> 3) * 256 + size_t(kk >> 2) * 128 + size_t(n & 7) * 16 +
         size_t(kk & 3) * 4;
}

void tc_b_image(int R, const double *B, uint8_t *img) {
  const int K = int(tc_k(R));
  std::memset(img, 0, tc_b_image_bytes(R));
  for (int n = 0; n < K; n++)
    for (int k = 0; k < K; k++) {
      const double x = B[n * K + k];
      const float hi = tf32_rn(float(x));
      const float lo = tf32_rn(float(x - double(hi)));
      std::memcpy(img + tc_b_offset(R, n, k), &hi, 4);
      std::memcpy(img + tc_b_offset(R, n + K, k), &lo, 4);
    }
}

cudaError_t tc_selftest(int R, const float *A_host, const double *B_host, float *D_host, int *status_host) {
  if (R != 4 && R != 5) return cudaErrorInvalidValue;
  const uint32_t K = tc_k(R), IMG = tc_b_image_bytes(R);
  std::vector<uint8_t> img(IMG);
  tc_b_image(R, B_host, img.data());
  const size_t abytes = size_t(128) * K * 4;
  float *dA = nullptr, *dD = nullptr;
  uint8_t *dB = nullptr;
  int *dS = nullptr;
  cudaError_t e = cudaMalloc(&dA, abytes);
  if (e == cudaSuccess) e = cudaMalloc(&dD, abytes);
  if (e == cudaSuccess) e = cudaMalloc(&dB, IMG);
  if (e == cudaSuccess) e = cudaMalloc(&dS, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(dA, A_host, abytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dB, img.data(), IMG, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(dD, 0, abytes);
  if (e == cudaSuccess) {
    if (R == 4) {
      k_tc_selftest<4><<<1, 128, IMG>>>(dA, dB, dD, dS);
    } else {
      e = cudaFuncSetAttribute(k_tc_selftest<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(IMG));
      if (e == cudaSuccess) k_tc_selftest<5><<<1, 128, IMG>>>(dA, dB, dD, dS);
    }
    count_launch();
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(D_host, dD, abytes, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(status_host, dS, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(dA);
  cudaFree(dD);
  cudaFree(dB);
  cudaFree(dS);
  return e;
}

}  // namespace svgb
