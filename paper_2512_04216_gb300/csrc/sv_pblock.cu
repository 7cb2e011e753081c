// sv_pblock.cu -- partitioned-block kernels (§II p-block simulation; §III-E:
// registers merge when their qubits first interact, and communication qubits
// leave the register once measured or reset).
//
//   merge: out = a (x) b with a on the low qubits, out[i_b * 2^n_a + i_a] = b[i_b] a[i_a];
//   take:  qubit q known to be |v> leaves: out[j] = psi[j with bit v inserted at q].
//
// Both are HBM streams: merge writes 8 * 2^(n_a + n_b) bytes and reads a and b
// (a stays in L2 while b's rows are expanded); take reads and writes half the
// state once.
#include <cstdint>

#include "sv_internal.h"

namespace svgb {

__global__ void k_kron(const float2 *__restrict__ a, int na, const float2 *__restrict__ b, int nb,
                       float2 *__restrict__ out) {
  const uint64_t N = uint64_t(1) << (na + nb);
  const uint64_t amask = (uint64_t(1) << na) - 1;
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += stride) {
    const float2 x = a[i & amask], y = __ldg(b + (i >> na));
    out[i] = make_float2(x.x * y.x - x.y * y.y, x.x * y.y + x.y * y.x);
  }
}

__global__ void k_take(const float2 *__restrict__ psi, int n, int q, int v, float2 *__restrict__ out) {
  const uint64_t half = uint64_t(1) << (n - 1);
  const uint64_t low = (uint64_t(1) << q) - 1;
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t j = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < half; j += stride)
    out[j] = psi[((j & ~low) << 1) | (j & low) | (uint64_t(v) << q)];
}

static unsigned grid_for(uint64_t items) {
  const uint64_t g = (items + 255) / 256;
  return unsigned(g < 152ull * 32 ? g : 152ull * 32);
}

cudaError_t launch_kron(const float2 *a, int na, const float2 *b, int nb, float2 *out, cudaStream_t st) {
  if (na < 1 || nb < 1 || na + nb > 36) return cudaErrorInvalidValue;
  k_kron<<<grid_for(uint64_t(1) << (na + nb)), 256, 0, st>>>(a, na, b, nb, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_take(const float2 *psi, int n, int q, int v, float2 *out, cudaStream_t st) {
  if (n < 2 || q < 0 || q >= n || (v != 0 && v != 1)) return cudaErrorInvalidValue;
  k_take<<<grid_for(uint64_t(1) << (n - 1)), 256, 0, st>>>(psi, n, q, v, out);
  count_launch();
  return cudaGetLastError();
}

}  // namespace svgb
