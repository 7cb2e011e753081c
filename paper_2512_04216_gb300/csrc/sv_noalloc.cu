// sv_noalloc.cu -- an allocation-free variant of the Z-string expectation.
//
// sv_expect_pauli needs scratch memory for its per-CTA partial sums and gets it
// from cudaMalloc (lazily, per state).  Some callers cannot allocate device
// memory at the point where they want an expectation value -- for example a
// serving process that reserved all free HBM for resident state vectors up
// front (a cudaMalloc then fails or fragments that reservation), or a
// latency-critical loop that cannot afford cudaMalloc's implicit device-wide
// synchronisation.  sv_expect_z_static serves them: its scratch is the
// file-scope array below, fixed in size, loaded with the library and held by
// every GPU that loads it until the process exits.
//
// The array's name in host code is a host-side stand-in, not a device
// address, so host code never passes `g_static_scratch` itself to a kernel:
// the entry point looks up the device address once per device with
// cudaGetSymbolAddress (with that device current) and passes that pointer.
#include <cstdint>
#include <mutex>

#include "../../include/sv.h"
#include "sv_internal.h"

namespace svgb {

// Largest state served: 2^28 amplitudes -> 2^16 reduction CTAs, two doubles
// each, plus the two totals.  1 MiB + 16 bytes.
constexpr int kStaticMaxQubits = 28;
constexpr size_t kStaticParts = size_t(1) << (kStaticMaxQubits - 12);
constexpr size_t kStaticDoubles = 2 * kStaticParts + 2;

static __device__ __align__(256) double g_static_scratch[kStaticDoubles];

// out[0] = <Z_mask> = sum p (-1)^parity / sum p, out[1] = sum p.
__global__ void k_finish_expect(const double *__restrict__ sums, double *__restrict__ out) {
  const double p = sums[0], pz = sums[1];
  out[0] = p > 0.0 ? pz / p : 0.0;
  out[1] = p;
}

static double *g_scratch_dev[64] = {nullptr};
static std::mutex g_scratch_mu;

static cudaError_t static_scratch(int dev, double **out) {
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_dev[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_dev[dev] = static_cast<double *>(p);
  }
  *out = g_scratch_dev[dev];
  return cudaSuccess;
}

}  // namespace svgb

using namespace svgb;

extern "C" int sv_expect_z_static(const void *amplitudes, int n_qubits, uint64_t z_mask, double *out,
                                  void *cuda_stream) {
  if (!amplitudes || !out) return set_last_error(SV_ERR_ARG, "amplitudes and out must be device pointers");
  if (n_qubits < 1 || n_qubits > kStaticMaxQubits)
    return set_last_error(SV_ERR_ARG, "n_qubits must be in [1, %d] (fixed scratch of %zu bytes), got %d",
                          kStaticMaxQubits, kStaticDoubles * sizeof(double), n_qubits);
  if (z_mask >> n_qubits) return set_last_error(SV_ERR_ARG, "z_mask has bits beyond n_qubits");
  if (reinterpret_cast<uintptr_t>(amplitudes) % 16)
    return set_last_error(SV_ERR_ARG, "amplitudes must be 16-byte aligned");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess && (dev < 0 || dev >= 64)) e = cudaErrorInvalidDevice;
  double *scratch = nullptr;
  if (e == cudaSuccess) e = static_scratch(dev, &scratch);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  if (e == cudaSuccess)
    e = launch_reduce_pz(static_cast<const float2 *>(amplitudes), n_qubits, z_mask, scratch, kStaticParts,
                         scratch + 2 * kStaticParts, st);
  if (e == cudaSuccess) {
    k_finish_expect<<<1, 1, 0, st>>>(scratch + 2 * kStaticParts, out);
    count_launch();
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return set_last_error(SV_ERR_CUDA, "sv_expect_z_static: %s", cudaGetErrorString(e));
  return set_last_error(SV_OK, "");
}
