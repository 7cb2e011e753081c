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
// every call looks up the array's device address on the current device with
// cudaGetSymbolAddress (which allocates nothing) and passes that pointer.  The
// lookup is not cached, so the address stays right if the device's context is
// torn down and rebuilt (cudaDeviceReset) and the module is loaded again
// elsewhere.
#include <cmath>
#include <cstdint>

#include "../../include/sv.h"
#include "sv_internal.h"
#include <math_constants.h>

namespace svgb {

// Largest state served: 2^28 amplitudes -> 2^16 reduction CTAs, two doubles
// each, plus the two totals.  1 MiB + 16 bytes.
constexpr int kStaticMaxQubits = 28;
constexpr size_t kStaticParts = size_t(1) << (kStaticMaxQubits - 12);
constexpr size_t kStaticDoubles = 2 * kStaticParts + 2;
static_assert(kStaticParts >= reduce_parts_c(kStaticMaxQubits),
              "the fixed scratch must hold one partial pair per reduction CTA at the largest size");

static __device__ __align__(256) double g_static_scratch[kStaticDoubles];

// out[0] = <Z_mask> = sum p (-1)^parity / sum p, out[1] = sum p.  A state whose
// norm is zero or not finite gives out[0] = NaN (sv_expect_pauli reports the
// same case as SV_ERR_ARG; this call cannot, as it does not synchronise).
__global__ void k_finish_expect(const double *__restrict__ sums, double *__restrict__ out) {
  const double p = sums[0], pz = sums[1];
  out[0] = (p > 0.0 && isfinite(p)) ? pz / p : CUDART_NAN;
  out[1] = p;
}

static cudaError_t static_scratch(double **out) {
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  *out = static_cast<double *>(p);
  return e;
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
  double *scratch = nullptr;
  cudaError_t e = static_scratch(&scratch);
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
