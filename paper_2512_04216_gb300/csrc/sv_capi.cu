// sv_capi.cu -- the extern "C" entry points declared in include/sv.h.
//
// State handles own (or wrap) the amplitude buffer, a device copy of the
// current plan, and scratch buffers for the measurement kernels.  Every entry
// point validates its arguments, switches to the state's device for the
// duration of the call, and maps CUDA failures to status codes.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/sv.h"
#include "sv_internal.h"
#include "sv_plan.h"
#include "sv_tc.h"
#include "../../include/sv_diag.h"

using namespace svgb;

std::atomic<uint64_t> svgb::g_launches{0};

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

struct ProfRec {
  const char *name;
  cudaEvent_t a, b;
  double bytes;
};

}  // namespace

int svgb::set_last_error(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

// Pinned host staging + device copy of one chunk of a plan; reusable once the
// event recorded after the chunk's last kernel has completed.
struct PlanSlab {
  uint8_t *host = nullptr;
  uint8_t *dev = nullptr;
  size_t cap = 0;
  cudaEvent_t done = nullptr;
  bool live = false;
};

struct sv_state {
  int n = 0;
  int device = 0;
  float2 *amp = nullptr;
  bool owned = false;
  bool poisoned = false;
  cudaStream_t stream = nullptr;
  // measurement scratch
  MeasureScratch ms;
  double *dscal = nullptr;       // device scalars: [0] sum p, [1] sum pz, [2] total, [4..7] norm tracking
  uint64_t *dcount = nullptr;    // boundary counter
  int *derr = nullptr;           // device error word written by bounded waits
  double *hscal = nullptr;       // pinned host scalars
  void *stage = nullptr;         // device staging for host in/out buffers
  size_t stage_cap = 0;
  std::vector<PlanSlab> slabs;  // streamed plan chunks
  uint64_t *alias_table = nullptr;  // Walker alias table of the last sv_alias_build
  uint64_t *alias_tot = nullptr;    // build totals and error word (AliasScratch::tot)
  int alias_n = 0;
  // profiling
  bool prof = false;
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> evpool;
};

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

int cuda_fail(sv_state *s, cudaError_t e, const char *what) {
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();  // allocation failures do not poison the context
    return fail(SV_ERR_OOM, "%s: out of memory", what);
  }
  if (s) s->poisoned = true;
  return fail(SV_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(s, expr)                                         \
  do {                                                      \
    cudaError_t _e = (expr);                                \
    if (_e != cudaSuccess) return cuda_fail((s), _e, #expr); \
  } while (0)

#define CHECK_STATE(s)                                                                     \
  do {                                                                                     \
    if (!(s)) return fail(SV_ERR_ARG, "null state");                                       \
    if ((s)->poisoned) return fail(SV_ERR_STATE, "state poisoned by an earlier CUDA error"); \
  } while (0)

cudaEvent_t take_event(sv_state *s) {
  if (!s->evpool.empty()) {
    cudaEvent_t e = s->evpool.back();
    s->evpool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Runs `launch` bracketed by profiling events when profiling is on.
template <class F>
cudaError_t timed(sv_state *s, const char *name, double bytes, F &&launch) {
  if (!s->prof) return launch();
  ProfRec r{name, take_event(s), take_event(s), bytes};
  if (!r.a || !r.b) return launch();
  cudaEventRecord(r.a, s->stream);
  cudaError_t e = launch();
  cudaEventRecord(r.b, s->stream);
  s->recs.push_back(r);
  return e;
}

int ensure_dev(sv_state *s, void **p, size_t *cap, size_t need, const char *what) {
  if (*cap >= need) return SV_OK;
  if (*p) {
    CK(s, cudaStreamSynchronize(s->stream));
    cudaFree(*p);
    *p = nullptr;
    *cap = 0;
  }
  size_t bytes = need < 256 ? 256 : need;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) return cuda_fail(s, e, what);
  *cap = bytes;
  return SV_OK;
}

int ensure_scalars(sv_state *s) {
  if (!s->dscal) {
    CK(s, cudaMalloc(&s->dscal, 8 * sizeof(double)));
  }
  if (!s->dcount) {
    CK(s, cudaMalloc(&s->dcount, 8 * sizeof(uint64_t)));
  }
  if (!s->hscal) {
    CK(s, cudaMallocHost(&s->hscal, 8 * sizeof(double)));
  }
  if (!s->derr) {
    CK(s, cudaMalloc(&s->derr, sizeof(int)));
    CK(s, cudaMemsetAsync(s->derr, 0, sizeof(int), s->stream));
  }
  return SV_OK;
}

// After a stream synchronisation: report (and clear) a device-side timeout.
int check_device_error(sv_state *s) {
  if (!s->derr) return SV_OK;
  int e = 0;
  CK(s, cudaMemcpy(&e, s->derr, sizeof(int), cudaMemcpyDeviceToHost));
  if (e) {
    CK(s, cudaMemsetAsync(s->derr, 0, sizeof(int), s->stream));  // ordered before the state's later kernels
    if (e & 2) {
      s->poisoned = true;
      return fail(SV_ERR_STATE, "a pass found its device plan records different from the host's; the state is "
                                "not updated by that pass");
    }
    return fail(SV_ERR_TIMEOUT, "a bounded device-side wait gave up (tensor-core pass)");
  }
  return SV_OK;
}

int ensure_reduce(sv_state *s) {
  int rc = ensure_scalars(s);
  if (rc) return rc;
  const size_t parts = reduce_parts(s->n);
  if (s->ms.n_part * 1 < parts) {
    if (s->ms.part) {
      CK(s, cudaStreamSynchronize(s->stream));
      cudaFree(s->ms.part);
      s->ms.part = nullptr;
    }
    CK(s, cudaMalloc(&s->ms.part, 2 * parts * sizeof(double)));
    s->ms.n_part = parts;
  }
  return SV_OK;
}

int ensure_cdf(sv_state *s) {
  int rc = ensure_reduce(s);
  if (rc) return rc;
  const uint64_t N = uint64_t(1) << s->n;
  const size_t nchunk = size_t((N + 63) >> kChunkBits);
  const size_t nblock = size_t((N + 4095) >> kBlockBits);
  if (s->ms.n_chunk < nchunk) {
    if (s->ms.chunk) {
      CK(s, cudaStreamSynchronize(s->stream));
      cudaFree(s->ms.chunk);
      s->ms.chunk = nullptr;
    }
    CK(s, cudaMalloc(&s->ms.chunk, nchunk * sizeof(double)));
    s->ms.n_chunk = nchunk;
  }
  if (s->ms.n_block < nblock) {
    if (s->ms.block) {
      CK(s, cudaStreamSynchronize(s->stream));
      cudaFree(s->ms.block);
      s->ms.block = nullptr;
    }
    CK(s, cudaMalloc(&s->ms.block, nblock * sizeof(double)));
    s->ms.n_block = nblock;
  }
  return SV_OK;
}

int new_state(int n, int dtype, void *stream, sv_state **out) {
  if (!out) return fail(SV_ERR_ARG, "out is null");
  *out = nullptr;
  if (dtype == SV_C128) return fail(SV_ERR_UNSUPPORTED, "complex128 states are not supported");
  if (dtype != SV_C64) return fail(SV_ERR_ARG, "unknown dtype %d", dtype);
  if (n < 1 || n > 36) return fail(SV_ERR_ARG, "n_qubits must be in [1,36], got %d", n);
  sv_state *s = new sv_state();
  s->n = n;
  s->stream = static_cast<cudaStream_t>(stream);
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return fail(SV_ERR_CUDA, "no CUDA device");
  }
  *out = s;
  return SV_OK;
}

void free_state(sv_state *s) {
  if (!s) return;
  DeviceGuard g(s->device);
  cudaStreamSynchronize(s->stream);
  if (s->owned && s->amp) cudaFree(s->amp);
  if (s->ms.chunk) cudaFree(s->ms.chunk);
  if (s->ms.block) cudaFree(s->ms.block);
  if (s->ms.part) cudaFree(s->ms.part);
  if (s->dscal) cudaFree(s->dscal);
  if (s->dcount) cudaFree(s->dcount);
  if (s->derr) cudaFree(s->derr);
  if (s->hscal) cudaFreeHost(s->hscal);
  if (s->stage) cudaFree(s->stage);
  if (s->alias_table) cudaFree(s->alias_table);
  if (s->alias_tot) cudaFree(s->alias_tot);
  for (auto &r : s->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : s->evpool) cudaEventDestroy(e);
  for (auto &sl : s->slabs) {
    if (sl.host) cudaFreeHost(sl.host);
    if (sl.dev) cudaFree(sl.dev);
    if (sl.done) cudaEventDestroy(sl.done);
  }
  delete s;
}

}  // namespace

extern "C" {

const char *sv_last_error(void) { return g_err.c_str(); }

const char *sv_version(void) { return "svgb 0.1 (sm_103a)"; }

uint64_t sv_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

// A library-owned state whose buffer is left uninitialised when `reset` is
// false (for results that overwrite every amplitude: clone, merge, take).
static int create_state(int n_qubits, int dtype, void *cuda_stream, bool reset, sv_state **out) {
  int rc = new_state(n_qubits, dtype, cuda_stream, out);
  if (rc) return rc;
  sv_state *s = *out;
  const size_t bytes = (size_t(1) << n_qubits) * sizeof(float2);
  cudaError_t e = cudaMalloc(&s->amp, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete s;
    *out = nullptr;
    return fail(e == cudaErrorMemoryAllocation ? SV_ERR_OOM : SV_ERR_CUDA,
                "cudaMalloc of %zu bytes for a %d-qubit state: %s", bytes, n_qubits,
                cudaGetErrorString(e));
  }
  s->owned = true;
  if (!reset) return SV_OK;
  e = launch_reset(s->amp, n_qubits, 0, s->stream);
  if (e != cudaSuccess) {
    free_state(s);
    *out = nullptr;
    return fail(SV_ERR_CUDA, "reset: %s", cudaGetErrorString(e));
  }
  return SV_OK;
}

int sv_create(int n_qubits, int dtype, void *cuda_stream, sv_state **out) {
  return create_state(n_qubits, dtype, cuda_stream, true, out);
}

int sv_wrap(void *dev_ptr, int n_qubits, int dtype, void *cuda_stream, sv_state **out) {
  if (!dev_ptr) return fail(SV_ERR_ARG, "dev_ptr is null");
  if (reinterpret_cast<uintptr_t>(dev_ptr) % 16) return fail(SV_ERR_ARG, "dev_ptr must be 16-byte aligned");
  int rc = new_state(n_qubits, dtype, cuda_stream, out);
  if (rc) return rc;
  (*out)->amp = static_cast<float2 *>(dev_ptr);
  (*out)->owned = false;
  return SV_OK;
}

// dst waits for the work queued on src so far.
static cudaError_t stream_after(cudaStream_t dst, cudaStream_t src) {
  if (dst == src) return cudaSuccess;
  cudaEvent_t ev = nullptr;
  cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(ev, src);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(dst, ev, 0);
  if (ev) cudaEventDestroy(ev);
  return e;
}

int sv_destroy(sv_state *s) {
  free_state(s);
  return SV_OK;
}

int sv_set_stream(sv_state *s, void *cuda_stream) {
  CHECK_STATE(s);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  DeviceGuard g(s->device);
  // work queued on the new stream follows the work already queued on the old one
  // (scratch reallocations synchronise only the state's current stream)
  CK(s, stream_after(st, s->stream));
  s->stream = st;
  return SV_OK;
}

int sv_synchronize(sv_state *s) {
  CHECK_STATE(s);
  DeviceGuard g(s->device);
  CK(s, cudaStreamSynchronize(s->stream));
  return check_device_error(s);
}

int sv_num_qubits(const sv_state *s) { return s ? s->n : SV_ERR_ARG; }

void *sv_device_ptr(sv_state *s) { return s ? s->amp : nullptr; }

int sv_reset(sv_state *s, uint64_t basis_index) {
  CHECK_STATE(s);
  if (basis_index >> s->n) return fail(SV_ERR_ARG, "basis index out of range");
  DeviceGuard g(s->device);
  CK(s, timed(s, "reset", double(size_t(8) << s->n),
              [&] { return launch_reset(s->amp, s->n, basis_index, s->stream); }));
  return SV_OK;
}

int sv_plan_stats(int n_qubits, const sv_gate *ir, size_t n_gates, const sv_opts *opts,
                  sv_plan_info *out) {
  if (!out) return fail(SV_ERR_ARG, "out is null");
  if (n_qubits < 1 || n_qubits > 36) return fail(SV_ERR_ARG, "n_qubits must be in [1,36]");
  if (n_gates && !ir) return fail(SV_ERR_ARG, "ir is null");
  Plan plan;
  std::string err;
  if (!build_plan(n_qubits, ir, n_gates, opts, plan, err)) return fail(SV_ERR_ARG, "%s", err.c_str());
  *out = plan.info;
  return SV_OK;
}

// A plan slab of at least `bytes` whose previous chunk has finished (index into s->slabs).
static int acquire_slab(sv_state *s, size_t bytes, size_t *idx) {
  for (size_t i = 0; i < s->slabs.size(); i++) {
    PlanSlab &sl = s->slabs[i];
    if (sl.cap < bytes) continue;
    if (sl.live) {
      const cudaError_t q = cudaEventQuery(sl.done);
      if (q == cudaErrorNotReady) continue;
      if (q != cudaSuccess) return cuda_fail(s, q, "plan slab event");
      sl.live = false;
    }
    *idx = i;
    return SV_OK;
  }
  PlanSlab sl;
  sl.cap = std::max<size_t>(size_t(64) << 10, (bytes + 4095) & ~size_t(4095));
  cudaError_t e = cudaMallocHost(&sl.host, sl.cap);
  if (e == cudaSuccess) e = cudaMalloc(&sl.dev, sl.cap);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    if (sl.host) cudaFreeHost(sl.host);
    if (sl.dev) cudaFree(sl.dev);
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? SV_ERR_OOM : SV_ERR_CUDA, "plan slab: %s", cudaGetErrorString(e));
  }
  s->slabs.push_back(sl);
  *idx = s->slabs.size() - 1;
  return SV_OK;
}

// Plans in chunks of 2, 4, 8, ... passes: each chunk is uploaded and its passes
// launched before the next chunk is planned, so the GPU starts on the first
// passes while the host plans the rest.
int sv_apply_circuit(sv_state *s, const sv_gate *ir, size_t n_gates, const sv_opts *opts) {
  CHECK_STATE(s);
  if (n_gates == 0) return SV_OK;
  if (!ir) return fail(SV_ERR_ARG, "ir is null");
  PlanBuilder builder;
  std::string err;
  if (!builder.init(s->n, ir, n_gates, opts, err)) return fail(SV_ERR_ARG, "%s", err.c_str());
  DeviceGuard g(s->device);
  {
    int rc = ensure_scalars(s);
    if (rc) return rc;
  }
  const double pass_bytes = 16.0 * double(uint64_t(1) << s->n);
  // Tensor-core passes shrink the norm by ~1e-7 per stage (float32 accumulation
  // rounding toward zero); a unitary circuit keeps ||psi||^2, so its passes track
  // the norm (TcNorm): dscal[4] takes the first tensor-core pass's input sum,
  // dscal[5..7] the output sums of successive tensor-core passes in rotation, and
  // each later pass rescales what it loads by sqrt(dscal[4] / previous sum).
  const bool track = opts && opts->precision >= 1 && builder.unitary() && s->n >= 11;
  if (track) CK(s, cudaMemsetAsync(s->dscal + 4, 0, 2 * sizeof(double), s->stream));
  size_t n_tc = 0;
  size_t chunk = 2;
  while (!builder.done()) {
    Plan plan;
    if (!builder.next(plan, chunk, err)) return fail(SV_ERR_ARG, "%s", err.c_str());
    chunk = std::min<size_t>(chunk * 2, 64);
    const size_t bytes = plan.bytes.size();
    size_t si = 0;
    int rc = acquire_slab(s, bytes, &si);
    if (rc) return rc;
    PlanSlab &sl = s->slabs[si];
    std::memcpy(sl.host, plan.bytes.data(), bytes);
    CK(s, cudaMemcpyAsync(sl.dev, sl.host, bytes, cudaMemcpyHostToDevice, s->stream));
    for (size_t p = 0; p < plan.passes.size(); p++) {
      const bool tc = plan.passes[p].kind == KIND_TC;
      TcNorm nrm;
      if (tc && track) {
        double *slot = s->dscal + 5;
        if (n_tc == 0) {
          nrm.in_sum = s->dscal + 4;
        } else {
          nrm.ref = s->dscal + 4;
          nrm.prev = slot + (n_tc - 1) % 3;
        }
        nrm.out_sum = slot + n_tc % 3;      // zeroed by the memset or the previous pass
        nrm.clear = slot + (n_tc + 1) % 3;  // read by the previous pass, summed into by the next
        n_tc++;
      }
      const char *kname = tc ? "pass_tc" : "pass";
      CK(s, timed(s, kname, pass_bytes, [&] {
           return launch_pass(s->amp, sl.dev, plan.pass_offs[p], plan.passes[p], &plan.rparams[p], s->derr,
                              s->stream, &nrm);
         }));
    }
    CK(s, cudaEventRecord(sl.done, s->stream));
    sl.live = true;
  }
  return SV_OK;
}

int sv_norm(sv_state *s, double *out_norm2) {
  CHECK_STATE(s);
  if (!out_norm2) return fail(SV_ERR_ARG, "out is null");
  DeviceGuard g(s->device);
  int rc = ensure_reduce(s);
  if (rc) return rc;
  CK(s, timed(s, "reduce", double(size_t(8) << s->n), [&] {
       return launch_reduce_pz(s->amp, s->n, 0, s->ms.part, s->ms.n_part, s->dscal, s->stream);
     }));
  CK(s, cudaMemcpyAsync(s->hscal, s->dscal, 2 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  CK(s, cudaStreamSynchronize(s->stream));
  rc = check_device_error(s);
  if (rc) return rc;
  *out_norm2 = s->hscal[0];
  return SV_OK;
}

int sv_expect_pauli(sv_state *s, uint64_t x_mask, uint64_t z_mask, double *out) {
  CHECK_STATE(s);
  if (!out) return fail(SV_ERR_ARG, "out is null");
  if ((x_mask | z_mask) >> s->n) return fail(SV_ERR_ARG, "mask has bits beyond n_qubits");
  DeviceGuard g(s->device);
  int rc = ensure_reduce(s);
  if (rc) return rc;
  if (x_mask) {
    CK(s, timed(s, "reduce", double(size_t(8) << s->n), [&] {
         return launch_reduce_pauli(s->amp, s->n, x_mask, z_mask, s->ms.part, s->ms.n_part, s->dscal,
                                    s->stream);
       }));
  } else {
    CK(s, timed(s, "reduce", double(size_t(8) << s->n), [&] {
         return launch_reduce_pz(s->amp, s->n, z_mask, s->ms.part, s->ms.n_part, s->dscal, s->stream);
       }));
  }
  CK(s, cudaMemcpyAsync(s->hscal, s->dscal, 2 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  CK(s, cudaStreamSynchronize(s->stream));
  rc = check_device_error(s);
  if (rc) return rc;
  if (!(s->hscal[0] > 0.0)) return fail(SV_ERR_ARG, "state has zero norm");
  *out = (x_mask ? 2.0 * s->hscal[1] : s->hscal[1]) / s->hscal[0];
  return SV_OK;
}

// Masses of qubit q's two outcomes: m0 = sum p_i over bit q = 0, m1 over bit q = 1
// (one FP64 reduction of p and p * (-1)^bit; synchronises).
static int qubit_masses(sv_state *s, int q, double *m0, double *m1) {
  int rc = ensure_reduce(s);
  if (rc) return rc;
  const uint64_t zmask = uint64_t(1) << q;
  CK(s, timed(s, "reduce", double(size_t(8) << s->n), [&] {
       return launch_reduce_pz(s->amp, s->n, zmask, s->ms.part, s->ms.n_part, s->dscal, s->stream);
     }));
  CK(s, cudaMemcpyAsync(s->hscal, s->dscal, 2 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  CK(s, cudaStreamSynchronize(s->stream));
  rc = check_device_error(s);
  if (rc) return rc;
  const double total = s->hscal[0], z = s->hscal[1];
  *m0 = std::max(0.0, 0.5 * (total + z));
  *m1 = std::max(0.0, 0.5 * (total - z));
  return SV_OK;
}

static int measure_common(sv_state *s, int qubit, double u, int to_zero, int *outcome, double *prob) {
  CHECK_STATE(s);
  if (!outcome) return fail(SV_ERR_ARG, "outcome is null");
  if (qubit < 0 || qubit >= s->n) return fail(SV_ERR_ARG, "qubit %d out of range [0,%d)", qubit, s->n);
  if (!(u >= 0.0 && u < 1.0)) return fail(SV_ERR_ARG, "u must be in [0,1)");
  DeviceGuard g(s->device);
  double m0 = 0.0, m1 = 0.0;
  int rc = qubit_masses(s, qubit, &m0, &m1);
  if (rc) return rc;
  const double total = m0 + m1;
  if (!(total > 0.0)) return fail(SV_ERR_ARG, "state has zero norm");
  int b = (u * total < m0) ? 0 : 1;
  double m = b ? m1 : m0;
  if (!(m > 0.0)) {  // rounding left the drawn outcome without mass
    b ^= 1;
    m = b ? m1 : m0;
  }
  const float scale = float(1.0 / std::sqrt(m));
  CK(s, timed(s, "collapse", double(size_t(16) << s->n), [&] {
       return launch_collapse(s->amp, s->n, qubit, b, to_zero && b, scale, s->stream);
     }));
  *outcome = b;
  if (prob) *prob = m / total;
  return SV_OK;
}

int sv_measure_qubit(sv_state *s, int qubit, double u, int *outcome, double *prob) {
  return measure_common(s, qubit, u, 0, outcome, prob);
}

int sv_reset_qubit(sv_state *s, int qubit, double u, int *outcome) {
  return measure_common(s, qubit, u, 1, outcome, nullptr);
}

// Orders `dst`'s stream after all work queued on `src`'s stream.

int sv_clone(sv_state *src, void *cuda_stream, sv_state **out) {
  CHECK_STATE(src);
  if (!out) return fail(SV_ERR_ARG, "out is null");
  DeviceGuard g(src->device);
  int rc = create_state(src->n, SV_C64, cuda_stream, false, out);
  if (rc) return rc;
  sv_state *d = *out;
  const size_t bytes = (size_t(1) << src->n) * sizeof(float2);
  cudaError_t e = stream_after(d->stream, src->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d->amp, src->amp, bytes, cudaMemcpyDeviceToDevice, d->stream);
  // later work on the source (an apply that overwrites it, or its destroy) waits
  // for the copy that reads it on the clone's stream
  if (e == cudaSuccess) e = stream_after(src->stream, d->stream);
  if (e != cudaSuccess) {
    free_state(d);
    *out = nullptr;
    return fail(SV_ERR_CUDA, "clone: %s", cudaGetErrorString(e));
  }
  return SV_OK;
}

int sv_merge(sv_state *a, sv_state *b, void *cuda_stream, sv_state **out) {
  CHECK_STATE(a);
  CHECK_STATE(b);
  if (!out) return fail(SV_ERR_ARG, "out is null");
  if (a->device != b->device) return fail(SV_ERR_ARG, "registers live on different devices");
  if (a->n + b->n > 36) return fail(SV_ERR_ARG, "merged register would exceed 36 qubits");
  DeviceGuard g(a->device);
  int rc = create_state(a->n + b->n, SV_C64, cuda_stream, false, out);
  if (rc) return rc;
  sv_state *d = *out;
  cudaError_t e = stream_after(d->stream, a->stream);
  if (e == cudaSuccess) e = stream_after(d->stream, b->stream);
  if (e == cudaSuccess)
    e = timed(d, "merge", double(size_t(8) << d->n),
              [&] { return launch_kron(a->amp, a->n, b->amp, b->n, d->amp, d->stream); });
  // later work on either source waits for the merge that reads it
  if (e == cudaSuccess) e = stream_after(a->stream, d->stream);
  if (e == cudaSuccess) e = stream_after(b->stream, d->stream);
  if (e != cudaSuccess) {
    free_state(d);
    *out = nullptr;
    return fail(SV_ERR_CUDA, "merge: %s", cudaGetErrorString(e));
  }
  return SV_OK;
}

int sv_take_qubit(sv_state *s, int qubit, double tol, int *value, sv_state **out) {
  CHECK_STATE(s);
  if (!out || !value) return fail(SV_ERR_ARG, "out/value is null");
  if (s->n < 2) return fail(SV_ERR_ARG, "a register keeps at least one qubit");
  if (qubit < 0 || qubit >= s->n) return fail(SV_ERR_ARG, "qubit %d out of range [0,%d)", qubit, s->n);
  if (!(tol >= 0.0 && tol < 0.5)) return fail(SV_ERR_ARG, "tol must be in [0, 0.5)");
  DeviceGuard g(s->device);
  double m0 = 0.0, m1 = 0.0;
  int rc = qubit_masses(s, qubit, &m0, &m1);
  if (rc) return rc;
  const double total = m0 + m1;
  if (!(total > 0.0)) return fail(SV_ERR_ARG, "state has zero norm");
  const int v = (m1 > m0) ? 1 : 0;
  if ((v ? m0 : m1) > tol * total)
    return fail(SV_ERR_ARG, "qubit %d is not in a basis state (minority mass %.3g of %.3g)", qubit,
                v ? m0 : m1, total);
  rc = create_state(s->n - 1, SV_C64, s->stream, false, out);
  if (rc) return rc;
  sv_state *d = *out;
  cudaError_t e = timed(d, "take", double(size_t(8) << s->n),
                        [&] { return launch_take(s->amp, s->n, qubit, v, d->amp, d->stream); });
  if (e != cudaSuccess) {
    free_state(d);
    *out = nullptr;
    return fail(SV_ERR_CUDA, "take: %s", cudaGetErrorString(e));
  }
  *value = v;
  return SV_OK;
}

int sv_probabilities(sv_state *s, double *out, uint64_t offset, uint64_t count, int out_on_device) {
  CHECK_STATE(s);
  const uint64_t N = uint64_t(1) << s->n;
  if (offset > N || count > N - offset) return fail(SV_ERR_ARG, "range beyond the state");
  if (count == 0) return SV_OK;
  if (!out) return fail(SV_ERR_ARG, "out is null");
  DeviceGuard g(s->device);
  if (out_on_device) {
    CK(s, timed(s, "probabilities", 16.0 * double(count),
                [&] { return launch_probabilities(s->amp, offset, count, out, s->stream); }));
    return SV_OK;
  }
  const uint64_t step = uint64_t(1) << 22;
  int rc = ensure_dev(s, &s->stage, &s->stage_cap, step * sizeof(double), "staging buffer");
  if (rc) return rc;
  for (uint64_t o = 0; o < count; o += step) {
    const uint64_t c = (count - o < step) ? count - o : step;
    CK(s, launch_probabilities(s->amp, offset + o, c, static_cast<double *>(s->stage), s->stream));
    CK(s, cudaMemcpyAsync(out + o, s->stage, c * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    CK(s, cudaStreamSynchronize(s->stream));
  }
  return SV_OK;
}

int sv_get_amplitudes(sv_state *s, void *out, uint64_t offset, uint64_t count, int out_on_device) {
  CHECK_STATE(s);
  const uint64_t N = uint64_t(1) << s->n;
  if (offset > N || count > N - offset) return fail(SV_ERR_ARG, "range beyond the state");
  if (count == 0) return SV_OK;
  if (!out) return fail(SV_ERR_ARG, "out is null");
  DeviceGuard g(s->device);
  CK(s, cudaMemcpyAsync(out, s->amp + offset, count * sizeof(float2),
                        out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s->stream));
  if (!out_on_device) {
    CK(s, cudaStreamSynchronize(s->stream));
    return check_device_error(s);
  }
  return SV_OK;
}

int sv_set_amplitudes(sv_state *s, const void *in, uint64_t offset, uint64_t count, int in_on_device) {
  CHECK_STATE(s);
  const uint64_t N = uint64_t(1) << s->n;
  if (offset > N || count > N - offset) return fail(SV_ERR_ARG, "range beyond the state");
  if (count == 0) return SV_OK;
  if (!in) return fail(SV_ERR_ARG, "in is null");
  DeviceGuard g(s->device);
  CK(s, cudaMemcpyAsync(s->amp + offset, in, count * sizeof(float2),
                        in_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s->stream));
  if (!in_on_device) CK(s, cudaStreamSynchronize(s->stream));
  return SV_OK;
}

// With obs (non-null), the CDF build also forms sum p (-1)^popcount(i & zmask)
// from the same read: obs[0] = <Z_mask>, obs[1] = ||psi||^2 (the CDF total).
static int sample_impl(sv_state *s, const double *u, uint64_t seed, int use_seed, uint64_t shots,
                       uint64_t *out, uint64_t *out_nb, int on_device, uint64_t zmask = 0,
                       double *obs = nullptr) {
  CHECK_STATE(s);
  if (shots == 0 && !obs) {
    if (out_nb) *out_nb = 0;
    return SV_OK;
  }
  if (shots && !out) return fail(SV_ERR_ARG, "out is null");
  if (shots && !use_seed && !u) return fail(SV_ERR_ARG, "uniforms is null");
  if (obs && (zmask >> s->n)) return fail(SV_ERR_ARG, "z_mask has bits beyond n_qubits");
  DeviceGuard g(s->device);
  int rc = ensure_cdf(s);
  if (rc) return rc;
  const double nbytes = double(size_t(8) << s->n);
  CK(s, timed(s, "cdf", nbytes, [&] {
       return launch_build_cdf(s->amp, s->n, s->ms, s->dscal + 2, s->stream, zmask, obs ? s->dscal + 3 : nullptr);
     }));
  if (shots == 0) {  // readout of <Z_mask> and the norm only
    CK(s, cudaMemcpyAsync(s->hscal + 2, s->dscal + 2, 2 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    CK(s, cudaStreamSynchronize(s->stream));
    rc = check_device_error(s);
    if (rc) return rc;
    if (!(s->hscal[2] > 0.0)) return fail(SV_ERR_ARG, "state has zero norm");
    obs[0] = s->hscal[3] / s->hscal[2];
    obs[1] = s->hscal[2];
    if (out_nb) *out_nb = 0;
    return SV_OK;
  }
  const double *u_dev = u;
  uint64_t *out_dev = out;
  if (!on_device) {
    const size_t need = shots * (sizeof(uint64_t) + (use_seed ? 0 : sizeof(double)));
    rc = ensure_dev(s, &s->stage, &s->stage_cap, need, "staging buffer");
    if (rc) return rc;
    out_dev = static_cast<uint64_t *>(s->stage);
    if (!use_seed) {
      double *ud = reinterpret_cast<double *>(out_dev + shots);
      CK(s, cudaMemcpyAsync(ud, u, shots * sizeof(double), cudaMemcpyHostToDevice, s->stream));
      u_dev = ud;
    }
  }
  CK(s, cudaMemsetAsync(s->dcount, 0, sizeof(uint64_t), s->stream));
  CK(s, timed(s, "sample", 0.0, [&] {
       return launch_sample(s->amp, s->n, s->ms, s->dscal + 2, u_dev, seed, use_seed, shots, out_dev,
                            s->dcount, s->stream);
     }));
  if (!on_device)
    CK(s, cudaMemcpyAsync(out, out_dev, shots * sizeof(uint64_t), cudaMemcpyDeviceToHost, s->stream));
  if (out_nb || !on_device || obs) {
    CK(s, cudaMemcpyAsync(s->hscal, s->dcount, sizeof(uint64_t), cudaMemcpyDeviceToHost, s->stream));
    if (obs) CK(s, cudaMemcpyAsync(s->hscal + 2, s->dscal + 2, 2 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    CK(s, cudaStreamSynchronize(s->stream));
    uint64_t nb;
    std::memcpy(&nb, s->hscal, sizeof(nb));
    if (out_nb) *out_nb = nb;
    rc = check_device_error(s);
    if (rc) return rc;
    if (obs) {
      if (!(s->hscal[2] > 0.0)) return fail(SV_ERR_ARG, "state has zero norm");
      obs[0] = s->hscal[3] / s->hscal[2];
      obs[1] = s->hscal[2];
    }
    return SV_OK;
  }
  return SV_OK;
}

int sv_sample(sv_state *s, uint64_t shots, uint64_t seed, uint64_t *out_bitstrings, int on_device) {
  return sample_impl(s, nullptr, seed, 1, shots, out_bitstrings, nullptr, on_device);
}

int sv_sample_uniforms(sv_state *s, const double *uniforms, uint64_t shots, uint64_t *out_bitstrings,
                       uint64_t *out_n_boundary, int on_device) {
  return sample_impl(s, uniforms, 0, 0, shots, out_bitstrings, out_n_boundary, on_device);
}

int sv_sample_expect_z(sv_state *s, const double *uniforms, uint64_t shots, uint64_t *out_bitstrings,
                       uint64_t *out_n_boundary, int on_device, uint64_t z_mask, double *out_expect,
                       double *out_norm2) {
  if (!out_expect || !out_norm2) return fail(SV_ERR_ARG, "out_expect and out_norm2 are required");
  double obs[2] = {0.0, 0.0};
  const int rc = sample_impl(s, uniforms, 0, 0, shots, out_bitstrings, out_n_boundary, on_device, z_mask, obs);
  if (rc == SV_OK) {
    *out_expect = obs[0];
    *out_norm2 = obs[1];
  }
  return rc;
}

int sv_alias_release(sv_state *s) {
  if (!s) return fail(SV_ERR_ARG, "null state");
  DeviceGuard g(s->device);
  if (s->alias_table) {
    CK(s, cudaStreamSynchronize(s->stream));
    cudaFree(s->alias_table);
    s->alias_table = nullptr;
  }
  s->alias_n = 0;
  return SV_OK;
}

int sv_alias_build(sv_state *s) {
  CHECK_STATE(s);
  if (s->n > 32) return fail(SV_ERR_UNSUPPORTED, "alias tables hold 32-bit outcomes: n <= 32, got %d", s->n);
  DeviceGuard g(s->device);
  int rc = ensure_reduce(s);
  if (rc) return rc;
  const uint64_t N = uint64_t(1) << s->n;
  CK(s, timed(s, "reduce", double(N * 8), [&] {
       return launch_reduce_pz(s->amp, s->n, 0, s->ms.part, s->ms.n_part, s->dscal, s->stream);
     }));
  CK(s, cudaMemcpyAsync(s->hscal, s->dscal, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  CK(s, cudaStreamSynchronize(s->stream));
  rc = check_device_error(s);
  if (rc) return rc;
  const double W = s->hscal[0];
  if (!(W > 0.0) || !std::isfinite(W)) return fail(SV_ERR_ARG, "state weight %g: nothing to sample", W);
  const double scale = double(N) / W;
  const float s_hi = float(scale), s_lo = float(scale - double(s_hi));
  if (s->alias_table && s->alias_n != s->n) {
    cudaFree(s->alias_table);
    s->alias_table = nullptr;
  }
  if (!s->alias_table) CK(s, cudaMalloc(&s->alias_table, N * sizeof(uint64_t)));
  s->alias_n = 0;
  if (!s->alias_tot) CK(s, cudaMalloc(&s->alias_tot, 4 * sizeof(uint64_t)));
  AliasScratch sc;
  sc.tot = s->alias_tot;
  const size_t nblk = alias_blocks(s->n), nseg = alias_segments(s->n), nsplit = alias_splits(s->n);
  void *mem = nullptr;
  const size_t off_seg = 3 * nblk * sizeof(uint64_t);
  const size_t off_split = off_seg + 3 * nseg * sizeof(uint64_t);
  const size_t off_keys = (off_split + nsplit * sizeof(uint64_t) + 255) & ~size_t(255);
  const size_t off_qv = off_keys + N * sizeof(uint64_t);
  const size_t off_idx = off_qv + N * sizeof(uint32_t);
  const size_t bytes = off_idx + N * sizeof(uint32_t);
  CK(s, cudaMallocAsync(&mem, bytes, s->stream));
  uint8_t *base = static_cast<uint8_t *>(mem);
  sc.blk = reinterpret_cast<uint64_t *>(base);
  sc.seg = reinterpret_cast<uint64_t *>(base + off_seg);
  sc.splits = reinterpret_cast<uint64_t *>(base + off_split);
  sc.keys = reinterpret_cast<uint64_t *>(base + off_keys);
  sc.qv = reinterpret_cast<uint32_t *>(base + off_qv);
  sc.idx = reinterpret_cast<uint32_t *>(base + off_idx);
  cudaError_t e = timed(s, "alias_build", double(N) * 60.0,
                        [&] { return launch_alias_build(s->amp, s->n, s_hi, s_lo, sc, s->alias_table, s->stream); });
  cudaError_t e2 = cudaFreeAsync(mem, s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "alias table build");
  if (e2 != cudaSuccess) return cuda_fail(s, e2, "alias scratch release");
  uint64_t tot[4];
  CK(s, cudaMemcpyAsync(s->hscal, s->alias_tot, 4 * sizeof(uint64_t), cudaMemcpyDeviceToHost, s->stream));
  CK(s, cudaStreamSynchronize(s->stream));
  std::memcpy(tot, s->hscal, sizeof(tot));
  if (tot[3] || tot[0] >= N) return fail(SV_ERR_ARG, "no outcome reaches a full bucket: state weight too small");
  if (s->prof && !s->recs.empty() && std::strcmp(s->recs.back().name, "alias_build") == 0)
    // two state reads, list records written and read (12 B, +4 B of weight for light
    // outcomes), one table entry
    s->recs.back().bytes = double(N) * (16 + 24 + 8) + double(tot[0]) * 8;
  s->alias_n = s->n;
  return SV_OK;
}

static int alias_sample_impl(sv_state *s, const double *u, uint64_t seed, int use_seed, uint64_t shots,
                             uint64_t *out, int on_device) {
  CHECK_STATE(s);
  if (!s->alias_table || s->alias_n != s->n) return fail(SV_ERR_ARG, "no alias table: call sv_alias_build first");
  if (shots == 0) return SV_OK;
  if (!out) return fail(SV_ERR_ARG, "out is null");
  if (!use_seed && !u) return fail(SV_ERR_ARG, "uniforms is null");
  DeviceGuard g(s->device);
  const double *u_dev = u;
  uint64_t *out_dev = out;
  if (!on_device) {
    const size_t need = shots * (sizeof(uint64_t) + (use_seed ? 0 : sizeof(double)));
    int rc = ensure_dev(s, &s->stage, &s->stage_cap, need, "staging buffer");
    if (rc) return rc;
    out_dev = static_cast<uint64_t *>(s->stage);
    if (!use_seed) {
      double *ud = reinterpret_cast<double *>(out_dev + shots);
      CK(s, cudaMemcpyAsync(ud, u, shots * sizeof(double), cudaMemcpyHostToDevice, s->stream));
      u_dev = ud;
    }
  }
  CK(s, timed(s, "alias_sample", double(shots) * 16.0, [&] {
       return launch_alias_sample(s->alias_table, s->n, u_dev, seed, use_seed, shots, out_dev, s->stream);
     }));
  if (!on_device) {
    CK(s, cudaMemcpyAsync(out, out_dev, shots * sizeof(uint64_t), cudaMemcpyDeviceToHost, s->stream));
    CK(s, cudaStreamSynchronize(s->stream));
    return check_device_error(s);
  }
  return SV_OK;
}

int sv_alias_sample(sv_state *s, uint64_t shots, uint64_t seed, uint64_t *out_bitstrings, int on_device) {
  return alias_sample_impl(s, nullptr, seed, 1, shots, out_bitstrings, on_device);
}

int sv_alias_sample_uniforms(sv_state *s, const double *uniforms, uint64_t shots, uint64_t *out_bitstrings,
                             int on_device) {
  return alias_sample_impl(s, uniforms, 0, 0, shots, out_bitstrings, on_device);
}

int sv_alias_table(sv_state *s, uint64_t *out, uint64_t offset, uint64_t count, int on_device) {
  CHECK_STATE(s);
  if (!s->alias_table || s->alias_n != s->n) return fail(SV_ERR_ARG, "no alias table: call sv_alias_build first");
  const uint64_t N = uint64_t(1) << s->n;
  if (offset > N || count > N - offset) return fail(SV_ERR_ARG, "range beyond the table");
  if (count == 0) return SV_OK;
  if (!out) return fail(SV_ERR_ARG, "out is null");
  DeviceGuard g(s->device);
  CK(s, cudaMemcpyAsync(out, s->alias_table + offset, count * sizeof(uint64_t),
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s->stream));
  if (!on_device) CK(s, cudaStreamSynchronize(s->stream));
  return SV_OK;
}

int sv_tc_selftest_r(int r, const float *a, const double *b, float *d) {
  if (r != 4 && r != 5) return fail(SV_ERR_ARG, "r must be 4 or 5");
  if (!a || !b || !d) return fail(SV_ERR_ARG, "null argument");
  int status = 0;
  cudaError_t e = tc_selftest(r, a, b, d, &status);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "tensor-core self-test");
  if (status) return fail(SV_ERR_TIMEOUT, "tensor-core self-test: the MMA completion wait gave up");
  return SV_OK;
}

int sv_tc_selftest(const float *a, const double *b, float *d) { return sv_tc_selftest_r(4, a, b, d); }

int sv_diag_bounded_wait(int limit_ms) {
  if (limit_ms < 1 || limit_ms > 10000) return fail(SV_ERR_ARG, "limit_ms must be in [1, 10000]");
  int status = -1;
  cudaError_t e = wait_nothing(uint32_t(limit_ms), &status);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "bounded-wait check");
  if (status == 1) return fail(SV_ERR_TIMEOUT, "bounded wait gave up after %d ms (nothing arrived)", limit_ms);
  return fail(SV_ERR_CUDA, "bounded-wait check: unexpected status %d", status);
}

int sv_profile_enable(sv_state *s, int on) {
  if (!s) return fail(SV_ERR_ARG, "null state");
  s->prof = on != 0;
  return SV_OK;
}

int sv_profile_read(sv_state *s, sv_kernel_stat *out, int cap, int *n_out) {
  CHECK_STATE(s);
  DeviceGuard g(s->device);
  CK(s, cudaStreamSynchronize(s->stream));
  std::map<std::string, sv_kernel_stat> agg;
  std::vector<std::string> order;
  for (auto &r : s->recs) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    auto it = agg.find(r.name);
    if (it == agg.end()) {
      sv_kernel_stat st{};
      std::snprintf(st.name, sizeof(st.name), "%s", r.name);
      it = agg.emplace(r.name, st).first;
      order.push_back(r.name);
    }
    it->second.launches++;
    it->second.ms += ms;
    it->second.bytes += r.bytes;
    s->evpool.push_back(r.a);
    s->evpool.push_back(r.b);
  }
  s->recs.clear();
  int k = 0;
  for (auto &nm : order) {
    if (k < cap && out) out[k] = agg[nm];
    k++;
  }
  if (n_out) *n_out = k;
  return SV_OK;
}

}  // extern "C"
