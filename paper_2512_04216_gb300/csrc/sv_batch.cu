// sv_batch.cu -- many small circuits in one persistent launch (batched mode).
//
// The paper runs heterogeneous batches of circuits and notes that GPU
// simulation loses to the CPU on small or batched workloads when every
// circuit pays its own launches and transfers (§II, §IV-B).  Here a whole batch
// of independent circuits (10-20 qubits in the reference workload) runs in ONE
// persistent kernel, captured once in a CUDA graph and replayed:
//
//  * circuits are planned on the host with the same fusion/pass planner as
//    sv_apply_circuit (shared-memory sweep ops, k_max <= 3);
//  * each CTA takes whole circuits from an atomic work counter, largest first;
//  * a state of n <= 13 qubits (<= 64 KiB of complex64) lives in the CTA's
//    shared memory for the whole circuit -- it is never read from or written to
//    HBM; larger states live in a global arena and the CTA sweeps it tile by
//    tile once per pass (no other CTA touches the circuit, so no grid sync);
//  * the CTA then measures: chunk sums of |a|^2 in double, an inclusive double
//    prefix over chunks, and for every shot (counter-based SplitMix64 uniform
//    from the circuit's seed) the first index whose running sum exceeds
//    u * total -- the same rule as sv_sample.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/sv.h"
#include "sv_device.cuh"
#include "sv_internal.h"
#include "sv_plan.h"
#include "sv_regpass.cuh"

namespace svgb {

constexpr int kBatchNT = 256;
constexpr int kBatchSmemQubits = 13;  // states up to this size stay in shared memory
constexpr int kBatchMaxQubits = 24;
constexpr int kBatchMaxK = 3;
// Arena states (more than kBatchSmemQubits qubits) planned with tiles of
// kBatchRegT qubits run register-stage passes (16 amplitudes a thread, 256
// threads = 2^(kBatchRegT - 4)) in this much of the CTA's shared memory.
constexpr int kBatchRegT = 12;
constexpr size_t kBatchRegSmem = 96 * 1024;
// Largest register pass (records and tables) the batched kernel runs.
__host__ __device__ inline bool batch_reg_fits(uint32_t c, uint32_t ns, uint32_t data_bytes) {
  return ns >= 1 && ns <= uint32_t(kMaxStages) &&
         reg_layout(kBatchRegT, c, ns, data_bytes, 4, true).total + sizeof(RegPassParams) <= kBatchRegSmem;
}

struct alignas(16) BatchCirc {
  uint64_t plan_off;     // byte offset of the circuit's plan in the plan buffer
  uint64_t state_off;    // float2 offset in the arena (global-state circuits, or kept states)
  uint64_t scratch_off;  // double offset of the chunk-prefix array (global-state circuits)
  uint64_t out_off;      // uint64 offset of the circuit's samples
  uint64_t seed;
  uint64_t zmask;        // flags bit 1: <Z_zmask> and the norm go to ex[2 * slot]
  uint32_t n, n_passes, shots, flags;  // flags bit 0: copy the final state to the arena
};
static_assert(sizeof(BatchCirc) == 64, "BatchCirc layout");

struct BatchLayout {
  size_t off_tile, off_seg, off_mat, off_tab, off_acc, off_chunk, off_tot, total;
};
__host__ __device__ inline BatchLayout batch_layout(int kmax) {
  BatchLayout L;
  size_t o = 0;
  L.off_tile = o; o += (size_t(1) << kBatchSmemQubits) * 8;
  L.off_seg = o; o += 256 * 8;
  L.off_mat = o; o += (size_t(1) << (2 * kmax)) * 8;
  L.off_tab = o; o += 256 * 8;
  L.off_acc = o; o += 64 * 4;
  L.off_chunk = o; o += (size_t(1) << (kBatchSmemQubits - 6)) * 8;
  L.off_tot = o; o += kBatchNT * 8;
  L.total = (o + 15) & ~size_t(15);
  if (L.total < kBatchRegSmem) L.total = kBatchRegSmem;  // the arena's register passes use the same space
  return L;
}

__device__ __forceinline__ double p_of(float2 a) {
  const double re = a.x, im = a.y;
  return fma(re, re, im * im);
}

// Chunk sums, inclusive prefix, and shots for one state (CTA-wide).
__device__ void batch_measure(const float2 *amps, uint32_t n, uint64_t seed, uint32_t shots, uint64_t *out,
                              double *chunk, double *tot) {
  const uint32_t N = 1u << n;
  const uint32_t cs = N < 64 ? N : 64;
  const uint32_t nch = N / cs;
  for (uint32_t c = threadIdx.x; c < nch; c += blockDim.x) {
    double s = 0.0;
    for (uint32_t i = 0; i < cs; i++) s += p_of(amps[c * cs + i]);
    chunk[c] = s;
  }
  __syncthreads();
  // inclusive scan: contiguous segments per thread, then the segment totals
  const uint32_t seg = (nch + blockDim.x - 1) / blockDim.x;
  const uint32_t b0 = threadIdx.x * seg, b1 = min(b0 + seg, nch);
  double run = 0.0;
  for (uint32_t c = b0; c < b1; c++) {
    run += chunk[c];
    chunk[c] = run;
  }
  tot[threadIdx.x] = run;
  __syncthreads();
  if (threadIdx.x == 0) {
    double acc = 0.0;
    for (uint32_t t = 0; t < blockDim.x; t++) {
      const double v = tot[t];
      tot[t] = acc;
      acc += v;
    }
  }
  __syncthreads();
  const double off = tot[threadIdx.x];
  for (uint32_t c = b0; c < b1; c++) chunk[c] += off;
  __syncthreads();
  const double total = chunk[nch - 1];
  for (uint32_t s = threadIdx.x; s < shots; s += blockDim.x) {
    const double t = splitmix_uniform(seed, s) * total;
    uint32_t lo = 0, hi = nch;
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (chunk[mid] > t) hi = mid; else lo = mid + 1;
    }
    uint32_t c = lo < nch ? lo : nch - 1;
    if (lo == nch)
      while (c > 0 && !(chunk[c] > chunk[c - 1])) c--;
    double acc = c ? chunk[c - 1] : 0.0;
    uint32_t x = c * cs + cs, x_last = c * cs;
    for (uint32_t i = c * cs; i < c * cs + cs; i++) {
      const double p = p_of(amps[i]);
      if (p > 0.0) x_last = i;
      if (acc + p > t) {
        x = i;
        break;
      }
      acc += p;
    }
    out[s] = (x == c * cs + cs) ? x_last : x;
  }
  __syncthreads();
}

// sum p and sum p (-1)^popcount(i & zmask) over a state, double, CTA-wide;
// thread 0 writes {<Z>, norm} to ex.
__device__ void batch_expect(const float2 *amps, uint32_t n, uint64_t zmask, double *ex, double *tot) {
  const uint32_t N = 1u << n;
  double p = 0.0, pz = 0.0;
  for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) {
    const double q = p_of(amps[i]);
    p += q;
    pz += (__popcll(uint64_t(i) & zmask) & 1) ? -q : q;
  }
  __syncthreads();
  tot[threadIdx.x] = p;
  __syncthreads();
  double sp = 0.0;
  if (threadIdx.x == 0)
    for (uint32_t t = 0; t < blockDim.x; t++) sp += tot[t];
  __syncthreads();
  tot[threadIdx.x] = pz;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sz = 0.0;
    for (uint32_t t = 0; t < blockDim.x; t++) sz += tot[t];
    ex[0] = sp > 0.0 ? sz / sp : 0.0;
    ex[1] = sp;
  }
  __syncthreads();
}

// Whether a circuit's pass records and their ops stay inside the plan buffer
// and the kernel's shared-memory layout (the host builds them that way; this
// guards the launch against a corrupted buffer: the circuit is skipped and the
// error word set instead of indexing out of range).
template <int KMAX>
__device__ __forceinline__ bool batch_plan_ok(const uint8_t *plans, uint64_t plans_size, const BatchCirc &C) {
  if (C.n < 1 || C.n > uint32_t(kBatchMaxQubits)) return false;
  if (C.plan_off + uint64_t(C.n_passes) * sizeof(PlanPass) > plans_size) return false;
  const uint8_t *plan = plans + C.plan_off;
  for (uint32_t p = 0; p < C.n_passes; p++) {
    const PlanPass P = reinterpret_cast<const PlanPass *>(plan)[p];
    if (P.kind == KIND_REG) {  // arena register pass: the checks k_pass_reg makes, and the budget
      if (C.n <= uint32_t(kBatchSmemQubits) || P.T != uint32_t(kBatchRegT) || P.R != 4u || P.c < 1 ||
          P.c + 4 > P.T || P.n_tiles != (uint64_t(1) << (C.n - P.T)) || !batch_reg_fits(P.c, P.n_stages, P.data_bytes) ||
          !w_table_ok(&P))
        return false;
      if (C.plan_off + P.aux_off + sizeof(RegPassParams) > plans_size ||
          C.plan_off + P.ops_off + uint64_t(P.data_bytes) > plans_size || (P.aux_off & 15u) || (P.ops_off & 15u))
        return false;
      const RegPassParams *prm = reinterpret_cast<const RegPassParams *>(plan + P.aux_off);
      if (prm->chk[0] != P.T || prm->chk[1] != P.n_stages || prm->chk[2] != P.data_bytes || prm->chk[3] != P.ops_off)
        return false;
      continue;
    }
    if (P.kind != KIND_SMEM) return false;
    if (P.T < 1 || P.T > uint32_t(kBatchSmemQubits) || P.c < 1 || P.c > P.T || P.T > C.n) return false;
    if (C.n <= uint32_t(kBatchSmemQubits) && P.T != C.n) return false;
    if (P.n_tiles != (uint64_t(1) << (C.n - P.T))) return false;
    if (C.plan_off + P.ops_off + uint64_t(P.n_ops) * sizeof(OpRec) > plans_size) return false;
    const OpRec *ops = reinterpret_cast<const OpRec *>(plan + P.ops_off);
    for (uint32_t o = 0; o < P.n_ops; o++) {
      const OpRec op = ops[o];
      if (op.type == OP_DENSE) {
        if (op.k < 1 || op.k > KMAX) return false;
        for (int m = 0; m < op.k; m++)
          if (op.lb[m] >= P.T) return false;
        if (C.plan_off + op.data_off + (uint64_t(8) << (2 * op.k)) > plans_size) return false;
      } else if (op.type == OP_PHASE) {
        if (C.plan_off + op.data_off + uint64_t(op.count) * sizeof(PhaseTerm) > plans_size) return false;
        const PhaseTerm *t = reinterpret_cast<const PhaseTerm *>(plan + op.data_off);
        for (uint32_t i = 0; i < op.count; i++)
          if (t[i].la < -1 || t[i].la >= int32_t(P.T)) return false;
      } else {
        return false;
      }
    }
  }
  return true;
}

template <int KMAX>
__device__ __forceinline__ void batch_ops(float2 *tile, float2 *mat, uint32_t *acc, float2 *tab,
                                          const uint8_t *plan, const PlanPass &P, uint64_t base) {
  const OpRec *ops = reinterpret_cast<const OpRec *>(plan + P.ops_off);
  for (uint32_t o = 0; o < P.n_ops; o++) {
    const OpRec op = ops[o];
    if (op.type == OP_DENSE) {
      const float2 *src = reinterpret_cast<const float2 *>(plan + op.data_off);
      const uint32_t ne = 1u << (2 * op.k);
      for (uint32_t i = threadIdx.x; i < ne; i += blockDim.x) mat[i] = src[i];
      __syncthreads();
      switch (op.k) {
        case 1: apply_dense<1>(tile, mat, op.lb, P.T); break;
        case 2: if constexpr (KMAX >= 2) apply_dense<2>(tile, mat, op.lb, P.T); break;
        case 3: if constexpr (KMAX >= 3) apply_dense<3>(tile, mat, op.lb, P.T); break;
        default: break;
      }
    } else {
      apply_phase(tile, reinterpret_cast<const PhaseTerm *>(plan + op.data_off), op.count, base, P.T, acc, tab);
    }
    __syncthreads();
  }
}

template <int KMAX>
__global__ void __launch_bounds__(kBatchNT, KMAX <= 2 ? 2 : 1) k_batch(const uint8_t *__restrict__ plans,
                                                   const BatchCirc *__restrict__ circs, uint32_t n_circ,
                                                   float2 *__restrict__ arena, double *__restrict__ scratch,
                                                   uint64_t *__restrict__ out, double *__restrict__ ex,
                                                   uint32_t *__restrict__ counter, uint64_t plans_size) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint32_t s_next;
  const BatchLayout L = batch_layout(KMAX);
  float2 *tile = reinterpret_cast<float2 *>(smem + L.off_tile);
  uint64_t *segoff = reinterpret_cast<uint64_t *>(smem + L.off_seg);
  float2 *mat = reinterpret_cast<float2 *>(smem + L.off_mat);
  float2 *tab = reinterpret_cast<float2 *>(smem + L.off_tab);
  uint32_t *acc = reinterpret_cast<uint32_t *>(smem + L.off_acc);
  double *chunk_s = reinterpret_cast<double *>(smem + L.off_chunk);
  double *tot = reinterpret_cast<double *>(smem + L.off_tot);
  for (;;) {
    if (threadIdx.x == 0) s_next = atomicAdd(counter, 1u);
    __syncthreads();
    const uint32_t ci = s_next;
    __syncthreads();
    if (ci >= n_circ) break;
    const BatchCirc C = circs[ci];
    if (!batch_plan_ok<KMAX>(plans, plans_size, C)) {
      if (threadIdx.x == 0) atomicOr(counter + 1, 1u);
      continue;
    }
    const uint8_t *plan = plans + C.plan_off;
    const uint32_t n = C.n, N = 1u << n;
    if (n <= uint32_t(kBatchSmemQubits)) {
      for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) tile[i] = make_float2(i == 0 ? 1.f : 0.f, 0.f);
      __syncthreads();
      for (uint32_t p = 0; p < C.n_passes; p++) {
        const PlanPass P = reinterpret_cast<const PlanPass *>(plan)[p];
        batch_ops<KMAX>(tile, mat, acc, tab, plan, P, 0);
      }
      if (C.shots) batch_measure(tile, n, C.seed, C.shots, out + C.out_off, chunk_s, tot);
      if (C.flags & 2u) batch_expect(tile, n, C.zmask, ex + 2 * ci, tot);
      if (C.flags & 1u) {
        for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) arena[C.state_off + i] = tile[i];
      }
    } else {
      float2 *st = arena + C.state_off;
      for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) st[i] = make_float2(i == 0 ? 1.f : 0.f, 0.f);
      __syncthreads();
      for (uint32_t p = 0; p < C.n_passes; p++) {
        const PlanPass P = reinterpret_cast<const PlanPass *>(plan)[p];
        if (P.kind == KIND_REG) {
          // register stages over the circuit's tiles in order; the address tables
          // go to the end of the register region first
          RegPassParams *prm_s = reinterpret_cast<RegPassParams *>(smem + kBatchRegSmem - sizeof(RegPassParams));
          {
            const uint4 *src = reinterpret_cast<const uint4 *>(plan + P.aux_off);
            uint4 *dst = reinterpret_cast<uint4 *>(prm_s);
            for (uint32_t i = threadIdx.x; i < sizeof(RegPassParams) / 16; i += blockDim.x) dst[i] = src[i];
          }
          __syncthreads();
          reg_pass_tiles<4>(st, plan, reinterpret_cast<const PlanPass *>(plan) + p, *prm_s, smem, 0, 1);
          __syncthreads();
          continue;
        }
        const uint32_t Lt = 1u << P.T, nseg = 1u << (P.T - P.c);
        const uint32_t cs = P.c - 1u, cmask = (1u << cs) - 1u;
        for (uint32_t s = threadIdx.x; s < nseg; s += blockDim.x) segoff[s] = pdep_u64(s, P.high_mask);
        __syncthreads();
        for (uint64_t t = 0; t < P.n_tiles; t++) {
          const uint64_t base = pdep_u64(t, P.outer_mask);
          for (uint32_t i = threadIdx.x; i < (Lt >> 1); i += blockDim.x)
            cp_async16(tile + 2 * i, st + base + segoff[i >> cs] + (uint64_t(i & cmask) << 1));
          cp_async_wait_all();
          __syncthreads();
          batch_ops<KMAX>(tile, mat, acc, tab, plan, P, base);
          const float4 *t4 = reinterpret_cast<const float4 *>(tile);
          for (uint32_t i = threadIdx.x; i < (Lt >> 1); i += blockDim.x)
            *reinterpret_cast<float4 *>(st + base + segoff[i >> cs] + (uint64_t(i & cmask) << 1)) = t4[i];
          __syncthreads();
        }
      }
      if (C.shots) batch_measure(st, n, C.seed, C.shots, out + C.out_off, scratch + C.scratch_off, tot);
      if (C.flags & 2u) batch_expect(st, n, C.zmask, ex + 2 * ci, tot);
    }
  }
}

}  // namespace svgb

using namespace svgb;

struct sv_batch {
  int device = 0;
  cudaStream_t stream = nullptr;
  size_t n_circ = 0;
  int kmax = 2;
  std::vector<BatchCirc> circ;       // in launch (cost) order
  std::vector<size_t> order;         // order[i] = caller index of launch slot i
  std::vector<size_t> slot;          // slot[caller index] = launch slot
  uint8_t *plan_dev = nullptr;
  uint64_t plans_size = 0;
  BatchCirc *circ_dev = nullptr;
  float2 *arena = nullptr;
  double *scratch = nullptr;
  uint64_t *out = nullptr;
  double *ex = nullptr;
  uint32_t *counter = nullptr;
  size_t out_count = 0, arena_count = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool keep = false;
  unsigned grid = 1;
  uint64_t passes = 0, launch_bytes = 0;
};

namespace {

void free_batch(sv_batch *b) {
  if (!b) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  cudaFree(b->plan_dev);
  cudaFree(b->circ_dev);
  cudaFree(b->arena);
  cudaFree(b->scratch);
  cudaFree(b->out);
  cudaFree(b->ex);
  cudaFree(b->counter);
  cudaSetDevice(prev);
  delete b;
}

// Kernel attributes and grid size (outside any stream capture).
template <int KMAX>
cudaError_t prepare_batch(sv_batch *b) {
  const BatchLayout L = batch_layout(KMAX);
  cudaError_t e = cudaFuncSetAttribute(k_batch<KMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(L.total));
  if (e != cudaSuccess) return e;
  int per_sm = 0, sms = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<KMAX>, kBatchNT, L.total);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  if (e != cudaSuccess) return e;
  size_t grid = size_t(std::max(per_sm, 1)) * size_t(std::max(sms, 1));
  b->grid = unsigned(grid < b->n_circ ? grid : b->n_circ);
  return cudaSuccess;
}

// The captured work: reset the work counter, one persistent launch.
template <int KMAX>
cudaError_t enqueue_batch(sv_batch *b, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(b->counter, 0, sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  k_batch<KMAX><<<b->grid, kBatchNT, batch_layout(KMAX).total, st>>>(b->plan_dev, b->circ_dev, uint32_t(b->n_circ),
                                                                    b->arena, b->scratch, b->out, b->ex,
                                                                    b->counter, b->plans_size);
  return cudaGetLastError();
}

cudaError_t prepare_any(sv_batch *b) {
  switch (b->kmax) {
    case 1: return prepare_batch<1>(b);
    case 2: return prepare_batch<2>(b);
    default: return prepare_batch<3>(b);
  }
}

cudaError_t enqueue_any(sv_batch *b, cudaStream_t st) {
  switch (b->kmax) {
    case 1: return enqueue_batch<1>(b, st);
    case 2: return enqueue_batch<2>(b, st);
    default: return enqueue_batch<3>(b, st);
  }
}

}  // namespace

extern "C" {

int sv_batch_create(size_t n_circ, const sv_gate *const *irs, const size_t *n_gates, const int *n_qubits,
                    const uint64_t *shots, const uint64_t *seeds, const uint64_t *zmasks, const sv_opts *opts,
                    int keep_states, void *cuda_stream, sv_batch **out) {
  if (!out) return set_last_error(SV_ERR_ARG, "out is null");
  *out = nullptr;
  if (n_circ == 0 || !irs || !n_gates || !n_qubits || !shots || !seeds)
    return set_last_error(SV_ERR_ARG, "empty batch or null array");
  sv_opts o{};
  if (opts) o = *opts;
  const int kmax = o.k_max ? o.k_max : 2;
  const int T = o.tile_qubits ? std::min(o.tile_qubits, kBatchSmemQubits) : kBatchSmemQubits;
  if (kmax < 1 || kmax > kBatchMaxK) return set_last_error(SV_ERR_ARG, "batched k_max must be in [1,3]");
  if (T < 6) return set_last_error(SV_ERR_ARG, "batched tile_qubits must be >= 6");
  if (o.precision != 0) return set_last_error(SV_ERR_UNSUPPORTED, "batched mode computes in FP32 (precision 0)");
  sv_batch *b = new sv_batch();
  b->n_circ = n_circ;
  b->kmax = kmax;
  b->keep = keep_states != 0;
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  if (cudaGetDevice(&b->device) != cudaSuccess) {
    delete b;
    return set_last_error(SV_ERR_CUDA, "no CUDA device");
  }
  // plan every circuit (shared-memory sweep ops on tiles of <= T qubits)
  std::vector<uint8_t> plans;
  std::vector<BatchCirc> circ(n_circ);
  std::vector<double> cost(n_circ);
  sv_opts po{};
  po.k_max = kmax;
  po.low_qubits = 5;
  po.kernel_variant = 1;
  uint64_t arena = 0, scratch = 0, outs = 0;
  for (size_t i = 0; i < n_circ; i++) {
    const int n = n_qubits[i];
    if (n < 1 || n > kBatchMaxQubits) {
      free_batch(b);
      return set_last_error(SV_ERR_ARG, "circuit %zu: n_qubits must be in [1,%d]", i, kBatchMaxQubits);
    }
    if (shots[i] > 0xffffffffull) {
      free_batch(b);
      return set_last_error(SV_ERR_ARG, "circuit %zu: too many shots", i);
    }
    po.tile_qubits = n <= kBatchSmemQubits ? n : T;
    po.kernel_variant = 1;
    // arena states with tiles of kBatchRegT qubits: register-stage passes (16
    // amplitudes a thread) where every pass fits the kernel's register region
    const bool try_reg = n > kBatchSmemQubits && T == kBatchRegT;
    if (try_reg) po.kernel_variant = 2;
    Plan plan;
    std::string err;
    if (n_gates[i] && !irs[i]) {
      free_batch(b);
      return set_last_error(SV_ERR_ARG, "circuit %zu: ir is null", i);
    }
    if (!build_plan(n, irs[i], n_gates[i], &po, plan, err)) {
      free_batch(b);
      return set_last_error(SV_ERR_ARG, "circuit %zu: %s", i, err.c_str());
    }
    if (try_reg) {
      bool ok = true;
      for (auto &pp : plan.passes)
        if (pp.kind == KIND_REG && (pp.R != 4u || pp.T != uint32_t(kBatchRegT) || !batch_reg_fits(pp.c, pp.n_stages, pp.data_bytes)))
          ok = false;
      if (!ok) {  // shared-memory sweeps instead
        po.kernel_variant = 1;
        plan = Plan();
        if (!build_plan(n, irs[i], n_gates[i], &po, plan, err)) {
          free_batch(b);
          return set_last_error(SV_ERR_ARG, "circuit %zu: %s", i, err.c_str());
        }
      }
    }
    // address tables of the register passes follow the circuit's records; each
    // pass record points at its table (aux_off, from the circuit's plan base)
    while (plan.bytes.size() % 16) plan.bytes.push_back(0);
    for (size_t pi = 0; pi < plan.passes.size(); pi++) {
      if (plan.passes[pi].kind != KIND_REG) continue;
      const uint32_t aux = uint32_t(plan.bytes.size());
      const uint8_t *rp = reinterpret_cast<const uint8_t *>(&plan.rparams[pi]);
      plan.bytes.insert(plan.bytes.end(), rp, rp + sizeof(RegPassParams));
      plan.passes[pi].aux_off = aux;
      std::memcpy(plan.bytes.data() + plan.pass_offs[pi], &plan.passes[pi], sizeof(PlanPass));
    }
    for (auto &pp : plan.passes) {
      if (pp.kmax > uint32_t(kBatchMaxK)) {
        free_batch(b);
        return set_last_error(SV_ERR_UNSUPPORTED, "circuit %zu: a %u-qubit block exceeds the batched limit of %d",
                              i, pp.kmax, kBatchMaxK);
      }
      // the kernel instance covers the widest block planned (a gate wider than
      // k_max keeps a block of its own)
      b->kmax = std::max<int>(b->kmax, int(pp.kmax));
    }
    while (plans.size() % 16) plans.push_back(0);
    BatchCirc &c = circ[i];
    c.plan_off = plans.size();
    plans.insert(plans.end(), plan.bytes.begin(), plan.bytes.end());
    c.n = uint32_t(n);
    c.n_passes = uint32_t(plan.passes.size());
    c.shots = uint32_t(shots[i]);
    c.seed = seeds[i];
    c.flags = b->keep ? 1u : 0u;
    if (zmasks && zmasks[i]) {
      if (zmasks[i] >> n) {
        free_batch(b);
        return set_last_error(SV_ERR_ARG, "circuit %zu: zmask has bits beyond n_qubits", i);
      }
      c.zmask = zmasks[i];
      c.flags |= 2u;
    }
    c.out_off = outs;
    outs += shots[i];
    if (n > kBatchSmemQubits || b->keep) {
      c.state_off = arena;
      arena += uint64_t(1) << n;
    }
    if (n > kBatchSmemQubits) {
      c.scratch_off = scratch;
      scratch += uint64_t(1) << (n - 6);
    }
    cost[i] = std::ldexp(1.0, n) * double(plan.passes.size() + 1) * (n > kBatchSmemQubits ? 4.0 : 1.0) +
              double(shots[i]) * 64.0;
    b->passes += plan.passes.size();
    if (n > kBatchSmemQubits) b->launch_bytes += plan.passes.size() * (uint64_t(16) << n);
  }
  // largest first: the tail of the launch is short circuits
  b->order.resize(n_circ);
  for (size_t i = 0; i < n_circ; i++) b->order[i] = i;
  std::stable_sort(b->order.begin(), b->order.end(), [&](size_t x, size_t y) { return cost[x] > cost[y]; });
  b->slot.resize(n_circ);
  b->circ.resize(n_circ);
  for (size_t s = 0; s < n_circ; s++) {
    b->circ[s] = circ[b->order[s]];
    b->slot[b->order[s]] = s;
  }
  b->out_count = outs;
  b->arena_count = arena;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaError_t e = cudaMalloc(&b->plan_dev, std::max<size_t>(plans.size(), 16));
  if (e == cudaSuccess) e = cudaMalloc(&b->circ_dev, n_circ * sizeof(BatchCirc));
  if (e == cudaSuccess) e = cudaMalloc(&b->arena, std::max<uint64_t>(arena, 2) * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc(&b->scratch, std::max<uint64_t>(scratch, 2) * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&b->out, std::max<uint64_t>(outs, 2) * sizeof(uint64_t));
  if (e == cudaSuccess) e = cudaMalloc(&b->ex, 2 * n_circ * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&b->counter, 2 * sizeof(uint32_t));  // work queue, error word
  // The records, the circuit table and the zeroed words are written on the
  // batch's own stream, ahead of every launch of the graph on it.  (On the legacy
  // default stream they were not ordered before launches on a non-blocking
  // stream: a pageable cudaMemcpy may return before its DMA lands and cudaMemset
  // is asynchronous, so a launch under load could read stale records.)
  if (e == cudaSuccess) e = cudaMemsetAsync(b->ex, 0, 2 * n_circ * sizeof(double), b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->counter, 0, 2 * sizeof(uint32_t), b->stream);
  b->plans_size = plans.size();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->plan_dev, plans.data(), plans.size(), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->circ_dev, b->circ.data(), n_circ * sizeof(BatchCirc), cudaMemcpyHostToDevice, b->stream);
  // capture the launch once; sv_batch_launch replays the graph
  if (e == cudaSuccess) e = prepare_any(b);
  cudaStream_t cap = nullptr;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    const cudaError_t le = enqueue_any(b, cap);
    e = cudaStreamEndCapture(cap, &b->graph);
    if (le != cudaSuccess) e = le;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (cap) cudaStreamDestroy(cap);
  if (e != cudaSuccess) {
    const int code = e == cudaErrorMemoryAllocation ? SV_ERR_OOM : SV_ERR_CUDA;
    cudaGetLastError();
    free_batch(b);
    return set_last_error(code, "sv_batch_create: %s", cudaGetErrorString(e));
  }
  *out = b;
  return set_last_error(SV_OK, "");
}

int sv_batch_launch(sv_batch *b) {
  if (!b) return set_last_error(SV_ERR_ARG, "null batch");
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != b->device) cudaSetDevice(b->device);
  const cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
  count_launch();
  if (prev != b->device) cudaSetDevice(prev);
  if (e != cudaSuccess) return set_last_error(SV_ERR_CUDA, "sv_batch_launch: %s", cudaGetErrorString(e));
  return SV_OK;
}

int sv_batch_synchronize(sv_batch *b) {
  if (!b) return set_last_error(SV_ERR_ARG, "null batch");
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return set_last_error(SV_ERR_CUDA, "sv_batch_synchronize: %s", cudaGetErrorString(e));
  uint32_t bad = 0;
  e = cudaMemcpy(&bad, b->counter + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return set_last_error(SV_ERR_CUDA, "sv_batch_synchronize: %s", cudaGetErrorString(e));
  if (bad) return set_last_error(SV_ERR_STATE, "batched launch skipped circuits whose plan records failed validation");
  return SV_OK;
}

int sv_batch_samples(sv_batch *b, size_t circuit, uint64_t *out, int on_device) {
  if (!b || !out) return set_last_error(SV_ERR_ARG, "null argument");
  if (circuit >= b->n_circ) return set_last_error(SV_ERR_ARG, "circuit index out of range");
  const BatchCirc &c = b->circ[b->slot[circuit]];
  const cudaError_t e = cudaMemcpyAsync(out, b->out + c.out_off, size_t(c.shots) * sizeof(uint64_t),
                                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess && !on_device) cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return set_last_error(SV_ERR_CUDA, "sv_batch_samples: %s", cudaGetErrorString(e));
  return SV_OK;
}

int sv_batch_expectation(sv_batch *b, size_t circuit, double *out2) {
  if (!b || !out2) return set_last_error(SV_ERR_ARG, "null argument");
  if (circuit >= b->n_circ) return set_last_error(SV_ERR_ARG, "circuit index out of range");
  const size_t slot = b->slot[circuit];
  if (!(b->circ[slot].flags & 2u)) return set_last_error(SV_ERR_ARG, "circuit %zu has no zmask", circuit);
  cudaError_t e = cudaMemcpyAsync(out2, b->ex + 2 * slot, 2 * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return set_last_error(SV_ERR_CUDA, "sv_batch_expectation: %s", cudaGetErrorString(e));
  return SV_OK;
}

int sv_batch_amplitudes(sv_batch *b, size_t circuit, void *out) {
  if (!b || !out) return set_last_error(SV_ERR_ARG, "null argument");
  if (circuit >= b->n_circ) return set_last_error(SV_ERR_ARG, "circuit index out of range");
  const BatchCirc &c = b->circ[b->slot[circuit]];
  if (!b->keep && c.n <= uint32_t(kBatchSmemQubits))
    return set_last_error(SV_ERR_ARG, "states of <= %d qubits are kept only with keep_states", kBatchSmemQubits);
  cudaError_t e = cudaMemcpyAsync(out, b->arena + c.state_off, (size_t(1) << c.n) * sizeof(float2),
                                  cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return set_last_error(SV_ERR_CUDA, "sv_batch_amplitudes: %s", cudaGetErrorString(e));
  return SV_OK;
}

int sv_batch_stats(const sv_batch *b, uint64_t *n_passes, uint64_t *hbm_bytes) {
  if (!b) return set_last_error(SV_ERR_ARG, "null batch");
  if (n_passes) *n_passes = b->passes;
  if (hbm_bytes) *hbm_bytes = b->launch_bytes;
  return SV_OK;
}

int sv_batch_destroy(sv_batch *b) {
  free_batch(b);
  return SV_OK;
}

int sv_batch_autotune(size_t n_circ, const sv_gate *const *irs, const size_t *n_gates, const int *n_qubits,
                      const uint64_t *shots, const uint64_t *seeds, int reps, sv_opts *best, double *best_ms) {
  if (!best) return set_last_error(SV_ERR_ARG, "best is null");
  if (reps < 1) reps = 1;
  const int ks[] = {1, 2, 3};
  const int ts[] = {10, 11, 12, 13};
  double best_t = 1e300;
  sv_opts best_o{};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return set_last_error(SV_ERR_CUDA, "sv_batch_autotune: event creation failed");
  int rc = SV_OK;
  for (int k : ks)
    for (int t : ts) {
      sv_opts o{};
      o.k_max = k;
      o.tile_qubits = t;
      sv_batch *b = nullptr;
      rc = sv_batch_create(n_circ, irs, n_gates, n_qubits, shots, seeds, nullptr, &o, 0, nullptr, &b);
      if (rc == SV_ERR_UNSUPPORTED) continue;  // a block wider than this k_max
      if (rc) break;
      rc = sv_batch_launch(b);  // warm-up
      if (rc == SV_OK) cudaEventRecord(e0, b->stream);
      for (int r = 0; rc == SV_OK && r < reps; r++) rc = sv_batch_launch(b);
      if (rc == SV_OK) cudaEventRecord(e1, b->stream);
      if (rc == SV_OK) rc = sv_batch_synchronize(b);
      float ms = 0.f;
      if (rc == SV_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms / reps < best_t) {
        best_t = ms / reps;
        best_o = o;
      }
      sv_batch_destroy(b);
      if (rc) break;
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  if (best_t >= 1e300) return set_last_error(SV_ERR_UNSUPPORTED, "sv_batch_autotune: no candidate ran");
  *best = best_o;
  if (best_ms) *best_ms = best_t;
  return SV_OK;
}

int sv_batch_run(const sv_gate *const *irs, const size_t *n_gates, const int *n_qubits, size_t n_circ,
                 const uint64_t *shots, const uint64_t *seeds, uint64_t *const *out, const sv_opts *opts) {
  if (!out) return set_last_error(SV_ERR_ARG, "out is null");
  sv_batch *b = nullptr;
  int rc = sv_batch_create(n_circ, irs, n_gates, n_qubits, shots, seeds, nullptr, opts, 0, nullptr, &b);
  if (rc) return rc;
  rc = sv_batch_launch(b);
  for (size_t i = 0; rc == SV_OK && i < n_circ; i++)
    if (out[i]) rc = sv_batch_samples(b, i, out[i], 0);
  if (rc == SV_OK) rc = sv_batch_synchronize(b);
  sv_batch_destroy(b);
  return rc;
}

}  // extern "C"
