// sv_apply.cu -- the HBM pass kernels of sv_apply_circuit.
//
// One launch applies one pass of the plan (see sv_internal.h): every CTA owns
// the 2^T amplitudes whose indices share the values of the qubits outside the
// pass's tile set.  Those amplitudes sit in 2^(T-c) runs of 2^c contiguous
// amplitudes (the c lowest qubits are always in the tile).  The state is read
// once and written once per pass: 16 bytes per amplitude.
//
// k_pass_reg (register stages, the default): each thread holds 2^R amplitudes
// in registers.  The first stage loads them straight from HBM (lanes on the
// low tile bits, so a warp reads contiguous runs), every op of a stage is
// applied in registers with compile-time register indices, the tile is
// re-distributed between stages through XOR-swizzled shared memory, and the
// last stage stores straight to HBM.
//
// k_pass (shared-memory sweeps): gathers the tile into shared memory with
// cp.async and applies each op as a sweep over the tile (one thread per group
// of 2^k amplitudes).  Used for tiles too small for register stages.
//
// Diagonal phase ops tabulate a per-tile phase table from 32-bit turn
// fractions (exact modulo 2*pi) over the low and high halves of the tile index.
#include <algorithm>
#include <atomic>
#include <cstdint>

#include "sv_device.cuh"
#include "sv_internal.h"
#include "sv_regpass.cuh"
#include "sv_tc_ptx.cuh"

namespace svgb {

constexpr int kNT = 256;  // threads per CTA

template <int KMAX>
__global__ void __launch_bounds__(kNT) k_pass(float2 *__restrict__ amp, const uint8_t *__restrict__ plan,
                                              uint32_t pass_off) {
  extern __shared__ __align__(16) unsigned char smem[];
  const PlanPass *P = reinterpret_cast<const PlanPass *>(plan + pass_off);
  const uint32_t T = P->T, c = P->c;
  const uint32_t L = 1u << T;
  const uint32_t nseg = 1u << (T - c);
  float2 *tile = reinterpret_cast<float2 *>(smem);
  uint64_t *segoff = reinterpret_cast<uint64_t *>(smem + size_t(L) * sizeof(float2));
  float2 *mat = reinterpret_cast<float2 *>(segoff + nseg);
  float2 *tab = mat + (1u << (2 * KMAX));
  uint32_t *acc = reinterpret_cast<uint32_t *>(tab + 256);

  const uint64_t tile_id = uint64_t(blockIdx.x) + uint64_t(gridDim.x) * blockIdx.y;
  const uint64_t base = pdep_u64(tile_id, P->outer_mask);
  const uint64_t hm = P->high_mask;
  for (uint32_t s = threadIdx.x; s < nseg; s += blockDim.x) segoff[s] = base + pdep_u64(s, hm);
  __syncthreads();

  const uint32_t cs = c - 1u;  // log2(16-byte chunks per run)
  const uint32_t cmask = (1u << cs) - 1u;
  for (uint32_t i = threadIdx.x; i < (L >> 1); i += blockDim.x)
    cp_async16(tile + 2 * i, amp + segoff[i >> cs] + (uint64_t(i & cmask) << 1));
  cp_async_wait_all();
  __syncthreads();

  const OpRec *ops = reinterpret_cast<const OpRec *>(plan + P->ops_off);
  const uint32_t nops = P->n_ops;
  for (uint32_t o = 0; o < nops; o++) {
    const OpRec op = ops[o];
    if (op.type == OP_DENSE) {
      const float2 *src = reinterpret_cast<const float2 *>(plan + op.data_off);
      const uint32_t ne = 1u << (2 * op.k);
      for (uint32_t i = threadIdx.x; i < ne; i += blockDim.x) mat[i] = src[i];
      __syncthreads();
      switch (op.k) {
        case 1: apply_dense<1>(tile, mat, op.lb, T); break;
        case 2: if constexpr (KMAX >= 2) apply_dense<2>(tile, mat, op.lb, T); break;
        case 3: if constexpr (KMAX >= 3) apply_dense<3>(tile, mat, op.lb, T); break;
        case 4: if constexpr (KMAX >= 4) apply_dense<4>(tile, mat, op.lb, T); break;
        case 5: if constexpr (KMAX >= 5) apply_dense<5>(tile, mat, op.lb, T); break;
        default: break;
      }
    } else if (op.type == OP_PHASE) {
      apply_phase(tile, reinterpret_cast<const PhaseTerm *>(plan + op.data_off), op.count, base, T,
                  acc, tab);
    }
    __syncthreads();
  }

  const float4 *t4 = reinterpret_cast<const float4 *>(tile);
  for (uint32_t i = threadIdx.x; i < (L >> 1); i += blockDim.x) {
    float4 *dst = reinterpret_cast<float4 *>(amp + segoff[i >> cs] + (uint64_t(i & cmask) << 1));
    *dst = t4[i];
  }
}


// 16 amplitudes per thread (blocks up to 4 qubits): two CTAs of 256 threads
// per SM; 32 amplitudes per thread (blocks up to 2 qubits): four CTAs of 128
// threads per SM (128 registers a thread).
template <int R, int NTMAX>
__global__ void __launch_bounds__(NTMAX, R == 5 ? (NTMAX <= 128 ? 4 : 2) : (NTMAX <= 256 ? 2 : 1))
    k_pass_reg(float2 *__restrict__ amp, const uint8_t *__restrict__ plan, uint32_t pass_off,
               const __grid_constant__ RegPassParams prm, int *__restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem[];
  const PlanPass *P = reinterpret_cast<const PlanPass *>(plan + pass_off);
  const uint32_t T = P->T, c = P->c;
  const uint32_t ns = P->n_stages;
  const uint32_t data_off = P->ops_off, data_bytes = P->data_bytes;
  const uint64_t outer_mask = P->outer_mask, n_tiles = P->n_tiles;
  // the launch's shared memory was sized from the host's copy of these fields
  if (T != prm.chk[0] || ns != prm.chk[1] || data_bytes != prm.chk[2] || data_off != prm.chk[3] ||
      P->R != uint32_t(R) || ns == 0 || ns > uint32_t(kMaxStages) || !w_table_ok(P)) {
    if (threadIdx.x == 0) atomicOr(err, kPlanMismatch);
    return;
  }
  reg_pass_tiles<R>(amp, plan, P, prm, smem, blockIdx.x, gridDim.x);
}

constexpr size_t kSmemOptIn = 232448;  // 227 KiB per CTA on sm_100-class parts

// One-time per-device setup of a kernel (its shared-memory opt-in) and the
// device's SM count.  Host threads may launch concurrently (the serving loop
// does): the bit for a device is published with release order after its SM
// count is stored, so a reader that sees the bit also sees the count.
template <class F>
static cudaError_t once_per_device(std::atomic<uint64_t> &done, std::atomic<int> *sms, int dev, F &&setup,
                                   int *n_sms) {
  if (dev >= 0 && dev < 64 && ((done.load(std::memory_order_acquire) >> dev) & 1ull)) {
    *n_sms = sms[dev].load(std::memory_order_relaxed);
    return cudaSuccess;
  }
  cudaError_t e = setup();
  if (e != cudaSuccess) return e;
  int v = 0;
  e = cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64) {
    sms[dev].store(v, std::memory_order_relaxed);
    done.fetch_or(1ull << dev, std::memory_order_release);
  }
  *n_sms = v;
  return cudaSuccess;
}

template <int R, int NTMAX>
static cudaError_t launch_reg(float2 *amp, const uint8_t *plan, uint32_t off, const PlanPass &hp,
                              const RegPassParams &prm, int *err, cudaStream_t st) {
  const RegLayout lay = reg_layout(hp.T, hp.c, hp.n_stages, hp.data_bytes, R, true);
  static std::atomic<uint64_t> configured{0};
  static std::atomic<int> sms[64];
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = once_per_device(configured, sms, dev, [] {
    return cudaFuncSetAttribute(k_pass_reg<R, NTMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(kSmemOptIn));
  }, &nsm);
  if (e != cudaSuccess) return e;
  const unsigned nt = 1u << (hp.T - R);
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pass_reg<R, NTMAX>, int(nt), lay.total);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const uint64_t want = uint64_t(nsm > 0 ? nsm : 1) * per_sm;
  const unsigned grid = unsigned(hp.n_tiles < want ? hp.n_tiles : want);
  k_pass_reg<R, NTMAX><<<grid, nt, lay.total, st>>>(amp, plan, off, prm, err);
  count_launch();
  return cudaGetLastError();
}

// Whether a KIND_REG pass fits the persistent kernel's shared-memory tables.
bool reg_pass_fits(uint32_t T, uint32_t c, uint32_t R, uint32_t n_stages, uint32_t data_bytes) {
  return (R == 4 || R == 5) && T <= uint32_t(kMaxTile) && T >= R + 5 && n_stages <= uint32_t(kMaxStages) &&
         data_bytes <= kMaxPassData && reg_layout(T, c, n_stages, data_bytes, R, true).total <= kSmemOptIn;
}


// ---------------------------------------------------------------------------
// tensor-core stages (KIND_TC): the register-stage skeleton with 2^R amplitudes
// per thread (R = 4; R = 5 for 5-qubit stages) and each stage's dense blocks
// applied as one 3xTF32 tcgen05 product (sv_tc.cu).  Per stage and 128-row
// group, the threads split their rows into A_hi / A_lo in tensor memory, one
// thread of the group issues the stage's MMAs (8 for R = 4, 16 for R = 5) and
// commits them to the group's mbarrier, and the group reads D back.  Between
// stages the tile moves through one swizzled exchange buffer with one plain
// CTA barrier per exchange: a thread writes its amplitudes back
// to exactly the positions it read them from at the previous stage, which no
// other thread reads, so no barrier is needed before the writes.  The next tile
// is prefetched (16-byte cp.async, natural order) into a separate load buffer as
// soon as every thread has read the current tile from it (the first exchange's
// barrier), so the load overlaps most of the tile's stages.  The group's threads
// wait for the product on the group's mbarrier themselves.  (The tensor cores'
// float32 accumulation rounds toward zero and shrinks the state by ~1e-7 of its
// norm per stage; for a unitary circuit the passes track the norm, see TcNorm
// and NormAcc.)
// ---------------------------------------------------------------------------

constexpr int kTcErrTimeout = 1;
constexpr size_t kTcStaticSmem = 1024;  // mbarriers and the TMEM base (the static region's size)

struct TcLayout {
  uint32_t L, NT;
  size_t off_in, off_x, off_tt, off_data, total;
};

__host__ __device__ inline TcLayout tc_layout(uint32_t T, uint32_t ns, uint32_t data_bytes, uint32_t R) {
  TcLayout r;
  r.L = 1u << T;
  r.NT = 1u << (T - R);
  size_t o = 0;
  r.off_in = o; o += size_t(r.L) * 8;  // load buffer (natural order)
  r.off_x = o; o += size_t(r.L) * 8;   // exchange buffer (swizzled)
  r.off_tt = o; o += size_t(ns) * r.NT * 4;
  o = (o + 15) & ~size_t(15);
  r.off_data = o; o += data_bytes;
  r.total = (o + 15) & ~size_t(15);
  return r;
}

// Barrier 1 + g over the 128 threads of row group g (literal ids, so ptxas
// reserves only the barriers used).
__device__ __forceinline__ void group_bar_sync(uint32_t g) {
  switch (g) {
    case 0: asm volatile("bar.sync 1, 128;\n" ::: "memory"); break;
    case 1: asm volatile("bar.sync 2, 128;\n" ::: "memory"); break;
    case 2: asm volatile("bar.sync 3, 128;\n" ::: "memory"); break;
    default: asm volatile("bar.sync 4, 128;\n" ::: "memory"); break;
  }
}

// Running sum of |a|^2 over a thread's tiles: each tile's row of amplitudes in
// float32 pairs (re^2, im^2), then added to a float32 sum with its rounding
// error kept in a second float (TwoSum, Knuth), so the sum over hundreds of tiles
// keeps ~2^-44 relative accuracy without per-tile FP64 instructions (slow on this
// part).  The pair goes to double once, at the end of the kernel.
struct NormAcc {
  float s = 0.f, c = 0.f;
  template <int NV>
  __device__ __forceinline__ void add_row(const float2 (&v)[NV]) {
    float2 a = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < NV; j++) a = __ffma2_rn(v[j], v[j], a);
    const float x = __fadd_rn(a.x, a.y);
    const float t = __fadd_rn(s, x);
    const float bp = __fsub_rn(t, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp));
    s = t;
    c = __fadd_rn(c, e);
  }
  // warp sum in double, one atomic add per warp
  __device__ __forceinline__ void flush(double *dst) const {
    double x = double(s) + double(c);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31u) == 0) atomicAdd(dst, x);
  }
};

// R = 4: 16 amplitudes a thread, T = 11, 12, 13 with 128, 256, 512 threads (4, 2,
// 1 CTAs per SM: at most 128 registers a thread); R = 5: 32 amplitudes a thread
// (5-qubit stages), T = 12, 13 with 128, 256 threads.
template <int NT, int R>
__global__ void __launch_bounds__(NT, R == 5 ? 1 : (NT <= 128 ? 4 : (NT <= 256 ? 2 : 1)))
    k_pass_tc(float2 *__restrict__ amp, const uint8_t *__restrict__ plan, uint32_t pass_off,
              const __grid_constant__ RegPassParams prm, int *__restrict__ err, const TcNorm nrm) {
  constexpr int NR = 1 << R;  // amplitudes per thread
  constexpr uint32_t kT = uint32_t(R) + (NT == 128 ? 7u : (NT == 256 ? 8u : 9u));
  constexpr uint32_t NG = NT / 128;
  constexpr uint32_t kCols = tc_cols_per_group(R);
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar[NG];
  __shared__ uint32_t tbase_s;
  const PlanPass *P = reinterpret_cast<const PlanPass *>(plan + pass_off);
  const uint32_t T = P->T, c = P->c, ns = P->n_stages;
  const uint32_t data_off = P->ops_off, data_bytes = P->data_bytes;
  const uint64_t outer_mask = P->outer_mask, n_tiles = P->n_tiles;
  // the launch's shared memory was sized from the host's copy of these fields
  if (T != kT || T != prm.chk[0] || ns != prm.chk[1] || data_bytes != prm.chk[2] || data_off != prm.chk[3] ||
      P->R != uint32_t(R) || P->kind != KIND_TC || ns == 0 || ns > uint32_t(kMaxStages) || !w_table_ok(P)) {
    if (threadIdx.x == 0) atomicOr(err, kPlanMismatch);
    return;
  }
  const TcLayout lay = tc_layout(T, ns, data_bytes, R);
  uint32_t *tt = reinterpret_cast<uint32_t *>(smem + lay.off_tt);
  uint8_t *data = smem + lay.off_data;
  const uint32_t tid = threadIdx.x, warp = tid >> 5, g = tid >> 7;

  {
    const uint4 *src = reinterpret_cast<const uint4 *>(plan + data_off);
    uint4 *dst = reinterpret_cast<uint4 *>(data);
    for (uint32_t i = tid; i < data_bytes / 16; i += NT) dst[i] = src[i];
  }
  fence_proxy_async_smem();  // stage images are read by the tensor cores
  if (warp == 0) {
    tmem_alloc(&tbase_s, NG * kCols);  // 4 x 2^(R+1) columns per row group
    tmem_relinquish();
  }
  if (tid < NG) mbar_init(&bar[tid], 1);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const StageRec *stages = reinterpret_cast<const StageRec *>(data + (P->stages_off - data_off));
  const OpRec *ops = reinterpret_cast<const OpRec *>(data);
  // outer-term slots of the phase ops, their per-tile sums in alternate halves
  const uint32_t n_w = P->n_w;
  const uint8_t *wrec = data + (n_w ? P->w_off - data_off : 0u);
  uint32_t *wsum = reinterpret_cast<uint32_t *>(data + (n_w ? P->w_off - data_off + rphase_w_sums(n_w) : 0u));
  uint32_t wpar = 0;
  // per-thread stage tables (own entries only): low 16 bits local index part, high 16 swizzled
  for (uint32_t s = 0; s < ns; s++) {
    uint32_t LB = 0;
    for (uint32_t i = 0; i < T - uint32_t(R); i++)
      if ((tid >> i) & 1u) LB |= 1u << stages[s].tb[i];
    tt[s * NT + tid] = LB | (swz(LB) << 16);
  }
  const uint64_t hm = P->high_mask;
  const uint32_t cs = c - 1u, cmask = (1u << cs) - 1u;
  constexpr int NK = NR / 2;  // 16-byte chunks per thread per tile
  const uint32_t sin = smem_u32(smem + lay.off_in), sx = smem_u32(smem + lay.off_x);
  const uint32_t tbase = tbase_s;
  const uint32_t gcols = tbase + g * kCols;
  const uint32_t tq = gcols + (((warp & 3u) * 32u) << 16);  // this thread's lane
  // the load buffer is swizzled (swzl): the first stage reads local index l at
  // swzl(l) = swzl(thread part) ^ swzl(register part); 16-byte chunk q lands at swzl(2q)
  const uint32_t t_ldx = swzl(tt[tid] & 0xffffu) * 8u;
  uint64_t t_st = 0;
  {
    const uint32_t LB = tt[(ns - 1) * NT + tid] & 0xffffu;
    for (uint32_t x = 0; x < T; x++)
      if ((LB >> x) & 1u) t_st |= uint64_t(1) << prm.oq[x];
  }
  const uint64_t t_cp = pdep_u64(tid >> cs, hm) + (uint64_t(tid & cmask) << 1);
  const uint32_t t_sd = swzl(2u * tid) * 8u;  // chunks tid + k * NT: swzl(2 k NT) xor-ed in per k

  uint64_t tile = blockIdx.x;
  uint64_t base = tile < n_tiles ? pdep_u64(tile, outer_mask) : 0;
  if (tile < n_tiles) {
#pragma unroll
    for (int k = 0; k < NK; k++)
      cp_async16_s(sin + (t_sd ^ (swzl(2u * uint32_t(k) * NT) * 8u)), amp + base + t_cp + prm.ko[k]);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  uint32_t parity = 0;
  bool bad = false, aborted = false;
  float2 v[NR];
  // the previous pass's norm drift, undone on load: a <- a + a * delta with
  // delta = sqrt(ref / prev) - 1 (~1e-7, far finer than float32 steps of 1)
  float delta = 0.f;
  if (nrm.ref && nrm.prev) {
    const double r = *nrm.ref, q = *nrm.prev;
    if (r > 0.0 && q > 0.0 && r < 1e300 && q < 1e300) delta = float(sqrt(r / q) - 1.0);
  }
  if (nrm.clear && blockIdx.x == 0 && tid == 0) *nrm.clear = 0.0;
  NormAcc acc_in, acc_out;
  while (tile < n_tiles) {
    const uint64_t next = tile + gridDim.x;
    const uint64_t base_next = next < n_tiles ? pdep_u64(next, outer_mask) : 0;
    if (n_w) rphase_tile_sums(wrec, n_w, data_bytes - (P->w_off - data_off), base, wsum + wpar * n_w);
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    if (__syncthreads_or(bad)) {  // the tile has landed; the previous tile is done
      aborted = true;
      break;
    }
#pragma unroll
    for (int j = 0; j < NR; j++) v[j] = lds64(sin + (t_ldx ^ prm.lo[j]));
    if (nrm.in_sum) acc_in.add_row(v);
    if (delta != 0.f) {
      const float2 d2 = make_float2(delta, delta);
#pragma unroll
      for (int j = 0; j < NR; j++) v[j] = __ffma2_rn(v[j], d2, v[j]);
    }
    if (ns == 1) {  // no exchange barrier: make sure every thread has read the load buffer
      if (__syncthreads_or(bad)) {
        aborted = true;
        break;
      }
      if (next < n_tiles) {
#pragma unroll
        for (int k = 0; k < NK; k++)
          cp_async16_s(sin + (t_sd ^ (swzl(2u * uint32_t(k) * NT) * 8u)), amp + base_next + t_cp + prm.ko[k]);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
      }
    }
    for (uint32_t s = 0; s < ns; s++) {
      const StageRec &st = stages[s];
      const uint32_t w = tt[s * NT + tid];
      if (s > 0) {
        const uint32_t PBp = (tt[(s - 1) * NT + tid] >> 16) * 8u, PB = (w >> 16) * 8u;
        uint32_t xo[NR];
        const uint4 *q = reinterpret_cast<const uint4 *>(stages[s - 1].xo);
#pragma unroll
        for (int j = 0; j < NR / 4; j++) {
          const uint4 t4 = q[j];
          xo[4 * j] = t4.x; xo[4 * j + 1] = t4.y; xo[4 * j + 2] = t4.z; xo[4 * j + 3] = t4.w;
        }
#pragma unroll
        for (int j = 0; j < NR; j++) sts64(sx + (xo[j] ^ PBp), v[j]);
        // a plain barrier (an OR-reducing one measured 3% slower per pass): a
        // timed-out wait is reported at the next tile's barrier, after at most
        // one bounded wait per remaining stage
        __syncthreads();
        if (s == 1 && next < n_tiles) {  // every thread has read the load buffer at stage 0
#pragma unroll
          for (int k = 0; k < NK; k++)
            cp_async16_s(sin + (t_sd ^ (swzl(2u * uint32_t(k) * NT) * 8u)), amp + base_next + t_cp + prm.ko[k]);
          asm volatile("cp.async.commit_group;\n" ::: "memory");
        }
        q = reinterpret_cast<const uint4 *>(st.xo);
#pragma unroll
        for (int j = 0; j < NR / 4; j++) {
          const uint4 t4 = q[j];
          xo[4 * j] = t4.x; xo[4 * j + 1] = t4.y; xo[4 * j + 2] = t4.z; xo[4 * j + 3] = t4.w;
        }
#pragma unroll
        for (int j = 0; j < NR; j++) v[j] = lds64(sx + (xo[j] ^ PB));
      }
      if (st.flags & 4u) {
        store_row_split<R>(tq, v);
        tmem_wait_st();
        tc_fence_before();
        group_bar_sync(g);  // the group's rows are in tensor memory
        if ((tid & 127u) == 0) {  // one thread issues and commits
          tc_fence_after();
          issue_stage_mma<R>(gcols, smem_u32(data + (st.b_off - data_off)));
          mma_commit(&bar[g]);
        }
        // every thread of the group waits for the commit's phase itself (a
        // thread cannot reach the next stage's wait before the whole group has
        // passed the next group barrier, so phases cannot be skipped)
        if (!mbar_wait_bounded(&bar[g], parity)) bad = true;
        parity ^= 1u;
        tc_fence_after();
        load_row_sum<R>(tq, v);
      }
      const uint32_t oe = st.op_end;
      for (uint32_t o = st.op_begin; o < oe; o++) {
        const OpRec op = ops[o];
        reg_rphase<R>(v, data + (op.data_off - data_off), wsum + wpar * n_w, tid);
      }
    }
    if (aborted) break;
    if (nrm.out_sum) acc_out.add_row(v);
    {
      float2 *dst = amp + base + t_st;
#pragma unroll
      for (int j = 0; j < NR; j++) __stcs(dst + prm.go[j], v[j]);
    }
    tile = next;
    base = base_next;
    wpar ^= 1u;
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tbase, NG * kCols);
  if (tid == 0 && aborted) atomicOr(err, kTcErrTimeout);
  if (nrm.in_sum) acc_in.flush(nrm.in_sum);
  if (nrm.out_sum) acc_out.flush(nrm.out_sum);
}

// Smallest dynamic shared memory that keeps (512 / TMEM columns) CTAs per SM at
// most, so tcgen05.alloc never waits for a CTA that only finishes at the end.
static size_t tc_smem_floor(uint32_t cols_per_cta) {
  const size_t per_sm = 233472;  // 228 KiB of shared memory per SM
  const uint32_t ctas = 512u / cols_per_cta;
  return per_sm / (ctas + 1) + 1024;
}

template <int NT, int R>
static cudaError_t launch_tc(float2 *amp, const uint8_t *plan, uint32_t off, const PlanPass &hp,
                             const RegPassParams &prm, int *err, cudaStream_t st, const TcNorm &nrm) {
  constexpr uint32_t cols = (NT / 128) * tc_cols_per_group(R);
  const TcLayout lay = tc_layout(hp.T, hp.n_stages, hp.data_bytes, R);
  size_t smem = lay.total;
  const size_t floor_ = tc_smem_floor(cols);
  if (smem < floor_) smem = floor_;
  if (smem + kTcStaticSmem > kSmemOptIn) return cudaErrorInvalidValue;
  static std::atomic<uint64_t> configured{0};
  static std::atomic<int> sms[64];
  static std::atomic<int> regs{0};
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = once_per_device(configured, sms, dev, [] {
    cudaError_t r = cudaFuncSetAttribute(k_pass_tc<NT, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(kSmemOptIn - kTcStaticSmem));
    // all of the SM's unified memory as shared memory, so the occupancy below
    // (and the launch) can place two ~110 KB CTAs per SM
    if (r == cudaSuccess)
      r = cudaFuncSetAttribute(k_pass_tc<NT, R>, cudaFuncAttributePreferredSharedMemoryCarveout,
                               int(cudaSharedmemCarveoutMaxShared));
    cudaFuncAttributes fa{};
    if (r == cudaSuccess) r = cudaFuncGetAttributes(&fa, k_pass_tc<NT, R>);
    if (r == cudaSuccess) regs.store(fa.numRegs, std::memory_order_relaxed);
    return r;
  }, &nsm);
  if (e != cudaSuccess) return e;
  // CTAs per SM: shared memory (228 KiB per SM, 1 KiB reserved per CTA), tensor
  // memory (512 columns) and registers (the kernel's count, allocated in
  // 8-register steps).  The runtime's occupancy query is not used: it reported
  // one CTA per SM for ~108 KB CTAs that fit twice.
  const int nregs = std::max(8, (regs.load(std::memory_order_relaxed) + 7) & ~7);
  int per_sm = int(233472 / (smem + kTcStaticSmem + 1024));
  per_sm = std::min(per_sm, int(512 / cols));
  per_sm = std::min(per_sm, int(65536 / (NT * nregs)));
  if (per_sm < 1) per_sm = 1;
  if (nsm < 1) nsm = 1;
  const uint64_t want = uint64_t(nsm) * per_sm;
  const unsigned grid = unsigned(hp.n_tiles < want ? hp.n_tiles : want);
  k_pass_tc<NT, R><<<grid, NT, smem, st>>>(amp, plan, off, prm, err, nrm);
  count_launch();
  return cudaGetLastError();
}

bool tc_pass_fits(uint32_t T, uint32_t c, uint32_t n_stages, uint32_t data_bytes, uint32_t R) {
  if (R != 4 && R != 5) return false;
  if (T < R + 7 || T > R + (R == 4 ? 9 : 8) || T < c + R || c < 1 || n_stages < 1 ||
      n_stages > uint32_t(kMaxStages) || data_bytes > kMaxPassData)
    return false;
  return tc_layout(T, n_stages, data_bytes, R).total + kTcStaticSmem <= kSmemOptIn;
}

static size_t pass_smem(uint32_t T, uint32_t c, int kmax) {
  return (size_t(1) << T) * sizeof(float2) + (size_t(1) << (T - c)) * sizeof(uint64_t) +
         (size_t(1) << (2 * kmax)) * sizeof(float2) + 256 * sizeof(float2) + 64 * sizeof(uint32_t);
}

template <int KMAX>
static cudaError_t launch_k(float2 *amp, const uint8_t *plan, uint32_t off, const PlanPass &hp,
                            cudaStream_t st) {
  const size_t smem = pass_smem(hp.T, hp.c, KMAX);
  static std::atomic<uint64_t> configured{0};
  static std::atomic<int> sms[64];
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = once_per_device(configured, sms, dev, [] {
    return cudaFuncSetAttribute(k_pass<KMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(pass_smem(kMaxTile, 1, KMAX)));
  }, &nsm);
  if (e != cudaSuccess) return e;
  const uint64_t tiles = hp.n_tiles;
  dim3 grid;
  if (tiles <= (uint64_t(1) << 30)) {
    grid = dim3(unsigned(tiles), 1, 1);
  } else {
    grid = dim3(1u << 30, unsigned(tiles >> 30), 1);
  }
  k_pass<KMAX><<<grid, kNT, smem, st>>>(amp, plan, off);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_pass(float2 *amp, const uint8_t *plan_dev, uint32_t pass_off,
                        const PlanPass &hp, const RegPassParams *prm, int *err, cudaStream_t stream,
                        const TcNorm *norm) {
  if (hp.kind == KIND_TC) {
    if (!prm || !err) return cudaErrorInvalidValue;
    const TcNorm nrm = norm ? *norm : TcNorm{};
    if (hp.R == 4) {
      if (hp.T == 11) return launch_tc<128, 4>(amp, plan_dev, pass_off, hp, *prm, err, stream, nrm);
      if (hp.T == 12) return launch_tc<256, 4>(amp, plan_dev, pass_off, hp, *prm, err, stream, nrm);
      if (hp.T == 13) return launch_tc<512, 4>(amp, plan_dev, pass_off, hp, *prm, err, stream, nrm);
    } else if (hp.R == 5) {
      if (hp.T == 12) return launch_tc<128, 5>(amp, plan_dev, pass_off, hp, *prm, err, stream, nrm);
      if (hp.T == 13) return launch_tc<256, 5>(amp, plan_dev, pass_off, hp, *prm, err, stream, nrm);
    }
    return cudaErrorInvalidValue;
  }
  if (hp.kind == KIND_REG) {
    if (!prm || !err) return cudaErrorInvalidValue;
    if (hp.R == 5) {
      if (hp.T <= 12) return launch_reg<5, 128>(amp, plan_dev, pass_off, hp, *prm, err, stream);
      return launch_reg<5, 256>(amp, plan_dev, pass_off, hp, *prm, err, stream);
    }
    if (hp.R != 4) return cudaErrorInvalidValue;
    if (hp.T <= 12) return launch_reg<4, 256>(amp, plan_dev, pass_off, hp, *prm, err, stream);
    return launch_reg<4, 512>(amp, plan_dev, pass_off, hp, *prm, err, stream);
  }
  switch (hp.kmax) {
    case 0:
    case 1: return launch_k<1>(amp, plan_dev, pass_off, hp, stream);
    case 2: return launch_k<2>(amp, plan_dev, pass_off, hp, stream);
    case 3: return launch_k<3>(amp, plan_dev, pass_off, hp, stream);
    case 4: return launch_k<4>(amp, plan_dev, pass_off, hp, stream);
    default: return launch_k<5>(amp, plan_dev, pass_off, hp, stream);
  }
}

}  // namespace svgb
