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


// ---------------------------------------------------------------------------
// register stages
// ---------------------------------------------------------------------------

__host__ __device__ constexpr int popc_c(int m) { return m ? (m & 1) + popc_c(m >> 1) : 0; }

// deposit the bits of j into the set bits of mask (ascending)
__host__ __device__ constexpr int dep_c(int j, int mask) {
  int out = 0, bit = 0;
  for (int p = 0; p < 8; p++)
    if ((mask >> p) & 1) {
      if ((j >> bit) & 1) out |= 1 << p;
      bit++;
    }
  return out;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// out = sum_j M[r][j] x[j] for one output row, element (a + ib) stored as
// (a, a, -b, b): each complex product-accumulate is two paired FMAs,
// (a, a) * (x.re, x.im) + (-b, b) * (x.im, x.re).
template <int KK>
__device__ __forceinline__ float2 row_dot(const float4 (&e)[KK], const float2 (&x)[KK]) {
  float2 o = __fmul2_rn(make_float2(e[0].x, e[0].y), x[0]);
  o = __ffma2_rn(make_float2(e[0].z, e[0].w), make_float2(x[0].y, x[0].x), o);
#pragma unroll
  for (int j = 1; j < KK; j++) {
    o = __ffma2_rn(make_float2(e[j].x, e[j].y), x[j], o);
    o = __ffma2_rn(make_float2(e[j].z, e[j].w), make_float2(x[j].y, x[j].x), o);
  }
  return o;
}

// acc[g] (+)= M[r][j] x_g[j] for every group g of the thread, loop over j
// outermost so consecutive paired FMAs belong to independent chains.
// Element (a + ib) is stored as (a, a, -b, b): each complex product-accumulate
// is two paired FMAs, (a, a) * (x.re, x.im) + (-b, b) * (x.im, x.re).
template <int R, int MASK, int ROW>
__device__ __forceinline__ void rows_all_groups(const float2 (&v)[1 << R], const float4 (&e)[1 << popc_c(MASK)],
                                                float2 (&acc)[(1 << R) >> popc_c(MASK)]) {
  constexpr int KK = 1 << popc_c(MASK);
#pragma unroll
  for (int j = 0; j < KK; j++) {
    int gi = 0;
#pragma unroll
    for (int g = 0; g < (1 << R); g++) {
      if (g & MASK) continue;
      const float2 x = v[g | dep_c(j, MASK)];
      if (j == 0) acc[gi] = __fmul2_rn(make_float2(e[0].x, e[0].y), x);
      else acc[gi] = __ffma2_rn(make_float2(e[j].x, e[j].y), x, acc[gi]);
      acc[gi] = __ffma2_rn(make_float2(e[j].z, e[j].w), make_float2(x.y, x.x), acc[gi]);
      gi++;
    }
  }
}

// Dense block on the register positions in MASK (matrix bit i <-> i-th set bit).
// Blocks of one and two qubits take the matrix one or two rows at a time and
// apply them to every group of the thread at once (independent FMA chains);
// outputs wait in registers until every row has read the group's inputs.
// Wider blocks read each row from shared memory per group.
template <int R, int MASK>
__device__ __forceinline__ void reg_dense(float2 (&v)[1 << R], const float4 *__restrict__ m) {
  constexpr int K = popc_c(MASK);
  constexpr int KK = 1 << K;
  constexpr int NG = (1 << R) / KK;
  if constexpr (K == 1) {
    float4 e0[2], e1[2];
    e0[0] = m[0]; e0[1] = m[1]; e1[0] = m[2]; e1[1] = m[3];
    float2 t0[NG], t1[NG];
    rows_all_groups<R, MASK, 0>(v, e0, t0);
    rows_all_groups<R, MASK, 1>(v, e1, t1);
    int gi = 0;
#pragma unroll
    for (int g = 0; g < (1 << R); g++) {
      if (g & MASK) continue;
      v[g | dep_c(0, MASK)] = t0[gi];
      v[g | dep_c(1, MASK)] = t1[gi];
      gi++;
    }
  } else if constexpr (K == 2) {
    float2 t0[NG], t1[NG], t2[NG], t3[NG];
    {
      asm volatile("" ::: "memory");
      float4 e0[4], e1[4];
#pragma unroll
      for (int j = 0; j < 4; j++) {
        e0[j] = m[j];
        e1[j] = m[4 + j];
      }
      rows_all_groups<R, MASK, 0>(v, e0, t0);
      rows_all_groups<R, MASK, 1>(v, e1, t1);
    }
    {
      asm volatile("" ::: "memory");
      float4 e2[4], e3[4];
#pragma unroll
      for (int j = 0; j < 4; j++) {
        e2[j] = m[8 + j];
        e3[j] = m[12 + j];
      }
      rows_all_groups<R, MASK, 2>(v, e2, t2);
      rows_all_groups<R, MASK, 3>(v, e3, t3);
    }
    int gi = 0;
#pragma unroll
    for (int g = 0; g < (1 << R); g++) {
      if (g & MASK) continue;
      v[g | dep_c(0, MASK)] = t0[gi];
      v[g | dep_c(1, MASK)] = t1[gi];
      v[g | dep_c(2, MASK)] = t2[gi];
      v[g | dep_c(3, MASK)] = t3[gi];
      gi++;
    }
  } else {
#pragma unroll
    for (int g = 0; g < (1 << R); g++) {
      if (g & MASK) continue;
      float2 x[KK];
#pragma unroll
      for (int j = 0; j < KK; j++) x[j] = v[g | dep_c(j, MASK)];
#pragma unroll
      for (int r = 0; r < KK; r++) {
        asm volatile("" ::: "memory");
        float4 e[KK];
#pragma unroll
        for (int j = 0; j < KK; j++) e[j] = m[r * KK + j];
        v[g | dep_c(r, MASK)] = row_dot<KK>(e, x);
      }
    }
  }
}

#define SV_CASE(M) \
  case M: if constexpr ((M) < (1 << R) && popc_c(M) <= (R == 5 ? 2 : 4)) reg_dense<R, (M)>(v, m); break;

template <int R>
__device__ __forceinline__ void reg_dense_dispatch(float2 (&v)[1 << R], uint32_t mask,
                                                   const float4 *__restrict__ m) {
  switch (mask) {
    SV_CASE(1) SV_CASE(2) SV_CASE(3) SV_CASE(4) SV_CASE(5) SV_CASE(6) SV_CASE(7)
    SV_CASE(8) SV_CASE(9) SV_CASE(10) SV_CASE(11) SV_CASE(12) SV_CASE(13) SV_CASE(14) SV_CASE(15)
    SV_CASE(16) SV_CASE(17) SV_CASE(18) SV_CASE(19) SV_CASE(20) SV_CASE(21) SV_CASE(22) SV_CASE(23)
    SV_CASE(24) SV_CASE(25) SV_CASE(26) SV_CASE(27) SV_CASE(28) SV_CASE(29) SV_CASE(30) SV_CASE(31)
    default: break;
  }
}
#undef SV_CASE

// exp(2*pi*i * sum of the turns of terms [i0, i1) that apply to this thread)
__device__ __forceinline__ float2 rphase_exp(const RegPhaseTerm *__restrict__ t, uint32_t i0, uint32_t i1,
                                             uint64_t base, uint32_t LB) {
  uint32_t a = 0;
  for (uint32_t i = i0; i < i1; i++) {
    const RegPhaseTerm x = t[i];
    if ((base & x.outer_mask) == x.outer_mask && (LB & x.tmask) == x.tmask) a += x.turn;
  }
  if (a == 0) return make_float2(1.f, 0.f);
  float sn, cs;
  sincospif(static_cast<float>(static_cast<int32_t>(a)) * 4.656612873077393e-10f, &sn, &cs);
  return make_float2(cs, sn);
}

template <int J>
struct LowBit {
  static constexpr int v = (J & 1) ? 0 : 1 + LowBit<(J >> 1)>::v;
};
template <>
struct LowBit<0> {
  static constexpr int v = 0;
};

// f[j] = f[j without its lowest bit] * e[1 + lowest bit of j], j = J .. 2^R - 1
template <int J, int R>
__device__ __forceinline__ void phase_tree(float2 (&f)[1 << R], const float2 (&e)[R + 1]) {
  if constexpr (J < (1 << R)) {
    f[J] = cmul(f[J & (J - 1)], e[1 + LowBit<J>::v]);
    phase_tree<J + 1, R>(f, e);
  }
}

// OP_RPHASE on the 2^R register amplitudes of one thread (record layout in
// RegPhaseHdr).  The thread sums the turns of the terms that apply to it into
// P and alpha_i (exact modulo 2^32), takes the 1 + R exponentials, and forms
// the 2^R amplitude phases as products along a binary tree (at most R complex
// products deep), times D[j].
template <int R>
__device__ __forceinline__ void reg_rphase(float2 (&v)[1 << R], const uint8_t *__restrict__ rec, uint64_t base,
                                           uint32_t LB) {
  const RegPhaseHdr *h = reinterpret_cast<const RegPhaseHdr *>(rec);
  const RegPhaseTerm *t = reinterpret_cast<const RegPhaseTerm *>(rec + sizeof(RegPhaseHdr));
  float2 e[R + 1];
#pragma unroll
  for (int k = 0; k <= R; k++) {
    const uint32_t i0 = k ? h->end[k - 1] : 0u, i1 = h->end[k];
    e[k] = rphase_exp(t, i0, i1, base, LB);
  }
  const bool has_d = h->has_d != 0;
  // f[j] = e[0] * prod_{bit i of j} e[1 + i], built from f[j without its lowest bit]
  float2 f[1 << R];
  f[0] = e[0];
  phase_tree<1, R>(f, e);
#pragma unroll
  for (int j = 0; j < (1 << R); j++) {
    float2 p = f[j];
    if (has_d) p = cmul(p, h->d[j]);
    v[j] = cmul(v[j], p);
  }
}

// Persistent register-stage kernel.  Every CTA copies its pass's records
// (ops, matrices, phase terms, stages) into shared memory once, builds the
// per-thread stage index tables once, then walks tiles blockIdx.x,
// blockIdx.x + gridDim.x, ...  The next tile's amplitudes stream into shared
// memory with cp.async while the current one is computed (into `buf_in` with
// 16 amplitudes per thread; with 32, into the exchange buffer `buf_x` during the
// last stage, which no longer needs it); stage 0 reads them in natural order
// (its lanes are the low tile bits), later stages exchange through the
// swizzled `buf_x`, and the last stage stores straight to HBM.
constexpr int kMaxStages = 64;     // stage tables kept in shared memory
constexpr int kPlanMismatch = 2;   // error word bit: a pass's device records differ from the host's
constexpr uint32_t kMaxPassData = 160 * 1024;

struct RegLayout {
  uint32_t L, nseg, NT, ns;
  size_t off_in, off_x, off_seg, off_tt, off_data, total;
};

// KIND_REG passes with 32 amplitudes per thread keep no separate prefetch buffer:
// the next tile is prefetched into the exchange buffer during the last stage, so
// four CTAs fit an SM.  Register passes keep no segment table.
__host__ __device__ constexpr bool reg_shared_prefetch(uint32_t R) { return R == 5; }

__host__ __device__ inline RegLayout reg_layout(uint32_t T, uint32_t c, uint32_t ns, uint32_t data_bytes,
                                                uint32_t R = 4, bool reg = false) {
  RegLayout r;
  r.L = 1u << T;
  r.nseg = 1u << (T - c);
  r.NT = 1u << (T - R);
  r.ns = ns;
  size_t o = 0;
  r.off_in = o;
  if (!(reg && reg_shared_prefetch(R))) o += size_t(r.L) * 8;
  r.off_x = o; o += size_t(r.L) * 8;
  r.off_seg = o;
  if (!reg) o += size_t(r.nseg) * 8;
  r.off_tt = o; o += size_t(ns) * r.NT * 4;
  o = (o + 15) & ~size_t(15);
  r.off_data = o; o += data_bytes;
  r.total = (o + 15) & ~size_t(15);
  return r;
}

// 16 amplitudes per thread (blocks up to 4 qubits): two CTAs of 256 threads
// per SM; 32 amplitudes per thread (blocks up to 2 qubits): four CTAs of 128
// threads per SM (128 registers a thread).
template <int R, int NTMAX>
__global__ void __launch_bounds__(NTMAX, R == 5 ? (NTMAX <= 128 ? 4 : 2) : (NTMAX <= 256 ? 2 : 1))
    k_pass_reg(float2 *__restrict__ amp, const uint8_t *__restrict__ plan, uint32_t pass_off,
               const __grid_constant__ RegPassParams prm, int *__restrict__ err) {
  constexpr int NR = 1 << R;
  extern __shared__ __align__(16) unsigned char smem[];
  const PlanPass *P = reinterpret_cast<const PlanPass *>(plan + pass_off);
  const uint32_t T = P->T, c = P->c;
  const uint32_t ns = P->n_stages;
  const uint32_t data_off = P->ops_off, data_bytes = P->data_bytes;
  const uint64_t outer_mask = P->outer_mask, n_tiles = P->n_tiles;
  // the launch's shared memory was sized from the host's copy of these fields
  if (T != prm.chk[0] || ns != prm.chk[1] || data_bytes != prm.chk[2] || data_off != prm.chk[3] ||
      P->R != uint32_t(R) || ns == 0 || ns > uint32_t(kMaxStages)) {
    if (threadIdx.x == 0) atomicOr(err, kPlanMismatch);
    return;
  }
  constexpr bool kShared = reg_shared_prefetch(R);
  const RegLayout lay = reg_layout(T, c, ns, data_bytes, R, true);
  float2 *buf_in = reinterpret_cast<float2 *>(smem + lay.off_in);
  float2 *buf_x = reinterpret_cast<float2 *>(smem + lay.off_x);
  uint32_t *tt = reinterpret_cast<uint32_t *>(smem + lay.off_tt);
  uint8_t *data = smem + lay.off_data;
  const uint32_t tid = threadIdx.x, NT = blockDim.x;

  // pass records -> shared memory (offsets below are relative to ops_off)
  {
    const uint4 *src = reinterpret_cast<const uint4 *>(plan + data_off);
    uint4 *dst = reinterpret_cast<uint4 *>(data);
    for (uint32_t i = tid; i < data_bytes / 16; i += NT) dst[i] = src[i];
  }
  const uint64_t hm = P->high_mask;
  __syncthreads();
  const StageRec *stages = reinterpret_cast<const StageRec *>(data + (P->stages_off - data_off));
  const OpRec *ops = reinterpret_cast<const OpRec *>(data);
  // per-thread stage tables: low 16 bits = local index part, high 16 = swizzled
  for (uint32_t s = 0; s < ns; s++) {
    uint32_t LB = 0;
    for (uint32_t i = 0; i < T - R; i++)
      if ((tid >> i) & 1u) LB |= 1u << stages[s].tb[i];
    tt[s * NT + tid] = LB | (swz(LB) << 16);
  }
  const uint32_t cs = c - 1u, cmask = (1u << cs) - 1u;
  constexpr int NK = NR / 2;  // 16-byte chunks per thread per tile
  const uint32_t sin = static_cast<uint32_t>(__cvta_generic_to_shared(buf_in));
  const uint32_t sx = static_cast<uint32_t>(__cvta_generic_to_shared(buf_x));
  // tile-invariant per-thread parts of the addresses
  const uint32_t t_ld = sin + (tt[tid] & 0xffffu) * 8u;
  uint64_t t_st = 0;
  {
    const uint32_t LB = tt[(ns - 1) * NT + tid] & 0xffffu;
    for (uint32_t x = 0; x < T; x++)
      if ((LB >> x) & 1u) t_st |= uint64_t(1) << prm.oq[x];
  }
  const uint64_t t_cp = pdep_u64(tid >> cs, hm) + (uint64_t(tid & cmask) << 1);

  // 32-amplitude passes prefetch the next tile into the exchange buffer while
  // their last stage computes (the buffer is free once the last exchange is read)
  const uint32_t t_ldx = (tt[tid] & 0xffffu) * 8u;
  uint64_t tile = blockIdx.x;
  uint64_t base = tile < n_tiles ? pdep_u64(tile, outer_mask) : 0;
  if (tile < n_tiles) {
    const uint32_t dst = kShared ? sx : sin;
#pragma unroll
    for (int k = 0; k < NK; k++) cp_async16_s(dst + (tid + k * NT) * 16u, amp + base + t_cp + prm.ko[k]);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  __syncthreads();

  float2 v[NR];
  while (tile < n_tiles) {
    const uint64_t next = tile + gridDim.x;
    const uint64_t base_next = next < n_tiles ? pdep_u64(next, outer_mask) : 0;
    if constexpr (kShared) {
      asm volatile("cp.async.wait_all;\n" ::: "memory");
      __syncthreads();
#pragma unroll
      for (int j = 0; j < NR; j++) v[j] = lds64(sx + t_ldx + prm.lo[j]);
    } else {
      asm volatile("cp.async.wait_all;\n" ::: "memory");
      __syncthreads();
#pragma unroll
      for (int j = 0; j < NR; j++) v[j] = lds64(t_ld + prm.lo[j]);
      __syncthreads();  // buf_in is free: prefetch the next tile
      if (next < n_tiles) {
#pragma unroll
        for (int k = 0; k < NK; k++) cp_async16_s(sin + (tid + k * NT) * 16u, amp + base_next + t_cp + prm.ko[k]);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
      }
    }
    for (uint32_t s = 0; s < ns; s++) {
      const StageRec &st = stages[s];
      const uint32_t w = tt[s * NT + tid];
      const uint32_t LB = w & 0xffffu;
      if (s > 0) {
        const StageRec &pv = stages[s - 1];
        const uint32_t PBp = (tt[(s - 1) * NT + tid] >> 16) * 8u, PB = (w >> 16) * 8u;
        uint32_t xo[NR];
        const uint4 *q = reinterpret_cast<const uint4 *>(pv.xo);
#pragma unroll
        for (int j = 0; j < NR / 4; j++) {
          const uint4 t4 = q[j];
          xo[4 * j] = t4.x; xo[4 * j + 1] = t4.y; xo[4 * j + 2] = t4.z; xo[4 * j + 3] = t4.w;
        }
        // A thread writes its amplitudes back to exactly the positions it read
        // them from at stage s - 1, which no other thread reads, so only the first
        // exchange after a stage-0 read of the natural-order tile from this same
        // buffer (32-amplitude passes) must wait for every thread's reads.
        if (kShared && s == 1) __syncthreads();
#pragma unroll
        for (int j = 0; j < NR; j++) sts64(sx + (xo[j] ^ PBp), v[j]);
        q = reinterpret_cast<const uint4 *>(st.xo);
#pragma unroll
        for (int j = 0; j < NR / 4; j++) {
          const uint4 t4 = q[j];
          xo[4 * j] = t4.x; xo[4 * j + 1] = t4.y; xo[4 * j + 2] = t4.z; xo[4 * j + 3] = t4.w;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < NR; j++) v[j] = lds64(sx + (xo[j] ^ PB));
      }
      if (kShared && s + 1 == ns) {
        __syncthreads();  // every thread has read the exchange buffer
        if (next < n_tiles) {
#pragma unroll
          for (int k = 0; k < NK; k++) cp_async16_s(sx + (tid + k * NT) * 16u, amp + base_next + t_cp + prm.ko[k]);
          asm volatile("cp.async.commit_group;\n" ::: "memory");
        }
      }
      const uint32_t oe = st.op_end;
      for (uint32_t o = st.op_begin; o < oe; o++) {
        const OpRec op = ops[o];
        if (op.type == OP_DENSE) {
          reg_dense_dispatch<R>(v, op.rmask, reinterpret_cast<const float4 *>(data + (op.data_off - data_off)));
        } else {
          reg_rphase<R>(v, data + (op.data_off - data_off), base, LB);
        }
      }
    }
    {
      float2 *dst = amp + base + t_st;
#pragma unroll
      for (int j = 0; j < NR; j++) __stcs(dst + prm.go[j], v[j]);
    }
    tile = next;
    base = base_next;
  }
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
// tensor-core stages (KIND_TC): the register-stage skeleton with 16 amplitudes
// per thread (R = 4) and each stage's dense blocks applied as one 3xTF32
// tcgen05 product (sv_tc.cu).  Per stage and 128-row group, the threads split
// their rows into A_hi / A_lo in tensor memory, one thread of the group issues
// the stage's 8 MMAs and commits them to the group's mbarrier, and the group
// reads D back.  Between stages the tile moves through one swizzled exchange
// buffer with one CTA barrier per exchange: a thread writes its amplitudes back
// to exactly the positions it read them from at the previous stage, which no
// other thread reads, so no barrier is needed before the writes.  The next tile
// is prefetched (16-byte cp.async, natural order) into a separate load buffer as
// soon as every thread has read the current tile from it (the first exchange's
// barrier), so the load overlaps most of the tile's stages.  Passes of unitary ops (kPassUnitary) restore each
// tile's norm before the store: the exact pass keeps it, and the tensor cores'
// float32 accumulation rounds toward zero, which would otherwise shrink the
// state by ~1e-7 per stage.
// ---------------------------------------------------------------------------

constexpr int kTcErrTimeout = 1;
constexpr size_t kTcStaticSmem = 1024;  // mbarriers and the TMEM base (the static region's size)

struct TcLayout {
  uint32_t L, NT;
  size_t off_in, off_x, off_red, off_tt, off_data, total;
};

__host__ __device__ inline TcLayout tc_layout(uint32_t T, uint32_t ns, uint32_t data_bytes) {
  TcLayout r;
  r.L = 1u << T;
  r.NT = 1u << (T - 4);
  size_t o = 0;
  r.off_in = o; o += size_t(r.L) * 8;  // load buffer (natural order)
  r.off_x = o; o += size_t(r.L) * 8;   // exchange buffer (swizzled)
  r.off_red = o; o += size_t(r.NT / 32) * 8;  // per warp: the tile-norm partials
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

template <int NT>
__global__ void __launch_bounds__(NT, NT <= 128 ? 3 : (NT <= 256 ? 2 : 1))
    k_pass_tc(float2 *__restrict__ amp, const uint8_t *__restrict__ plan, uint32_t pass_off,
              const __grid_constant__ RegPassParams prm, int *__restrict__ err) {
  constexpr int NR = 16;  // R = 4 register qubits
  constexpr uint32_t kT = NT == 128 ? 11u : (NT == 256 ? 12u : 13u);
  constexpr uint32_t NW = NT / 32, NG = NT / 128;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar[NG];
  __shared__ uint32_t tbase_s;
  const PlanPass *P = reinterpret_cast<const PlanPass *>(plan + pass_off);
  const uint32_t T = P->T, c = P->c, ns = P->n_stages;
  const uint32_t data_off = P->ops_off, data_bytes = P->data_bytes;
  const uint64_t outer_mask = P->outer_mask, n_tiles = P->n_tiles;
  const bool unitary = (P->flags & kPassUnitary) != 0u;
  // the launch's shared memory was sized from the host's copy of these fields
  if (T != kT || T != prm.chk[0] || ns != prm.chk[1] || data_bytes != prm.chk[2] || data_off != prm.chk[3] ||
      P->R != 4u || P->kind != KIND_TC || ns == 0 || ns > uint32_t(kMaxStages)) {
    if (threadIdx.x == 0) atomicOr(err, kPlanMismatch);
    return;
  }
  const TcLayout lay = tc_layout(T, ns, data_bytes);
  uint32_t *tt = reinterpret_cast<uint32_t *>(smem + lay.off_tt);
  float2 *red = reinterpret_cast<float2 *>(smem + lay.off_red);
  uint8_t *data = smem + lay.off_data;
  const uint32_t tid = threadIdx.x, warp = tid >> 5, g = tid >> 7;

  {
    const uint4 *src = reinterpret_cast<const uint4 *>(plan + data_off);
    uint4 *dst = reinterpret_cast<uint4 *>(data);
    for (uint32_t i = tid; i < data_bytes / 16; i += NT) dst[i] = src[i];
  }
  fence_proxy_async_smem();  // stage images are read by the tensor cores
  if (warp == 0) {
    tmem_alloc(&tbase_s, NT);  // 128 columns per row group
    tmem_relinquish();
  }
  if (tid < NG) mbar_init(&bar[tid], 1);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const StageRec *stages = reinterpret_cast<const StageRec *>(data + (P->stages_off - data_off));
  const OpRec *ops = reinterpret_cast<const OpRec *>(data);
  // per-thread stage tables (own entries only): low 16 bits local index part, high 16 swizzled
  for (uint32_t s = 0; s < ns; s++) {
    uint32_t LB = 0;
    for (uint32_t i = 0; i < T - 4; i++)
      if ((tid >> i) & 1u) LB |= 1u << stages[s].tb[i];
    tt[s * NT + tid] = LB | (swz(LB) << 16);
  }
  const uint64_t hm = P->high_mask;
  const uint32_t cs = c - 1u, cmask = (1u << cs) - 1u;
  constexpr int NK = NR / 2;  // 16-byte chunks per thread per tile
  const uint32_t sin = smem_u32(smem + lay.off_in), sx = smem_u32(smem + lay.off_x);
  const uint32_t tbase = tbase_s;
  const uint32_t gcols = tbase + g * kTcColsPerGroup;
  const uint32_t tq = gcols + (((warp & 3u) * 32u) << 16);  // this thread's lane
  const uint32_t t_ldx = (tt[tid] & 0xffffu) * 8u;
  uint64_t t_st = 0;
  {
    const uint32_t LB = tt[(ns - 1) * NT + tid] & 0xffffu;
    for (uint32_t x = 0; x < T; x++)
      if ((LB >> x) & 1u) t_st |= uint64_t(1) << prm.oq[x];
  }
  const uint64_t t_cp = pdep_u64(tid >> cs, hm) + (uint64_t(tid & cmask) << 1);

  uint64_t tile = blockIdx.x;
  uint64_t base = tile < n_tiles ? pdep_u64(tile, outer_mask) : 0;
  if (tile < n_tiles) {
#pragma unroll
    for (int k = 0; k < NK; k++) cp_async16_s(sin + (tid + k * NT) * 16u, amp + base + t_cp + prm.ko[k]);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  uint32_t parity = 0;
  bool bad = false, aborted = false;
  float2 v[NR];
  while (tile < n_tiles) {
    const uint64_t next = tile + gridDim.x;
    const uint64_t base_next = next < n_tiles ? pdep_u64(next, outer_mask) : 0;
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    if (__syncthreads_or(bad)) {  // the tile has landed; the previous tile is done
      aborted = true;
      break;
    }
#pragma unroll
    for (int j = 0; j < NR; j++) v[j] = lds64(sin + t_ldx + prm.lo[j]);
    float2 nin = make_float2(0.f, 0.f);
    if (unitary) {
#pragma unroll
      for (int j = 0; j < NR; j++) nin = __ffma2_rn(v[j], v[j], nin);
    }
    if (ns == 1) {  // no exchange barrier: make sure every thread has read the load buffer
      if (__syncthreads_or(bad)) {
        aborted = true;
        break;
      }
      if (next < n_tiles) {
#pragma unroll
        for (int k = 0; k < NK; k++) cp_async16_s(sin + (tid + k * NT) * 16u, amp + base_next + t_cp + prm.ko[k]);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
      }
    }
    for (uint32_t s = 0; s < ns; s++) {
      const StageRec &st = stages[s];
      const uint32_t w = tt[s * NT + tid];
      const uint32_t LB = w & 0xffffu;
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
        if (__syncthreads_or(bad)) {
          aborted = true;
          break;
        }
        if (s == 1 && next < n_tiles) {  // every thread has read the load buffer at stage 0
#pragma unroll
          for (int k = 0; k < NK; k++)
            cp_async16_s(sin + (tid + k * NT) * 16u, amp + base_next + t_cp + prm.ko[k]);
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
        store_row_split(tq, v);
        tmem_wait_st();
        tc_fence_before();
        group_bar_sync(g);  // the group's rows are in tensor memory
        if ((tid & 127u) == 0) {  // one thread issues, commits and waits; the others block
          tc_fence_after();
          issue_stage_mma(gcols, smem_u32(data + (st.b_off - data_off)));
          mma_commit(&bar[g]);
          if (!mbar_wait_bounded(&bar[g], parity)) bad = true;
        }
        parity ^= 1u;
        group_bar_sync(g);  // the product is in tensor memory
        tc_fence_after();
        load_row_sum(tq, v);
      }
      const uint32_t oe = st.op_end;
      for (uint32_t o = st.op_begin; o < oe; o++) {
        const OpRec op = ops[o];
        reg_rphase<4>(v, data + (op.data_off - data_off), base, LB);
      }
    }
    if (aborted) break;
    if (unitary) {
      float2 nout = make_float2(0.f, 0.f);
#pragma unroll
      for (int j = 0; j < NR; j++) nout = __ffma2_rn(v[j], v[j], nout);
      float a = nin.x + nin.y, b = nout.x + nout.y;
#pragma unroll
      for (int m = 16; m > 0; m >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, m);
        b += __shfl_xor_sync(0xffffffffu, b, m);
      }
      if ((tid & 31u) == 0) red[warp] = make_float2(a, b);
      if (__syncthreads_or(bad)) {
        aborted = true;
        break;
      }
      float si = 0.f, so = 0.f;
#pragma unroll
      for (uint32_t x = 0; x < NW; x++) {
        const float2 r = red[x];
        si += r.x;
        so += r.y;
      }
      if (si > 0.f && so > 0.f) {
        const float sc = sqrtf(__fdiv_rn(si, so));
        const float2 s2 = make_float2(sc, sc);
#pragma unroll
        for (int j = 0; j < NR; j++) v[j] = __fmul2_rn(v[j], s2);
      }
    }
    {
      float2 *dst = amp + base + t_st;
#pragma unroll
      for (int j = 0; j < NR; j++) __stcs(dst + prm.go[j], v[j]);
    }
    tile = next;
    base = base_next;
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tbase, NT);
  if (tid == 0 && aborted) atomicOr(err, kTcErrTimeout);
}

// Smallest dynamic shared memory that keeps (512 / TMEM columns) CTAs per SM at
// most, so tcgen05.alloc never waits for a CTA that only finishes at the end.
static size_t tc_smem_floor(uint32_t nt) {
  const size_t per_sm = 233472;  // 228 KiB of shared memory per SM
  const uint32_t ctas = 512u / nt;  // TMEM columns per CTA = nt
  return per_sm / (ctas + 1) + 1024;
}

template <int NT>
static cudaError_t launch_tc(float2 *amp, const uint8_t *plan, uint32_t off, const PlanPass &hp,
                             const RegPassParams &prm, int *err, cudaStream_t st) {
  const TcLayout lay = tc_layout(hp.T, hp.n_stages, hp.data_bytes);
  size_t smem = lay.total;
  const size_t floor_ = tc_smem_floor(NT);
  if (smem < floor_) smem = floor_;
  if (smem + kTcStaticSmem > kSmemOptIn) return cudaErrorInvalidValue;
  static std::atomic<uint64_t> configured{0};
  static std::atomic<int> sms[64];
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = once_per_device(configured, sms, dev, [] {
    cudaError_t r = cudaFuncSetAttribute(k_pass_tc<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(kSmemOptIn - kTcStaticSmem));
    // all of the SM's unified memory as shared memory, so the occupancy below
    // (and the launch) can place two ~110 KB CTAs per SM
    if (r == cudaSuccess)
      r = cudaFuncSetAttribute(k_pass_tc<NT>, cudaFuncAttributePreferredSharedMemoryCarveout,
                               int(cudaSharedmemCarveoutMaxShared));
    return r;
  }, &nsm);
  if (e != cudaSuccess) return e;
  // CTAs per SM: shared memory (228 KiB per SM, 1 KiB reserved per CTA), tensor
  // memory (512 columns, NT per CTA) and registers (128 per thread).  The
  // runtime's occupancy query is not used: it reported one CTA per SM for ~108 KB
  // CTAs that fit twice.
  int per_sm = int(233472 / (smem + kTcStaticSmem + 1024));
  per_sm = std::min(per_sm, int(512 / NT));
  per_sm = std::min(per_sm, int(65536 / (NT * 128)));
  if (per_sm < 1) per_sm = 1;
  if (nsm < 1) nsm = 1;
  const uint64_t want = uint64_t(nsm) * per_sm;
  const unsigned grid = unsigned(hp.n_tiles < want ? hp.n_tiles : want);
  k_pass_tc<NT><<<grid, NT, smem, st>>>(amp, plan, off, prm, err);
  count_launch();
  return cudaGetLastError();
}

bool tc_pass_fits(uint32_t T, uint32_t c, uint32_t n_stages, uint32_t data_bytes) {
  if (T < 11 || T > 13 || T < c + 4 || c < 1 || n_stages < 1 || n_stages > uint32_t(kMaxStages) ||
      data_bytes > kMaxPassData)
    return false;
  return tc_layout(T, n_stages, data_bytes).total + kTcStaticSmem <= kSmemOptIn;
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
                        const PlanPass &hp, const RegPassParams *prm, int *err, cudaStream_t stream) {
  if (hp.kind == KIND_TC) {
    if (!prm || !err) return cudaErrorInvalidValue;
    if (hp.T == 11) return launch_tc<128>(amp, plan_dev, pass_off, hp, *prm, err, stream);
    if (hp.T == 12) return launch_tc<256>(amp, plan_dev, pass_off, hp, *prm, err, stream);
    if (hp.T == 13) return launch_tc<512>(amp, plan_dev, pass_off, hp, *prm, err, stream);
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
