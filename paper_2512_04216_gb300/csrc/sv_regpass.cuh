// sv_regpass.cuh -- register-stage pass machinery (KIND_REG, see sv_internal.h):
// in-register dense blocks with paired FMAs, register phase ops, the
// shared-memory layout of a register pass, and its tile loop.  Used by the
// single-state pass kernel (sv_apply.cu) and by the batched kernel for states
// kept in the global arena (sv_batch.cu).
#pragma once

#include <cstdint>

#include "sv_device.cuh"
#include "sv_internal.h"

namespace svgb {

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

// exp(2*pi*i * a / 2^32)
__device__ __forceinline__ float2 turn_exp(uint32_t a) {
  if (a == 0) return make_float2(1.f, 0.f);
  float sn, cs;
  sincospif(static_cast<float>(static_cast<int32_t>(a)) * 4.656612873077393e-10f, &sn, &cs);
  return make_float2(cs, sn);
}

// Whether a pass's outer-term slot table lies inside its records (its scratch
// and terms included: the kernels keep term indices below the records' end).
__device__ __forceinline__ bool w_table_ok(const PlanPass *P) {
  const uint32_t n = P->n_w, o = P->w_off - P->ops_off;
  return n == 0 || (P->w_off >= P->ops_off && (o & 15u) == 0 && n <= 4096u && o + rphase_w_terms(n) <= P->data_bytes);
}

// The per-tile sums of a pass's outer-term slots (RegPhaseSlot) for the tile
// at `base`, into `sums` (n_w words): warp w takes slots w, w + nwarps, ...,
// its lanes the slot's terms; sums wrap modulo 2^32.  `w` is the table in the
// records' copy, `w_bytes` the bytes from it to the records' end (term indices
// beyond them are not read).  Called by every thread of the CTA before the
// barrier that precedes the tile's first stage.
__device__ __forceinline__ void rphase_tile_sums(const uint8_t *__restrict__ w, uint32_t n_w, uint32_t w_bytes,
                                                 uint64_t base, uint32_t *sums) {
  const RegPhaseSlot *sl = reinterpret_cast<const RegPhaseSlot *>(w);
  const RegPhaseOuter *t = reinterpret_cast<const RegPhaseOuter *>(w + rphase_w_terms(n_w));
  const uint32_t lim = (w_bytes - rphase_w_terms(n_w)) / uint32_t(sizeof(RegPhaseOuter));
  const uint32_t lane = threadIdx.x & 31u, nw = blockDim.x >> 5;
  for (uint32_t s = threadIdx.x >> 5; s < n_w; s += nw) {
    const RegPhaseSlot r = sl[s];
    const uint32_t e = r.end < lim ? r.end : lim;
    uint32_t a = 0;
    for (uint32_t i = r.begin + lane; i < e; i += 32) {
      const RegPhaseOuter x = t[i];
      if ((base & x.outer_mask) == x.outer_mask) a += x.turn;
    }
    a = __reduce_add_sync(0xffffffffu, a);
    if (lane == 0) sums[s] = a;
  }
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

// OP_RPHASE on the 2^R register amplitudes of thread `tid` (record layout in
// RegPhaseHdr).  The thread adds its pre-summed turns of each class (terms on
// tile qubits) to the tile's sums of the terms on outer qubits (`sums`, this
// tile's half of the pass's scratch), takes the 1 + R exponentials, and forms
// the 2^R amplitude phases as products along a binary tree (at most R complex
// products deep), times D[j].
template <int R>
__device__ __forceinline__ void reg_rphase(float2 (&v)[1 << R], const uint8_t *__restrict__ rec,
                                           const uint32_t *__restrict__ sums, uint32_t tid) {
  const RegPhaseHdr *h = reinterpret_cast<const RegPhaseHdr *>(rec);
  const uint32_t *pre = reinterpret_cast<const uint32_t *>(rec + sizeof(RegPhaseHdr));
  const uint32_t pm = h->pre_mask, wu = h->w_used, nt = h->nt, ntb = h->ntb;
  const uint32_t *w = sums + h->w_slot;
  uint32_t a[R + 1];
#pragma unroll
  for (int k = 0; k <= R; k++)
    a[k] = ((pm >> k) & 1u) ? pre[uint32_t(__popc(pm & ((1u << k) - 1u))) * nt + tid] : 0u;
  if (wu & 1u) a[0] += w[0];
  if (wu & 2u)
    for (uint32_t i = 0; i < ntb; i++)
      if ((tid >> i) & 1u) a[0] += w[1 + i];
#pragma unroll
  for (int r = 0; r < R; r++)
    if ((wu >> (2 + r)) & 1u) a[1 + r] += w[1 + ntb + r];
  float2 e[R + 1];
#pragma unroll
  for (int k = 0; k <= R; k++) e[k] = turn_exp(a[k]);
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


// The tile loop of a KIND_REG pass (see k_pass_reg): this CTA takes tiles
// tile0, tile0 + tile_step, ...; `smem` holds the pass's shared-memory layout
// (reg_layout) and prm its address tables.  The caller has checked the pass
// record against prm.chk.
template <int R>
__device__ __forceinline__ void reg_pass_tiles(float2 *__restrict__ amp, const uint8_t *__restrict__ plan,
                                               const PlanPass *P, const RegPassParams &prm, unsigned char *smem,
                                               uint64_t tile0, uint64_t tile_step) {
  constexpr int NR = 1 << R;
  const uint32_t T = P->T, c = P->c;
  const uint32_t ns = P->n_stages;
  const uint32_t data_off = P->ops_off, data_bytes = P->data_bytes;
  const uint64_t outer_mask = P->outer_mask, n_tiles = P->n_tiles;
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
  // outer-term slots of the phase ops and their per-tile sums (two halves, used
  // by alternate tiles: a tile's sums are written before the barrier that starts
  // it, when every thread has finished the tile before the previous one)
  const uint32_t n_w = P->n_w;
  const uint8_t *wrec = data + (n_w ? P->w_off - data_off : 0u);
  uint32_t *wsum = reinterpret_cast<uint32_t *>(data + (n_w ? P->w_off - data_off + rphase_w_sums(n_w) : 0u));
  uint32_t wpar = 0;
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
  uint64_t tile = tile0;
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
    const uint64_t next = tile + tile_step;
    const uint64_t base_next = next < n_tiles ? pdep_u64(next, outer_mask) : 0;
    if (n_w) rphase_tile_sums(wrec, n_w, data_bytes - (P->w_off - data_off), base, wsum + wpar * n_w);
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
          reg_rphase<R>(v, data + (op.data_off - data_off), wsum + wpar * n_w, tid);
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
    wpar ^= 1u;
  }
}

}  // namespace svgb
