// sv_apply.cu -- the HBM pass kernel of sv_apply_circuit.
//
// One launch applies one pass of the plan (see sv_internal.h): every CTA owns
// the 2^T amplitudes whose indices share the values of the qubits outside the
// pass's tile set.  Those amplitudes sit in 2^(T-c) runs of 2^c contiguous
// amplitudes (the c lowest qubits are always in the tile).  The CTA
//   1. gathers its runs into shared memory with 16-byte cp.async copies,
//   2. applies the pass's ops in order -- dense fused blocks (each thread owns
//      one group of 2^k amplitudes at a time) and diagonal phase ops (a
//      per-tile table of phases, exact modulo 2*pi in 32-bit turn arithmetic),
//   3. writes the tile back in place.
// The state is read once and written once per pass: 16 bytes per amplitude.
#include <cstdint>

#include "sv_internal.h"

namespace svgb {

constexpr int kNT = 256;  // threads per CTA

__device__ __forceinline__ uint64_t pdep_u64(uint64_t src, uint64_t mask) {
  uint64_t out = 0;
  while (mask) {
    const uint64_t low = mask & (~mask + 1);
    if (src & 1) out |= low;
    src >>= 1;
    mask &= mask - 1;
  }
  return out;
}

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Dense k-qubit block on local bits lb[0..K-1]: for every group (the 2^(T-K)
// index patterns with those bits clear) gather 2^K amplitudes, multiply by the
// 2^K x 2^K matrix, scatter back.
template <int K>
__device__ __forceinline__ void apply_dense(float2 *__restrict__ tile, const float2 *__restrict__ mat,
                                            const uint8_t *lb, uint32_t T) {
  constexpr int KK = 1 << K;
  uint32_t sp[K];
#pragma unroll
  for (int m = 0; m < K; m++) sp[m] = lb[m];
  // ascending order for zero-bit insertion
#pragma unroll
  for (int a = 0; a < K; a++)
#pragma unroll
    for (int b = 0; b + 1 < K - a; b++)
      if (sp[b] > sp[b + 1]) {
        const uint32_t t = sp[b];
        sp[b] = sp[b + 1];
        sp[b + 1] = t;
      }
  uint32_t off[KK];
#pragma unroll
  for (int j = 0; j < KK; j++) {
    uint32_t o = 0;
#pragma unroll
    for (int m = 0; m < K; m++)
      if ((j >> m) & 1) o |= 1u << lb[m];
    off[j] = o;
  }
  const uint32_t groups = 1u << (T - K);
  for (uint32_t g = threadIdx.x; g < groups; g += blockDim.x) {
    uint32_t b = g;
#pragma unroll
    for (int m = 0; m < K; m++) b = ((b >> sp[m]) << (sp[m] + 1)) | (b & ((1u << sp[m]) - 1u));
    float2 v[KK];
#pragma unroll
    for (int j = 0; j < KK; j++) v[j] = tile[b + off[j]];
#pragma unroll
    for (int r = 0; r < KK; r++) {
      float re = 0.f, im = 0.f;
#pragma unroll
      for (int j = 0; j < KK; j++) {
        const float2 m = mat[r * KK + j];
        re = fmaf(m.x, v[j].x, re);
        re = fmaf(-m.y, v[j].y, re);
        im = fmaf(m.x, v[j].y, im);
        im = fmaf(m.y, v[j].x, im);
      }
      tile[b + off[r]] = make_float2(re, im);
    }
  }
}

// Diagonal phase op.  Each term adds `turn` (2*pi / 2^32 units) to the phase of
// every amplitude whose outer qubits in term.outer_mask are all 1 (fixed for
// this tile) and whose local bit term.la is 1 (or unconditionally if la < 0).
// The per-tile phase is then a sum of per-local-bit turns, tabulated over the
// low and high halves of the tile index.
__device__ __forceinline__ void apply_phase(float2 *__restrict__ tile, const PhaseTerm *__restrict__ terms,
                                            uint32_t count, uint64_t base, uint32_t T,
                                            uint32_t *acc, float2 *tab) {
  if (threadIdx.x <= T) acc[threadIdx.x] = 0u;
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < count; i += blockDim.x) {
    const PhaseTerm pt = terms[i];
    if ((base & pt.outer_mask) == pt.outer_mask) atomicAdd(&acc[pt.la + 1], pt.turn);
  }
  __syncthreads();
  const uint32_t h = T >> 1;
  const uint32_t nlo = 1u << h, nhi = 1u << (T - h);
  for (uint32_t e = threadIdx.x; e < nlo + nhi; e += blockDim.x) {
    uint32_t turn;
    if (e < nlo) {
      turn = acc[0];
      for (uint32_t j = 0; j < h; j++)
        if ((e >> j) & 1u) turn += acc[1 + j];
    } else {
      const uint32_t e2 = e - nlo;
      turn = 0u;
      for (uint32_t j = 0; j < T - h; j++)
        if ((e2 >> j) & 1u) turn += acc[1 + h + j];
    }
    float s, c;
    sincospif(static_cast<float>(static_cast<int32_t>(turn)) * 4.656612873077393e-10f, &s, &c);
    tab[e] = make_float2(c, s);
  }
  __syncthreads();
  const uint32_t L = 1u << T, lmask = nlo - 1u;
  for (uint32_t l = threadIdx.x; l < L; l += blockDim.x) {
    const float2 a = tab[l & lmask], b = tab[nlo + (l >> h)];
    const float2 f = make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
    const float2 v = tile[l];
    tile[l] = make_float2(v.x * f.x - v.y * f.y, v.x * f.y + v.y * f.x);
  }
}

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

static size_t pass_smem(uint32_t T, uint32_t c, int kmax) {
  return (size_t(1) << T) * sizeof(float2) + (size_t(1) << (T - c)) * sizeof(uint64_t) +
         (size_t(1) << (2 * kmax)) * sizeof(float2) + 256 * sizeof(float2) + 64 * sizeof(uint32_t);
}

template <int KMAX>
static cudaError_t launch_k(float2 *amp, const uint8_t *plan, uint32_t off, const PlanPass &hp,
                            cudaStream_t st) {
  const size_t smem = pass_smem(hp.T, hp.c, KMAX);
  static unsigned long long configured = 0;  // bit d: attribute set on device d
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 64 && !((configured >> dev) & 1ull)) {
    e = cudaFuncSetAttribute(k_pass<KMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(pass_smem(kMaxTile, 1, KMAX)));
    if (e != cudaSuccess) return e;
    configured |= 1ull << dev;
  }
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
                        const PlanPass &hp, cudaStream_t stream) {
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
