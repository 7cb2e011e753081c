// sv_device.cuh -- device helpers shared by the pass kernels (sv_apply.cu)
// and the batched kernel (sv_batch.cu): bit deposit, 16-byte async copies, and
// the shared-memory tile ops (dense k-qubit blocks, per-tile phase tables).
#pragma once

#include <cstdint>

#include "sv_internal.h"

namespace svgb {

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

// 16-byte async copy to a 32-bit shared-window address
__device__ __forceinline__ void cp_async16_s(uint32_t s, const void *gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}

// 8-byte shared-memory accesses at 32-bit shared-window addresses
__device__ __forceinline__ void sts64(uint32_t a, float2 v) {
  asm volatile("st.shared.v2.f32 [%0], {%1, %2};\n" ::"r"(a), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ float2 lds64(uint32_t a) {
  float2 v;
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];\n" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
  return v;
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
    if constexpr (K <= 3) {
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
    } else {
      // 16 / 32 outputs: one row at a time keeps the register footprint to the inputs
#pragma unroll 1
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
        uint32_t o = 0;
#pragma unroll
        for (int m = 0; m < K; m++)
          if ((r >> m) & 1) o |= 1u << lb[m];
        tile[b + o] = make_float2(re, im);
      }
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

}  // namespace svgb
