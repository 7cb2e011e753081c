// sv_tc_ptx.cuh -- inline-PTX wrappers for tcgen05 (TMEM, MMA, commit),
// mbarrier waits bounded by %globaltimer, and the 3xTF32 stage product used
// by the tensor-core pass kernel and its self-test.  See sv_tc.cu for the
// operand layouts.
#pragma once

#include <cstdint>

#include "sv_tc.h"

namespace svgb {

// ---- PTX wrappers ---------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(dst)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
  return t;
}

// Wait for phase `parity` of the barrier; false after ~1 s (the caller reports it).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_ns() - t0 > 1000000000ull) return false;
  }
  return true;
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                   smem_u32(bar))
               : "memory");
}

// D(tmem) (+)= A(tmem) * B(smem descriptor); kind::tf32, M=128, K=8, N from idesc.
__device__ __forceinline__ void mma_tf32_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
      "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// 32 consecutive 32-bit columns of this thread's lane.
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};\n" ::"r"(
          taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
      "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]),
      "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]),
      "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, no swizzle, core matrices of
// 8 rows x 16 bytes; LBO = 128 B between the two core matrices along K of one
// K step, SBO = 256 B between 8-row groups along N (see tc_b_offset).
__device__ __forceinline__ uint64_t b_desc(uint32_t saddr) {
  return uint64_t((saddr & 0x3FFFFu) >> 4) | (uint64_t(128 >> 4) << 16) | (uint64_t(256 >> 4) << 32) |
         (uint64_t(1) << 46);
}

// Instruction descriptors: D f32, A/B tf32, both K-major, M=128, N given.
constexpr uint32_t kIdescTf32(uint32_t n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((n >> 3) << 17) | ((128u >> 4) << 24);
}

// The 3xTF32 product of one stage for one 128-row group, issued by one thread:
//   [D_left | D_right] = A_hi * [B_hi | B_lo]^T   (N = 2K, K/8 K steps)
//   D_left            += A_lo * B_hi^T            (N = K, K/8 K steps)
// so D_left + D_right = A_hi B_hi + A_lo B_hi + A_hi B_lo.  Stacking B_hi and
// B_lo along N takes K/4 MMAs per stage instead of 3K/8.  cols: the group's
// TMEM columns (A_hi at +0, A_lo at +K, D at +2K); b_saddr: the stage image B'.
template <int R>
__device__ __forceinline__ void issue_stage_mma(uint32_t cols, uint32_t b_saddr) {
  constexpr uint32_t K = tc_k(R), KS = K / 8, STEP = tc_b_kstep(R);
  const uint32_t a_hi = cols, a_lo = cols + K, d = cols + 2 * K;
#pragma unroll
  for (uint32_t ks = 0; ks < KS; ks++)
    mma_tf32_ts(d, a_hi + 8 * ks, b_desc(b_saddr + ks * STEP), kIdescTf32(2 * K), ks > 0);
#pragma unroll
  for (uint32_t ks = 0; ks < KS; ks++) mma_tf32_ts(d, a_lo + 8 * ks, b_desc(b_saddr + ks * STEP), kIdescTf32(K), 1);
}

// Veltkamp splitting (Dekker 1971) of a float pair: with c = x * (2^13 + 1),
// hi = c - (c - x) keeps the 11 leading significant bits of x, rounded to
// nearest, which is exactly a TF32 value; lo = x - hi is exact in float32 and
// takes either sign, |lo| <= 2^-12 |x|.  Each step is one paired instruction
// (an FMA with multiplier -1 is a single-rounding subtraction).
__device__ __forceinline__ void split_pair(float2 x, float2 &hi, float2 &lo) {
  const float2 m1 = make_float2(-1.f, -1.f);
  const float2 c = __fmul2_rn(x, make_float2(8193.f, 8193.f));
  const float2 t = __ffma2_rn(x, m1, c);   // c - x
  hi = __ffma2_rn(t, m1, c);               // c - (c - x)
  lo = __ffma2_rn(hi, m1, x);              // x - hi
}

// Split the 2^R amplitudes of a row and store A_hi, A_lo (K columns each,
// interleaved re, im) at TMEM address a (this thread's lane), 16 amplitudes
// (32 columns) at a time.
template <int R>
__device__ __forceinline__ void store_row_split(uint32_t a, const float2 (&v)[1 << R]) {
  constexpr uint32_t K = tc_k(R);
#pragma unroll
  for (uint32_t hh = 0; hh < K / 32; hh++) {
    uint32_t h[32], l[32];
#pragma unroll
    for (int j = 0; j < 16; j++) {
      float2 hi, lo;
      split_pair(v[16 * hh + j], hi, lo);
      h[2 * j] = __float_as_uint(hi.x);
      h[2 * j + 1] = __float_as_uint(hi.y);
      l[2 * j] = __float_as_uint(lo.x);
      l[2 * j + 1] = __float_as_uint(lo.y);
    }
    tmem_st32(a + 32 * hh, h);
    tmem_st32(a + K + 32 * hh, l);
  }
}

// Read D_left, D_right of this thread's lane (columns 2K.. of the group) and
// return their sum (round to nearest) as 2^R amplitudes, 16 at a time.
template <int R>
__device__ __forceinline__ void load_row_sum(uint32_t a, float2 (&v)[1 << R]) {
  constexpr uint32_t K = tc_k(R);
#pragma unroll
  for (uint32_t hh = 0; hh < K / 32; hh++) {
    uint32_t dl[32], dr[32];
    tmem_ld32(a + 2 * K + 32 * hh, dl);
    tmem_ld32(a + 3 * K + 32 * hh, dr);
    tmem_wait_ld();
#pragma unroll
    for (int j = 0; j < 16; j++)
      v[16 * hh + j] = __fadd2_rn(make_float2(__uint_as_float(dl[2 * j]), __uint_as_float(dl[2 * j + 1])),
                                  make_float2(__uint_as_float(dr[2 * j]), __uint_as_float(dr[2 * j + 1])));
  }
}

}  // namespace svgb
