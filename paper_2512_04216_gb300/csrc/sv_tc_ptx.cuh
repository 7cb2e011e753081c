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

// D(tmem) (+)= A(tmem) * B(smem descriptor); kind::tf32, M=128, N=32, K=8.
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

// Instruction descriptor: D f32, A/B tf32, both K-major, N=32, M=128.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

// Half h (K steps 2h, 2h+1) of the 3xTF32 product of one stage for row group g,
// accumulated into its own D_h (columns 64 + 32h of the group); issued by one
// thread.  A single issuing thread waits ~230 cycles per tcgen05.mma whatever
// the shape, so each group's products are split over two issuers and the two
// partial accumulators are added after tcgen05.ld.
__device__ __forceinline__ void issue_stage_mma_half(uint32_t tbase, uint32_t g, uint32_t h, uint32_t b_saddr) {
  const uint32_t a_hi = tbase + g * kTcColsPerGroup, a_lo = a_hi + 32, d = a_hi + 64 + 32 * h;
  const uint32_t bhi = b_saddr, blo = b_saddr + 4 * 1024;
#pragma unroll
  for (uint32_t i = 0; i < 2; i++) {
    const uint32_t ks = 2 * h + i;
    mma_tf32_ts(d, a_hi + 8 * ks, b_desc(blo + ks * 1024), kIdesc, i > 0);
  }
#pragma unroll
  for (uint32_t i = 0; i < 2; i++) {
    const uint32_t ks = 2 * h + i;
    mma_tf32_ts(d, a_lo + 8 * ks, b_desc(bhi + ks * 1024), kIdesc, 1);
  }
#pragma unroll
  for (uint32_t i = 0; i < 2; i++) {
    const uint32_t ks = 2 * h + i;
    mma_tf32_ts(d, a_hi + 8 * ks, b_desc(bhi + ks * 1024), kIdesc, 1);
  }
}

// x_hi: x rounded to the nearest TF32 value (ties away from zero; the 13 low
// mantissa bits cleared), so x_lo = x - x_hi (exact in float32) takes either
// sign and |x_lo| <= 2^-11 |x|.  Truncating instead would give x_lo the sign
// of x, and the tensor core's own treatment of x_lo's low bits would then bias
// every product towards zero.
__device__ __forceinline__ uint32_t tf32_hi_bits(float x) {
  return (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u;
}

__device__ __forceinline__ void split_row(const float (&x)[32], uint32_t (&hi)[32], uint32_t (&lo)[32]) {
#pragma unroll
  for (int i = 0; i < 32; i++) {
    const uint32_t h = tf32_hi_bits(x[i]);
    hi[i] = h;
    lo[i] = __float_as_uint(__fsub_rn(x[i], __uint_as_float(h)));
  }
}

}  // namespace svgb
