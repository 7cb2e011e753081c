// sv_measure.cu -- probabilities, norm, Z-string expectation, CDF and sampling.
//
// Measurement of the final state (§III-B: end-of-circuit sampling from one
// state; expectation values from the cached state).  All sums that the CDF
// sampler searches are double precision.  |a|^2 is formed without rounding:
// each float32 square is split into its rounded value and its exact error
// (fmaf), and a thread's 16 amplitudes are added with a compensated (TwoSum)
// float32 accumulator whose error is O(2^-44) relative -- far below double
// rounding of the sums that follow.  Everything above 64-amplitude chunks is
// done in double precision.  Double-precision arithmetic per amplitude is
// avoided because GB300 executes it at a small fraction of the float32 rate.
//
// Sampler layout (per state, in scratch memory):
//   chunk[c] = sum of |a_i|^2 over chunk c (64 amplitudes), double;
//   block[b] = inclusive prefix over 4096-amplitude blocks, double;
//   shot s:  t = u_s * total; b = first block with block[b] > t; walk the
//            block's chunks, then the chunk's amplitudes, accumulating in
//            double, and return the first index whose running sum exceeds t.
#include <cstdint>

#include "sv_internal.h"

namespace svgb {

__host__ __device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }

constexpr int kRT = 256;                     // threads per reduction CTA
constexpr int kPerThread = 16;               // amplitudes per thread
constexpr int kCtaAmps = kRT * kPerThread;   // 4096 = one sampler block
static_assert(uint64_t(kCtaAmps) == kReduceCtaAmps, "reduce_parts_c must match the reduction kernel");

// ---- compensated float32 accumulation -----------------------------------
// __fadd_rn/__fmul_rn are never contracted into FMAs, which would break the
// error-free transformations.
__device__ __forceinline__ void two_sum_acc(float &s, float &c, float x) {
  const float t = __fadd_rn(s, x);
  const float z = __fsub_rn(t, s);
  const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(x, z));
  c = __fadd_rn(c, e);
  s = t;
}

// s + c += a^2 exactly split: a^2 = h + l with h = fl(a*a), l = fma(a,a,-h).
__device__ __forceinline__ void acc_sq(float &s, float &c, float a) {
  const float h = __fmul_rn(a, a);
  const float l = fmaf(a, a, -h);
  two_sum_acc(s, c, h);
  c = __fadd_rn(c, l);
}

__device__ __forceinline__ void acc_pair(float &s, float &c, float s2, float c2) {
  two_sum_acc(s, c, s2);
  c = __fadd_rn(c, c2);
}

__device__ __forceinline__ double cs_to_double(float s, float c) {
  return double(s) + double(c);
}

// Warp sum of compensated pairs (s, c), result in lane 0: the pairs' partial
// sums stay compensated float32 (relative error ~2^-44 for 32 terms); GB300
// runs float64 at a small fraction of the float32 rate, so only lane 0
// converts to double.
__device__ __forceinline__ void warp_acc_pair(float &s, float &c) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float s2 = __shfl_down_sync(0xffffffffu, s, o);
    const float c2 = __shfl_down_sync(0xffffffffu, c, o);
    acc_pair(s, c, s2, c2);
  }
}

// ---- staged load of a CTA's 4096 amplitudes ------------------------------
__device__ __forceinline__ void cp_async16m(void *smem_dst, const void *gsrc) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}

// Loads amplitudes [start, start + cnt) (cnt <= 4096, even) into smem tile.
__device__ __forceinline__ void stage_load(float2 *tile, const float2 *amp, uint64_t start, uint32_t cnt) {
  for (uint32_t i = threadIdx.x; i < (cnt >> 1); i += blockDim.x)
    cp_async16m(tile + 2 * i, amp + start + 2 * uint64_t(i));
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  if ((cnt & 1u) && threadIdx.x == 0) tile[cnt - 1] = amp[start + cnt - 1];
  __syncthreads();
}

// Thread t owns amplitudes [16t, 16t+16) of the staged tile.  The 16-byte
// words are visited in a lane-rotated order so a warp's reads spread over all
// shared-memory banks.  Returns the compensated sums of p and of p*(-1)^parity.
__device__ __forceinline__ void thread_sums(const float2 *tile, uint32_t cnt, uint64_t start,
                                            uint64_t zmask, float &ps, float &pc, float &zs,
                                            float &zc) {
  ps = pc = zs = zc = 0.f;
  const uint32_t t = threadIdx.x;
  const uint32_t lane = t & 31u;
  const float4 *t4 = reinterpret_cast<const float4 *>(tile);
#pragma unroll
  for (uint32_t jj = 0; jj < kPerThread / 2; jj++) {
    const uint32_t j = (jj + lane) & (kPerThread / 2 - 1);
    const uint32_t a0 = t * kPerThread + 2 * j;
    if (a0 >= cnt) continue;
    const float4 v = t4[a0 >> 1];
    float s0 = 0.f, c0 = 0.f;
    acc_sq(s0, c0, v.x);
    acc_sq(s0, c0, v.y);
    float s1 = 0.f, c1 = 0.f;
    if (a0 + 1 < cnt) {
      acc_sq(s1, c1, v.z);
      acc_sq(s1, c1, v.w);
    }
    acc_pair(ps, pc, s0, c0);
    acc_pair(ps, pc, s1, c1);
    if (zmask) {
      const uint64_t i0 = start + a0;
      const bool n0 = __popcll(i0 & zmask) & 1, n1 = __popcll((i0 + 1) & zmask) & 1;
      acc_pair(zs, zc, n0 ? -s0 : s0, n0 ? -c0 : c0);
      acc_pair(zs, zc, n1 ? -s1 : s1, n1 ? -c1 : c1);
    }
  }
}

// ---- norm / Z-expectation ------------------------------------------------
// part[2*b] = sum p, part[2*b+1] = sum p*(-1)^popcount(i & zmask) over CTA b.
// Totals only: a thread takes amplitude pairs j * 256 + t (coalesced 16-byte
// loads, all eight issued before any is used) instead of a staged run.
__global__ void __launch_bounds__(kRT) k_reduce_pz(const float2 *__restrict__ amp, int n,
                                                   uint64_t zmask, double *__restrict__ part) {
  __shared__ double red[2][kRT / 32];
  const uint64_t N = uint64_t(1) << n;
  const uint64_t start = uint64_t(blockIdx.x) * kCtaAmps;
  const uint32_t cnt = uint32_t(umin64(kCtaAmps, N - start));  // even: N >= 2
  const float4 *a4 = reinterpret_cast<const float4 *>(amp + start);
  constexpr int kPairs = kPerThread / 2;
  float4 f[kPairs];
#pragma unroll
  for (int j = 0; j < kPairs; j++) {
    const uint32_t pr = uint32_t(j) * kRT + threadIdx.x;
    f[j] = 2 * pr < cnt ? a4[pr] : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  float ps = 0.f, pc = 0.f, zs = 0.f, zc = 0.f;
#pragma unroll
  for (int j = 0; j < kPairs; j++) {
    float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f;
    acc_sq(s0, c0, f[j].x);
    acc_sq(s0, c0, f[j].y);
    acc_sq(s1, c1, f[j].z);
    acc_sq(s1, c1, f[j].w);
    acc_pair(ps, pc, s0, c0);
    acc_pair(ps, pc, s1, c1);
    if (zmask) {
      const uint64_t i0 = start + 2 * (uint64_t(j) * kRT + threadIdx.x);
      const bool n0 = __popcll(i0 & zmask) & 1, n1 = __popcll((i0 + 1) & zmask) & 1;
      acc_pair(zs, zc, n0 ? -s0 : s0, n0 ? -c0 : c0);
      acc_pair(zs, zc, n1 ? -s1 : s1, n1 ? -c1 : c1);
    }
  }
  if (!zmask) {  // Z_0 is the identity: every sign is +1
    zs = ps;
    zc = pc;
  }
  warp_acc_pair(ps, pc);
  warp_acc_pair(zs, zc);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[0][w] = cs_to_double(ps, pc);
    red[1][w] = cs_to_double(zs, zc);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < kRT / 32; i++) {
      a += red[0][i];
      b += red[1][i];
    }
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b;
  }
}

// Sums the per-CTA pairs in a fixed order: out2[0] = sum p, out2[1] = sum pz.
__global__ void __launch_bounds__(1024) k_sum_pairs(const double *__restrict__ part, size_t count,
                                                    double *__restrict__ out2) {
  __shared__ double red[2][32];
  double a = 0.0, b = 0.0;
  for (size_t i = threadIdx.x; i < count; i += blockDim.x) {
    a += part[2 * i];
    b += part[2 * i + 1];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = a;
    red[1][threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0.0, y = 0.0;
    for (int i = 0; i < int(blockDim.x >> 5); i++) {
      x += red[0][i];
      y += red[1][i];
    }
    out2[0] = x;
    out2[1] = y;
  }
}

size_t reduce_parts(int n) {
  const uint64_t N = uint64_t(1) << n;
  return size_t((N + kCtaAmps - 1) / kCtaAmps);
}

cudaError_t launch_reduce_pz(const float2 *amp, int n, uint64_t zmask, double *part, size_t n_part,
                             double *out2, cudaStream_t st) {
  const size_t ctas = reduce_parts(n);
  if (ctas > n_part) return cudaErrorInvalidValue;
  k_reduce_pz<<<unsigned(ctas), kRT, 0, st>>>(amp, n, zmask, part);
  k_sum_pairs<<<1, 1024, 0, st>>>(part, ctas, out2);
  count_launch(2);
  return cudaGetLastError();
}

// ---- Pauli-string expectation (x_mask != 0) ----------------------------------
// P = i^k X^x Z^z (Y = iXZ on the qubits in both masks, k = popcount(x & z)), so
// (P psi)_i = i^k (-1)^popcount((i^x) & z) psi_(i^x).  Over a pair (i, j = i ^ x),
// i with x's lowest set bit b clear, the two terms of <psi|P psi> add to
//   2 s_i Re(w) i^k (k even)  or  2i s_i Im(w) i^k (k odd),
// w = conj(psi_i) psi_j, s_i = (-1)^popcount(j & z): a real number.  Each
// amplitude is read once; the products are split error-free (fma) and summed
// with the compensated float32 accumulators, per CTA in double.
// part[2*c] = sum |psi|^2, part[2*c+1] = sum over the CTA's pairs of the real
// factor times Re(w) or Im(w); <P> = 2 part_sum[1] / part_sum[0].
constexpr int kPauliPairs = 8;  // pairs per thread

__global__ void __launch_bounds__(kRT) k_reduce_pauli(const float2 *__restrict__ amp, int n, uint64_t x,
                                                      uint64_t z, int b, int k, double *__restrict__ part) {
  __shared__ double red[2][kRT / 32];
  const uint64_t half = (uint64_t(1) << n) >> 1;  // pairs
  const uint64_t m0 = uint64_t(blockIdx.x) * (kRT * kPauliPairs);
  const uint64_t lowb = (uint64_t(1) << b) - 1u;
  float2 ai[kPauliPairs], aj[kPauliPairs];
  uint64_t jj[kPauliPairs];
#pragma unroll
  for (int r = 0; r < kPauliPairs; r++) {
    const uint64_t m = m0 + uint64_t(r) * kRT + threadIdx.x;
    const uint64_t i = ((m & ~lowb) << 1) | (m & lowb);
    jj[r] = i ^ x;
    if (m < half) {
      ai[r] = amp[i];
      aj[r] = amp[jj[r]];
    } else {
      ai[r] = aj[r] = make_float2(0.f, 0.f);
    }
  }
  // the real factor: (-1)^(k/2) on Re(w) for even k, -(-1)^((k-1)/2) on Im(w) for odd k
  const bool odd = k & 1;
  const bool neg = odd ? !(((k - 1) >> 1) & 1) : (((k >> 1) & 1) != 0);
  float ps = 0.f, pc = 0.f, qs = 0.f, qc = 0.f;
#pragma unroll
  for (int r = 0; r < kPauliPairs; r++) {
    acc_sq(ps, pc, ai[r].x);
    acc_sq(ps, pc, ai[r].y);
    acc_sq(ps, pc, aj[r].x);
    acc_sq(ps, pc, aj[r].y);
    // Re(w) = ai.x aj.x + ai.y aj.y ; Im(w) = ai.x aj.y - ai.y aj.x
    const float u1 = ai[r].x, v1 = odd ? aj[r].y : aj[r].x;
    const float u2 = ai[r].y, v2 = odd ? -aj[r].x : aj[r].y;
    const float h1 = __fmul_rn(u1, v1), l1 = fmaf(u1, v1, -h1);
    const float h2 = __fmul_rn(u2, v2), l2 = fmaf(u2, v2, -h2);
    const bool flip = neg != ((__popcll(jj[r] & z) & 1) != 0);
    two_sum_acc(qs, qc, flip ? -h1 : h1);
    two_sum_acc(qs, qc, flip ? -h2 : h2);
    const float l = __fadd_rn(l1, l2);
    qc = __fadd_rn(qc, flip ? -l : l);
  }
  warp_acc_pair(ps, pc);
  warp_acc_pair(qs, qc);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[0][w] = cs_to_double(ps, pc);
    red[1][w] = cs_to_double(qs, qc);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, c = 0.0;
    for (int i = 0; i < kRT / 32; i++) {
      a += red[0][i];
      c += red[1][i];
    }
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = c;
  }
}

cudaError_t launch_reduce_pauli(const float2 *amp, int n, uint64_t x_mask, uint64_t z_mask, double *part,
                                size_t n_part, double *out2, cudaStream_t st) {
  if (x_mask == 0 || n < 1) return cudaErrorInvalidValue;
  const uint64_t pairs = (uint64_t(1) << n) >> 1;
  const uint64_t per = uint64_t(kRT) * kPauliPairs;
  const size_t ctas = size_t((pairs + per - 1) / per);
  if (ctas > n_part) return cudaErrorInvalidValue;
  const int b = __builtin_ctzll(x_mask);
  const int k = __builtin_popcountll(x_mask & z_mask);
  k_reduce_pauli<<<unsigned(ctas), kRT, 0, st>>>(amp, n, x_mask, z_mask, b, k, part);
  k_sum_pairs<<<1, 1024, 0, st>>>(part, ctas, out2);
  count_launch(2);
  return cudaGetLastError();
}

// ---- CDF --------------------------------------------------------------------
// Chunk sums (64 amplitudes; four threads each) and 4096-amplitude block sums;
// with zblock, also the block's sum of p * (-1)^popcount(i & zmask), from the
// same read of the amplitudes.
__global__ void __launch_bounds__(kRT) k_chunk_block(const float2 *__restrict__ amp, int n,
                                                     double *__restrict__ chunk,
                                                     double *__restrict__ blocksum, uint64_t zmask,
                                                     double *__restrict__ zblock) {
  __shared__ __align__(16) float2 tile[kCtaAmps];
  __shared__ double cs[kCtaAmps / 64];
  __shared__ double zred[kRT / 32];
  const uint64_t N = uint64_t(1) << n;
  const uint64_t start = uint64_t(blockIdx.x) * kCtaAmps;
  const uint32_t cnt = uint32_t(umin64(kCtaAmps, N - start));
  stage_load(tile, amp, start, cnt);
  float ps, pc, zs, zc;
  thread_sums(tile, cnt, start, zblock ? zmask : 0, ps, pc, zs, zc);
  if (zblock) {
    if (!zmask) {  // Z_0 is the identity: every sign is +1
      zs = ps;
      zc = pc;
    }
    warp_acc_pair(zs, zc);
    if ((threadIdx.x & 31) == 0) zred[threadIdx.x >> 5] = cs_to_double(zs, zc);
  }
  // four consecutive threads hold one 64-amplitude chunk
#pragma unroll
  for (int o = 1; o < 4; o <<= 1) {
    const float s2 = __shfl_down_sync(0xffffffffu, ps, o);
    const float c2 = __shfl_down_sync(0xffffffffu, pc, o);
    if ((threadIdx.x & (2 * o - 1)) == 0) acc_pair(ps, pc, s2, c2);
  }
  const uint32_t nch = (cnt + 63) / 64;
  if ((threadIdx.x & 3) == 0) {
    const uint32_t c = threadIdx.x >> 2;
    if (c < nch) {
      const double v = cs_to_double(ps, pc);
      cs[c] = v;
      chunk[(start >> kChunkBits) + c] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = 0.0;
    for (uint32_t c = threadIdx.x; c < nch; c += 32) v += cs[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) {
      blocksum[blockIdx.x] = v;
      if (zblock) {
        double z = 0.0;
        for (int w = 0; w < kRT / 32; w++) z += zred[w];
        zblock[blockIdx.x] = z;
      }
    }
  }
}

// out[0] = sum of x[0 .. count) in a fixed order (one CTA).
__global__ void __launch_bounds__(1024) k_sum_doubles(const double *__restrict__ x, size_t count,
                                                      double *__restrict__ out) {
  __shared__ double red[32];
  double a = 0.0;
  for (size_t i = threadIdx.x; i < count; i += blockDim.x) a += x[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < int(blockDim.x >> 5); i++) t += red[i];
    out[0] = t;
  }
}

// Inclusive scan of doubles, in place, three phases over segments of 2048.
constexpr int kScanT = 256, kScanPer = 8, kScanSeg = kScanT * kScanPer;

__device__ __forceinline__ double cta_exclusive_scan(double v, double *sh, double &total) {
  // warp inclusive
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[w] = x;
  __syncthreads();
  if (w == 0) {
    double t = (lane < int(blockDim.x >> 5)) ? sh[lane] : 0.0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    sh[32 + lane] = t;
  }
  __syncthreads();
  total = sh[32 + int(blockDim.x >> 5) - 1];
  const double warp_excl = (w > 0) ? sh[32 + w - 1] : 0.0;
  return warp_excl + x - v;
}

__global__ void __launch_bounds__(kScanT) k_scan_reduce(const double *__restrict__ x, size_t count,
                                                        double *__restrict__ seg) {
  __shared__ double sh[64];
  const size_t base = size_t(blockIdx.x) * kScanSeg + size_t(threadIdx.x) * kScanPer;
  double v = 0.0;
  for (int j = 0; j < kScanPer; j++)
    if (base + j < count) v += x[base + j];
  double tot;
  cta_exclusive_scan(v, sh, tot);
  if (threadIdx.x == 0) seg[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanT) k_scan_top(double *__restrict__ seg, size_t count) {
  // exclusive scan of the segment totals by one CTA, in chunks of kScanSeg
  __shared__ double sh[64];
  double carry = 0.0;
  for (size_t b = 0; b < count; b += kScanSeg) {
    const size_t base = b + size_t(threadIdx.x) * kScanPer;
    double loc[kScanPer];
    double v = 0.0;
    for (int j = 0; j < kScanPer; j++) {
      loc[j] = (base + j < count) ? seg[base + j] : 0.0;
      v += loc[j];
    }
    double tot;
    double ex = cta_exclusive_scan(v, sh, tot) + carry;
    for (int j = 0; j < kScanPer; j++) {
      if (base + j < count) seg[base + j] = ex;
      ex += loc[j];
    }
    carry += tot;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kScanT) k_scan_apply(double *__restrict__ x, size_t count,
                                                       const double *__restrict__ seg) {
  __shared__ double sh[64];
  const size_t base = size_t(blockIdx.x) * kScanSeg + size_t(threadIdx.x) * kScanPer;
  double loc[kScanPer];
  double v = 0.0;
  for (int j = 0; j < kScanPer; j++) {
    loc[j] = (base + j < count) ? x[base + j] : 0.0;
    v += loc[j];
  }
  double tot;
  double run = cta_exclusive_scan(v, sh, tot) + seg[blockIdx.x];
  for (int j = 0; j < kScanPer; j++) {
    run += loc[j];
    if (base + j < count) x[base + j] = run;
  }
}

__global__ void k_copy_last(const double *__restrict__ x, size_t count, double *__restrict__ out) {
  out[0] = x[count - 1];
}

cudaError_t launch_build_cdf(const float2 *amp, int n, MeasureScratch &ms, double *total_dev,
                             cudaStream_t st, uint64_t zmask, double *ztotal_dev) {
  const uint64_t N = uint64_t(1) << n;
  const size_t nblk = size_t((N + kCtaAmps - 1) / kCtaAmps);
  const size_t nseg = (nblk + kScanSeg - 1) / kScanSeg;
  if (nblk > ms.n_block || nseg > ms.n_part) return cudaErrorInvalidValue;
  // per-block Z sums: the second half of the reduction scratch (2 * n_part
  // doubles; the scan uses the first nseg <= nblk)
  double *zblock = nullptr;
  if (ztotal_dev) {
    if (nblk > ms.n_part) return cudaErrorInvalidValue;
    zblock = ms.part + ms.n_part;
  }
  k_chunk_block<<<unsigned(nblk), kRT, 0, st>>>(amp, n, ms.chunk, ms.block, zmask, zblock);
  k_scan_reduce<<<unsigned(nseg), kScanT, 0, st>>>(ms.block, nblk, ms.part);
  k_scan_top<<<1, kScanT, 0, st>>>(ms.part, nseg);
  k_scan_apply<<<unsigned(nseg), kScanT, 0, st>>>(ms.block, nblk, ms.part);
  k_copy_last<<<1, 1, 0, st>>>(ms.block, nblk, total_dev);
  count_launch(5);
  if (zblock) {
    k_sum_doubles<<<1, 1024, 0, st>>>(zblock, nblk, ztotal_dev);
    count_launch();
  }
  return cudaGetLastError();
}

// ---- sampling -----------------------------------------------------------------
__device__ __forceinline__ double amp_p(float2 a) {
  const double re = a.x, im = a.y;
  return fma(re, re, im * im);
}

__global__ void __launch_bounds__(256) k_sample(const float2 *__restrict__ amp, int n,
                                                const double *__restrict__ chunk,
                                                const double *__restrict__ block,
                                                const double *__restrict__ total_dev,
                                                const double *__restrict__ u, uint64_t seed,
                                                int use_seed, uint64_t shots,
                                                uint64_t *__restrict__ out,
                                                unsigned long long *__restrict__ n_boundary) {
  const uint64_t s = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= shots) return;
  const uint64_t N = uint64_t(1) << n;
  const size_t nblk = size_t((N + kCtaAmps - 1) / kCtaAmps);
  const double total = total_dev[0];
  const double us = use_seed ? splitmix_uniform(seed, s) : u[s];
  const double t = us * total;
  // block: first b with inclusive prefix > t
  size_t lo = 0, hi = nblk;
  while (lo < hi) {
    const size_t mid = (lo + hi) >> 1;
    if (block[mid] > t) hi = mid; else lo = mid + 1;
  }
  size_t b = lo;
  if (b == nblk) {  // t rounded up to the total: last block with mass
    b = nblk - 1;
    while (b > 0 && !(block[b] > block[b - 1])) b--;
  }
  double acc = b ? block[b - 1] : 0.0;
  // chunk within the block
  const uint64_t a_begin = uint64_t(b) * kCtaAmps;
  const uint64_t a_end = umin64(a_begin + kCtaAmps, N);
  const uint64_t c_begin = a_begin >> kChunkBits;
  const uint64_t c_end = (a_end + 63) >> kChunkBits;
  uint64_t c = c_end, c_last = c_begin;
  double acc_last = acc;
  for (uint64_t cc = c_begin; cc < c_end; cc++) {
    const double v = chunk[cc];
    if (v > 0.0) {
      c_last = cc;
      acc_last = acc;
    }
    if (acc + v > t) {
      c = cc;
      break;
    }
    acc += v;
  }
  if (c == c_end) {
    c = c_last;
    acc = acc_last;
  }
  // amplitude within the chunk
  const uint64_t i_begin = c << kChunkBits;
  const uint64_t i_end = umin64(i_begin + 64, N);
  uint64_t x = i_end, x_last = i_begin;
  double below = acc, below_last = acc, p_last = 0.0, px = 0.0;
  for (uint64_t i = i_begin; i < i_end; i++) {
    const double p = amp_p(amp[i]);
    if (p > 0.0) {
      x_last = i;
      below_last = acc;
      p_last = p;
    }
    if (acc + p > t) {
      x = i;
      below = acc;
      px = p;
      break;
    }
    acc += p;
  }
  if (x == i_end) {
    x = x_last;
    below = below_last;
    px = p_last;
  }
  out[s] = x;
  const double above = below + px;
  const bool bnd = fabs(t - above) < 1e-9 || fabs(t - below) < 1e-9;
  if (bnd && n_boundary) atomicAdd(n_boundary, 1ull);
}

cudaError_t launch_sample(const float2 *amp, int n, const MeasureScratch &ms, const double *total_dev,
                          const double *u, uint64_t seed, int use_seed, uint64_t shots,
                          uint64_t *out, uint64_t *n_boundary, cudaStream_t st) {
  if (shots == 0) return cudaSuccess;
  const uint64_t grid = (shots + 255) / 256;
  if (grid > 0x7fffffffull) return cudaErrorInvalidValue;
  k_sample<<<unsigned(grid), 256, 0, st>>>(amp, n, ms.chunk, ms.block, total_dev, u, seed, use_seed,
                                           shots, out,
                                           reinterpret_cast<unsigned long long *>(n_boundary));
  count_launch();
  return cudaGetLastError();
}

// ---- probabilities / reset --------------------------------------------------------
__global__ void k_probabilities(const float2 *__restrict__ amp, uint64_t offset, uint64_t count,
                                double *__restrict__ out) {
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count;
       i += uint64_t(gridDim.x) * blockDim.x)
    out[i] = amp_p(amp[offset + i]);
}

cudaError_t launch_probabilities(const float2 *amp, uint64_t offset, uint64_t count, double *out,
                                 cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  const uint64_t g = umin64((count + 255) / 256, 152ull * 64);
  k_probabilities<<<unsigned(g), 256, 0, st>>>(amp, offset, count, out);
  count_launch();
  return cudaGetLastError();
}

// Collapse after measuring qubit q: over every pair (i0, i1 = i0 | 2^q) keep the
// outcome's half scaled by `scale` and zero the other; with `to_zero` (a reset
// whose outcome was 1) the kept half moves to bit q = 0.
__global__ void k_collapse(float2 *__restrict__ amp, int n, int q, int outcome, int to_zero, float scale) {
  const uint64_t half = uint64_t(1) << (n - 1);
  const float2 z = make_float2(0.f, 0.f);
  auto keep = [&](float2 a) { return make_float2(a.x * scale, a.y * scale); };
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  if (q == 0) {
    // i0 and i1 are adjacent: one 16-byte access per pair
    float4 *a4 = reinterpret_cast<float4 *>(amp);
    for (uint64_t k = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < half; k += stride) {
      const float4 v = a4[k];
      const float2 a = make_float2(v.x, v.y), b = make_float2(v.z, v.w);
      float2 r0, r1;
      if (outcome == 0) { r0 = keep(a); r1 = z; }
      else if (to_zero) { r0 = keep(b); r1 = z; }
      else { r0 = z; r1 = keep(b); }
      a4[k] = make_float4(r0.x, r0.y, r1.x, r1.y);
    }
    return;
  }
  // q >= 1: two consecutive pairs (i0, i0 + 1) and (i1, i1 + 1), 16 bytes each
  const uint64_t low = (uint64_t(1) << q) - 1;
  for (uint64_t k2 = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; k2 < (half >> 1); k2 += stride) {
    const uint64_t k = k2 << 1;
    const uint64_t i0 = ((k & ~low) << 1) | (k & low), i1 = i0 | (low + 1);
    float4 *p0 = reinterpret_cast<float4 *>(amp + i0), *p1 = reinterpret_cast<float4 *>(amp + i1);
    const float4 A = *p0, B = *p1;
    const float2 a0 = make_float2(A.x, A.y), a1 = make_float2(A.z, A.w);
    const float2 b0 = make_float2(B.x, B.y), b1 = make_float2(B.z, B.w);
    float2 r00, r01, r10, r11;
    if (outcome == 0) { r00 = keep(a0); r01 = keep(a1); r10 = z; r11 = z; }
    else if (to_zero) { r00 = keep(b0); r01 = keep(b1); r10 = z; r11 = z; }
    else { r00 = z; r01 = z; r10 = keep(b0); r11 = keep(b1); }
    *p0 = make_float4(r00.x, r00.y, r01.x, r01.y);
    *p1 = make_float4(r10.x, r10.y, r11.x, r11.y);
  }
}

cudaError_t launch_collapse(float2 *amp, int n, int q, int outcome, int to_zero, float scale,
                            cudaStream_t st) {
  if (n < 1 || q < 0 || q >= n) return cudaErrorInvalidValue;
  const uint64_t units = (uint64_t(1) << (n - 1)) >> (q == 0 ? 0 : 1);
  const uint64_t g = umin64((units + 255) / 256, 152ull * 16);
  if (units == 0) return cudaSuccess;
  k_collapse<<<unsigned(g), 256, 0, st>>>(amp, n, q, outcome, to_zero, scale);
  count_launch();
  return cudaGetLastError();
}

__global__ void k_set_one(float2 *amp, uint64_t idx) { amp[idx] = make_float2(1.f, 0.f); }

cudaError_t launch_reset(float2 *amp, int n, uint64_t basis, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(amp, 0, (size_t(1) << n) * sizeof(float2), st);
  if (e != cudaSuccess) return e;
  k_set_one<<<1, 1, 0, st>>>(amp, basis);
  count_launch();
  return cudaGetLastError();
}

}  // namespace svgb
