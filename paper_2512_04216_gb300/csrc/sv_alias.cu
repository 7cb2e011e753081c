// sv_alias.cu -- Walker alias table of the outcome distribution |a_i|^2 and
// O(1) draws from it (§III-C: shots are drawn by alias sampling, constant work
// per shot; Walker 1974).
//
// Units.  Every bucket holds C = 2^31 units.  Item i weighs
// Q_i = round(|a_i|^2 * N / W * 2^31) units (W = sum of |a|^2); Q is formed from
// the float32 amplitude with error-free float32 products (about 46 bits) so no
// per-item double arithmetic is needed -- GB300 runs float64 at a small
// fraction of the float32 rate.  Everything after Q is exact integer arithmetic.
//
// Table.  Items with Q < C are light, the others heavy.  The table is the one
// the sequential sweep builds (light items in index order take their deficits
// C - Q from heavy items in index order; a heavy item left with fewer than C
// units becomes a light bucket filled by the next heavy item; the last heavy
// item keeps a full bucket), evaluated in parallel from two exact prefix sums:
//   D_k = total deficit of light items before light item k (exclusive);
//   E_j = total excess Q - C of heavy items 0..j (inclusive).
// Light k aliases heavy #{ j : E_j < D_k } (clamped to the last heavy item).
// Heavy j (not the last) is used up by light c - 1 where c = #{ k : D_k <= E_j };
// with D_c the deficit prefix after that light item (the total deficit when
// c is the light count) it keeps C - (D_c - E_j) units and aliases heavy j + 1
// -- or keeps C units when D_c <= E_j (never used up).  Both counts are ranks
// in the merge of the increasing sequences D and E with D first on ties, found
// by a merge-path partition (Odeh, Green, Mwassi, Shmueli and Birk, "Merge
// Path", 2012): one search per CTA boundary in HBM (all in parallel), then one
// per thread in shared memory, then a short sequential merge.
//
// Build: k_alias_count (per-block light counts and sums) -> exclusive scan of
// the block triples -> k_alias_place (every light item's deficit prefix,
// weight and index, every heavy item's excess prefix and index, in rank order)
// -> k_alias_splits (the merge-path split at every CTA boundary) -> k_alias_merge
// (the table).  Draw: x = u N, i = floor(x), f = x - i;
// outcome i when f 2^31 < own_i, else alias_i.
#include <atomic>
#include <cstdint>

#include "sv_internal.h"

namespace svgb {

namespace {

constexpr int kAT = 256;                 // threads of the per-block kernels
constexpr int kAPer = 16;                // items per thread
constexpr int kABlock = kAT * kAPer;     // 4096 items per block
constexpr int kSegT = 256, kSegPer = 8;  // scan of block triples: 2048 per segment
constexpr int kSeg = kSegT * kSegPer;
constexpr int kMT = 128, kMPer = 8;      // merge: 1024 merged items per CTA
constexpr int kMItems = kMT * kMPer;

__host__ __device__ __forceinline__ uint64_t umin(uint64_t a, uint64_t b) { return a < b ? a : b; }

// round(X + Y) for X >= 0 exact in float and |Y| <= 2^-20 X, without
// float-to-integer conversion instructions (the 64-bit ones issue at the
// float64 rate on GB300): integer parts come from the float bits, and values
// below 2^22 are rounded by adding 2^23 (or 1.5 * 2^23 when signed), whose
// sum has a unit last place, then reading the mantissa bits.
__device__ __forceinline__ uint64_t round_pair(float X, float Y) {
  const uint32_t bx = __float_as_uint(X);
  const int ex = int(bx >> 23) - 150;  // X = mantissa * 2^ex
  if (ex >= 0) {                       // X >= 2^23: an integer
    const uint64_t xi = uint64_t((bx & 0x7fffffu) | 0x800000u) << ex;
    int64_t yi;
    const float ay = fabsf(Y);
    if (ay < 4194304.f) {
      yi = __float_as_int(__fadd_rn(Y, 12582912.f)) - 0x4B400000;
    } else {  // |Y| >= 2^22: a multiple of 1/2; halves round up (they need an exact tie)
      const uint32_t by = __float_as_uint(ay);
      const int ey = int(by >> 23) - 150;
      const uint64_t my = (by & 0x7fffffu) | 0x800000u;
      const uint64_t mag = ey >= 0 ? (my << ey) : ((my + 1) >> 1);
      yi = Y < 0.f ? -int64_t(mag) : int64_t(mag);
    }
    return uint64_t(int64_t(xi) + yi);
  }
  // X < 2^23: r = rint(X) exactly, then round the small remainder X - r + Y
  const float xr = __fadd_rn(X, 8388608.f);
  const int ri = __float_as_int(xr) - 0x4B000000;
  const float d = __fadd_rn(__fsub_rn(X, __fsub_rn(xr, 8388608.f)), Y);
  const int q = ri + (__float_as_int(__fadd_rn(d, 12582912.f)) - 0x4B400000);
  return q < 0 ? 0 : uint64_t(q);
}

// Q = round(|a|^2 * s * 2^31) with s = s_hi + s_lo.  |a|^2 and the product are
// carried as unevaluated float32 pairs (exact squares via fmaf, TwoSum), which
// keeps about 46 bits; the rounding to units then differs from a correctly
// rounded result only within ~2^-14 units of a half-unit boundary.
__device__ __forceinline__ uint64_t quantise(float2 a, float s_hi, float s_lo) {
  const float x2 = __fmul_rn(a.x, a.x), x2e = fmaf(a.x, a.x, -x2);
  const float y2 = __fmul_rn(a.y, a.y), y2e = fmaf(a.y, a.y, -y2);
  const float ph = __fadd_rn(x2, y2);
  const float z = __fsub_rn(ph, x2);
  const float pe = __fadd_rn(__fsub_rn(x2, __fsub_rn(ph, z)), __fsub_rn(y2, z));
  const float pl = __fadd_rn(pe, __fadd_rn(x2e, y2e));
  const float qh = __fmul_rn(ph, s_hi);
  const float qe = fmaf(ph, s_hi, -qh);
  const float ql = __fadd_rn(qe, fmaf(ph, s_lo, __fmul_rn(pl, s_hi)));
  // scaling by 2^31 is exact
  return round_pair(__fmul_rn(qh, 2147483648.f), __fmul_rn(ql, 2147483648.f));
}

// Block-wide exclusive scan of three 64-bit counters (thread order); returns the
// block totals in tot[3].
__device__ __forceinline__ void cta_scan3(uint64_t v[3], uint64_t ex[3], uint64_t tot[3],
                                          uint64_t (*sh)[3]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint64_t x[3] = {v[0], v[1], v[2]};
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, x[c], o);
      if (lane >= o) x[c] += y;
    }
  }
  if (lane == 31) {
#pragma unroll
    for (int c = 0; c < 3; c++) sh[w][c] = x[c];
  }
  __syncthreads();
  if (w == 0) {
    uint64_t t[3];
#pragma unroll
    for (int c = 0; c < 3; c++) t[c] = lane < nw ? sh[lane][c] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
      for (int c = 0; c < 3; c++) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, t[c], o);
        if (lane >= o) t[c] += y;
      }
    }
    if (lane < nw) {
#pragma unroll
      for (int c = 0; c < 3; c++) sh[32 + lane][c] = t[c];
    }
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < 3; c++) {
    ex[c] = (w > 0 ? sh[32 + w - 1][c] : 0) + x[c] - v[c];
    tot[c] = sh[32 + nw - 1][c];
  }
  __syncthreads();
}

// Per 4096-item block: light count, total deficit, total excess.
__global__ void __launch_bounds__(kAT) k_alias_count(const float2 *__restrict__ amp, int n, float s_hi,
                                                     float s_lo, uint64_t *__restrict__ blk) {
  __shared__ uint64_t sh[64][3];
  const uint64_t N = uint64_t(1) << n;
  const uint64_t start = uint64_t(blockIdx.x) * kABlock;
  const uint64_t cnt = umin(kABlock, N - start);  // even: N >= 2
  const float4 *a4 = reinterpret_cast<const float4 *>(amp + start);
  uint64_t v[3] = {0, 0, 0};
  // all eight 16-byte loads are issued before any is used (predicated, no early exit)
  float4 f[kABlock / 2 / kAT];
#pragma unroll
  for (uint32_t j = 0; j < kABlock / 2 / kAT; j++) {
    const uint64_t pr = uint64_t(j) * kAT + threadIdx.x;
    f[j] = 2 * pr < cnt ? a4[pr] : make_float4(0.f, 0.f, 0.f, 0.f);
  }
#pragma unroll
  for (uint32_t j = 0; j < kABlock / 2 / kAT; j++) {
    const uint64_t pr = uint64_t(j) * kAT + threadIdx.x;
    if (2 * pr >= cnt) continue;
    const uint64_t q0 = quantise(make_float2(f[j].x, f[j].y), s_hi, s_lo);
    const uint64_t q1 = quantise(make_float2(f[j].z, f[j].w), s_hi, s_lo);
    if (q0 < kAliasUnits) { v[0]++; v[1] += kAliasUnits - q0; } else { v[2] += q0 - kAliasUnits; }
    if (q1 < kAliasUnits) { v[0]++; v[1] += kAliasUnits - q1; } else { v[2] += q1 - kAliasUnits; }
  }
  uint64_t ex[3], tot[3];
  cta_scan3(v, ex, tot, sh);
  if (threadIdx.x == 0) {
    blk[3 * blockIdx.x + 0] = tot[0];
    blk[3 * blockIdx.x + 1] = tot[1];
    blk[3 * blockIdx.x + 2] = tot[2];
  }
}

// Scan of the block triples: segment totals, their exclusive scan (one CTA,
// which also writes the grand totals), then exclusive prefixes in place.
__global__ void __launch_bounds__(kSegT) k_alias_seg_reduce(const uint64_t *__restrict__ blk, size_t count,
                                                            uint64_t *__restrict__ seg) {
  __shared__ uint64_t sh[64][3];
  const size_t base = size_t(blockIdx.x) * kSeg + size_t(threadIdx.x) * kSegPer;
  uint64_t v[3] = {0, 0, 0};
  for (int j = 0; j < kSegPer; j++)
    if (base + j < count)
      for (int c = 0; c < 3; c++) v[c] += blk[3 * (base + j) + c];
  uint64_t ex[3], tot[3];
  cta_scan3(v, ex, tot, sh);
  if (threadIdx.x == 0)
    for (int c = 0; c < 3; c++) seg[3 * blockIdx.x + c] = tot[c];
}

__global__ void __launch_bounds__(kSegT) k_alias_seg_top(uint64_t *__restrict__ seg, size_t count,
                                                         uint64_t *__restrict__ totals) {
  __shared__ uint64_t sh[64][3];
  uint64_t carry[3] = {0, 0, 0};
  for (size_t b = 0; b < count; b += kSegT) {
    const size_t i = b + threadIdx.x;
    uint64_t v[3] = {0, 0, 0};
    if (i < count)
      for (int c = 0; c < 3; c++) v[c] = seg[3 * i + c];
    uint64_t ex[3], tot[3];
    cta_scan3(v, ex, tot, sh);
    if (i < count)
      for (int c = 0; c < 3; c++) seg[3 * i + c] = carry[c] + ex[c];
    for (int c = 0; c < 3; c++) carry[c] += tot[c];
  }
  if (threadIdx.x == 0) {
    for (int c = 0; c < 3; c++) totals[c] = carry[c];
    totals[3] = 0;
  }
}

__global__ void __launch_bounds__(kSegT) k_alias_seg_apply(uint64_t *__restrict__ blk, size_t count,
                                                           const uint64_t *__restrict__ seg) {
  __shared__ uint64_t sh[64][3];
  const size_t base = size_t(blockIdx.x) * kSeg + size_t(threadIdx.x) * kSegPer;
  uint64_t loc[kSegPer][3];
  uint64_t v[3] = {0, 0, 0};
  for (int j = 0; j < kSegPer; j++)
    for (int c = 0; c < 3; c++) {
      loc[j][c] = (base + j < count) ? blk[3 * (base + j) + c] : 0;
      v[c] += loc[j][c];
    }
  uint64_t ex[3], tot[3];
  cta_scan3(v, ex, tot, sh);
  uint64_t run[3];
  for (int c = 0; c < 3; c++) run[c] = ex[c] + seg[3 * blockIdx.x + c];
  for (int j = 0; j < kSegPer; j++)
    if (base + j < count)
      for (int c = 0; c < 3; c++) {
        blk[3 * (base + j) + c] = run[c];
        run[c] += loc[j][c];
      }
}

// Places every item in its list: light items (rank k) get keys[k] = deficit
// prefix before them, qv[k] = Q, idx[k] = item; heavy items (rank j) get
// keys[a + j] = excess prefix including them, idx[a + j] = item.  A block's
// records are gathered in shared memory (lights first, then heavies, each in
// index order) and written out as two contiguous runs.
constexpr uint32_t kPlaceSmem = kABlock * (8 + 4 + 4);

__global__ void __launch_bounds__(kAT, 3) k_alias_place(const float2 *__restrict__ amp, int n, float s_hi,
                                                     float s_lo, const uint64_t *__restrict__ blkpre,
                                                     const uint64_t *__restrict__ totals,
                                                     uint64_t *__restrict__ keys, uint32_t *__restrict__ qv,
                                                     uint32_t *__restrict__ idx) {
  extern __shared__ __align__(16) uint8_t smem[];
  float2 *tile = reinterpret_cast<float2 *>(smem);             // first 32 KiB, then reused:
  uint64_t *s_key = reinterpret_cast<uint64_t *>(smem);        //   keys, 8 B per record
  uint32_t *s_q = reinterpret_cast<uint32_t *>(smem + kABlock * 8);
  uint32_t *s_idx = reinterpret_cast<uint32_t *>(smem + kABlock * 12);
  __shared__ uint64_t sh[64][3];
  const uint64_t N = uint64_t(1) << n;
  const uint64_t start = uint64_t(blockIdx.x) * kABlock;
  const uint32_t cnt = uint32_t(umin(kABlock, N - start));
  // amplitude pair pr sits at pr ^ ((pr >> 3) & 7) in shared memory, so the
  // eight pairs a thread reads below fall in distinct banks across a phase
  {
    const float4 *a4 = reinterpret_cast<const float4 *>(amp + start);
    float4 *t4 = reinterpret_cast<float4 *>(tile);
    float4 f[kABlock / 2 / kAT];
#pragma unroll
    for (uint32_t r = 0; r < kABlock / 2 / kAT; r++) {
      const uint32_t pr = r * kAT + threadIdx.x;
      if (2 * pr < cnt) f[r] = a4[pr];
    }
#pragma unroll
    for (uint32_t r = 0; r < kABlock / 2 / kAT; r++) {
      const uint32_t pr = r * kAT + threadIdx.x;
      if (2 * pr < cnt) t4[pr ^ ((pr >> 3) & 7u)] = f[r];
    }
  }
  __syncthreads();
  // thread t owns items [16t, 16t + 16) of the block (pairs 8t .. 8t + 7), in index order
  const uint32_t t = threadIdx.x;
  const uint32_t first = t * kAPer;
  uint64_t q[kAPer];
  uint64_t v[3] = {0, 0, 0};
  const float4 *t4 = reinterpret_cast<const float4 *>(tile);
#pragma unroll
  for (uint32_t j = 0; j < kAPer / 2; j++) {
    if (first + 2 * j < cnt) {
      const float4 f = t4[(first >> 1) + (j ^ (t & 7u))];
      q[2 * j] = quantise(make_float2(f.x, f.y), s_hi, s_lo);
      q[2 * j + 1] = quantise(make_float2(f.z, f.w), s_hi, s_lo);
    } else {
      q[2 * j] = q[2 * j + 1] = 0;
    }
  }
#pragma unroll
  for (uint32_t j = 0; j < kAPer; j++) {
    if (first + j >= cnt) break;
    if (q[j] < kAliasUnits) { v[0]++; v[1] += kAliasUnits - q[j]; } else { v[2] += q[j] - kAliasUnits; }
  }
  uint64_t ex[3], tot[3];
  cta_scan3(v, ex, tot, sh);  // ends with a barrier: the tile is free from here on
  const uint32_t nl = uint32_t(tot[0]);  // light items of this block
  const uint64_t base_l = blkpre[3 * blockIdx.x + 0];
  uint32_t kl = uint32_t(ex[0]);                       // local light rank
  uint32_t jh = first - uint32_t(ex[0]);               // local heavy rank
  uint64_t dp = blkpre[3 * blockIdx.x + 1] + ex[1];    // deficit prefix before the next light item
  uint64_t ep = blkpre[3 * blockIdx.x + 2] + ex[2];    // excess prefix before the next heavy item
#pragma unroll
  for (uint32_t j = 0; j < kAPer; j++) {
    if (first + j >= cnt) break;
    const uint32_t i = uint32_t(start + first + j);
    if (q[j] < kAliasUnits) {
      s_key[kl] = dp;
      s_q[kl] = uint32_t(q[j]);
      s_idx[kl] = i;
      dp += kAliasUnits - q[j];
      kl++;
    } else {
      ep += q[j] - kAliasUnits;
      s_key[nl + jh] = ep;
      s_idx[nl + jh] = i;
      jh++;
    }
  }
  __syncthreads();
  const uint64_t a = totals[0];
  const uint64_t base_h = a + (start - base_l);  // heavy records of this block start here
  for (uint32_t x = threadIdx.x; x < cnt; x += kAT) {
    if (x < nl) {
      keys[base_l + x] = s_key[x];
      qv[base_l + x] = s_q[x];
      idx[base_l + x] = s_idx[x];
    } else {
      keys[base_h + (x - nl)] = s_key[x];
      idx[base_h + (x - nl)] = s_idx[x];
    }
  }
}

// Number of A elements among the first d of the merge of A (a) and B (b),
// A first on ties.
__device__ __forceinline__ uint64_t merge_split(const uint64_t *A, uint64_t a, const uint64_t *B, uint64_t b,
                                                uint64_t d) {
  uint64_t lo = d > b ? d - b : 0, hi = d < a ? d : a;
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1;
    if (A[mid] <= B[d - 1 - mid]) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// splits[b] = A elements among the first 1024 b merged items, for every merge CTA boundary.
__global__ void __launch_bounds__(256) k_alias_splits(const uint64_t *__restrict__ keys,
                                                      const uint64_t *__restrict__ totals, int n,
                                                      uint64_t n_splits, uint64_t *__restrict__ splits) {
  const uint64_t x = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (x >= n_splits) return;
  const uint64_t N = uint64_t(1) << n;
  const uint64_t a = totals[0], b = N - a;
  splits[x] = merge_split(keys, a, keys + a, b, umin(x * kMItems, N));
}

__device__ __forceinline__ uint64_t pack_entry(uint64_t own, uint32_t alias) { return (own << 32) | alias; }

// The table from the two lists (see the header).  Merged items
// [1024 blockIdx.x, +1024) per CTA; thread t takes 8 of them.
__global__ void __launch_bounds__(kMT) k_alias_merge(const uint64_t *__restrict__ keys,
                                                     const uint32_t *__restrict__ qv,
                                                     const uint32_t *__restrict__ idx,
                                                     const uint64_t *__restrict__ splits,
                                                     uint64_t *__restrict__ totals, int n,
                                                     uint64_t *__restrict__ table) {
  __shared__ uint64_t sA[kMItems + 1], sB[kMItems];
  __shared__ uint32_t sAq[kMItems], sAi[kMItems], sBi[kMItems + 1];
  const uint64_t N = uint64_t(1) << n;
  const uint64_t a = totals[0], b = N - a, dtot = totals[1];
  if (b == 0) {  // no heavy item: the state has no weight
    if (threadIdx.x == 0) totals[3] = 1;
    return;
  }
  const uint64_t *A = keys, *B = keys + a;
  const uint32_t *Ai = idx, *Bi = idx + a;
  const uint64_t d0 = uint64_t(blockIdx.x) * kMItems, d1 = umin(d0 + kMItems, N);
  const uint64_t ka0 = splits[blockIdx.x], ka1 = splits[blockIdx.x + 1];
  const uint64_t jb0 = d0 - ka0, jb1 = d1 - ka1;
  const uint32_t nA = uint32_t(ka1 - ka0), nB = uint32_t(jb1 - jb0);
  // segment loads: every thread issues all of its loads before storing any
  {
    uint64_t ka[kMPer], kb[kMPer];
    uint32_t qa[kMPer], ia[kMPer], ib[kMPer];
#pragma unroll
    for (int r = 0; r < kMPer; r++) {
      const uint32_t x = r * kMT + threadIdx.x;
      if (x < nA) { ka[r] = A[ka0 + x]; qa[r] = qv[ka0 + x]; ia[r] = Ai[ka0 + x]; }
      if (x < nB) { kb[r] = B[jb0 + x]; ib[r] = Bi[jb0 + x]; }
    }
#pragma unroll
    for (int r = 0; r < kMPer; r++) {
      const uint32_t x = r * kMT + threadIdx.x;
      if (x < nA) { sA[x] = ka[r]; sAq[x] = qa[r]; sAi[x] = ia[r]; }
      if (x < nB) { sB[x] = kb[r]; sBi[x] = ib[r]; }
    }
  }
  if (threadIdx.x == 0) {
    sA[nA] = ka1 < a ? A[ka1] : dtot;      // deficit prefix after the segment's last light item
    sBi[nB] = jb1 < b ? Bi[jb1] : Bi[b - 1];  // heavy item after the segment (clamped)
  }
  __syncthreads();
  const uint32_t tot_items = nA + nB;
  const uint32_t dd0 = umin(uint64_t(threadIdx.x) * kMPer, tot_items);
  const uint32_t dd1 = umin(uint64_t(dd0) + kMPer, tot_items);
  uint32_t ka, jb;
  {
    uint32_t lo = dd0 > nB ? dd0 - nB : 0, hi = dd0 < nA ? dd0 : nA;
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (sA[mid] <= sB[dd0 - 1 - mid]) lo = mid + 1; else hi = mid;
    }
    ka = lo;
    jb = dd0 - lo;
  }
  // entries in registers first; slot < nA: light item ka, else heavy item slot - nA
  uint64_t ent[kMPer];
  uint32_t slot[kMPer];
#pragma unroll
  for (int st = 0; st < kMPer; st++) {
    if (dd0 + st >= dd1) break;
    const bool take_light = ka < nA && (jb >= nB || sA[ka] <= sB[jb]);
    if (take_light) {
      // heavy items before it in the merge: those with E_j < D_k
      ent[st] = pack_entry(sAq[ka], sBi[jb]);
      slot[st] = ka;
      ka++;
    } else {
      const uint64_t j = jb0 + jb;
      uint64_t own = kAliasUnits;
      uint32_t al = sBi[jb];
      if (j + 1 < b) {
        const uint64_t dc = sA[ka];  // deficit prefix after the light items with D_k <= E_j
        const uint64_t e = sB[jb];
        if (dc > e) {
          own = kAliasUnits - (dc - e);
          al = sBi[jb + 1];
        }
      }
      ent[st] = pack_entry(own, al);
      slot[st] = nA + jb;
      jb++;
    }
  }
  // gather the entries in list order (reusing sA), then write each list with
  // consecutive threads on consecutive ranks: increasing, nearby table indices
  __syncthreads();
#pragma unroll
  for (int st = 0; st < kMPer; st++)
    if (dd0 + st < dd1) sA[slot[st]] = ent[st];
  __syncthreads();
  for (uint32_t x = threadIdx.x; x < tot_items; x += kMT)
    table[x < nA ? sAi[x] : sBi[x - nA]] = sA[x];
}

__global__ void __launch_bounds__(256) k_alias_sample(const uint64_t *__restrict__ table, int n,
                                                      const double *__restrict__ u, uint64_t seed,
                                                      int use_seed, uint64_t shots,
                                                      uint64_t *__restrict__ out) {
  const uint64_t s = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= shots) return;
  const uint64_t N = uint64_t(1) << n;
  const double us = use_seed ? splitmix_uniform(seed, s) : u[s];
  double x = us * double(N);
  if (!(x >= 0.0)) x = 0.0;
  uint64_t i = x < double(N) ? uint64_t(x) : N - 1;
  const double f = x - double(i);
  const uint64_t e = table[i];
  out[s] = (f * 2147483648.0 < double(e >> 32)) ? i : (e & 0xffffffffull);
}

}  // namespace

size_t alias_blocks(int n) {
  const uint64_t N = uint64_t(1) << n;
  return size_t((N + kABlock - 1) / kABlock);
}

size_t alias_segments(int n) { return (alias_blocks(n) + kSeg - 1) / kSeg; }

size_t alias_splits(int n) {
  const uint64_t N = uint64_t(1) << n;
  return size_t((N + kMItems - 1) / kMItems + 1);
}

cudaError_t launch_alias_build(const float2 *amp, int n, float s_hi, float s_lo, const AliasScratch &sc,
                               uint64_t *table, cudaStream_t st) {
  if (n < 1 || n > 32) return cudaErrorInvalidValue;
  const uint64_t N = uint64_t(1) << n;
  const size_t nblk = alias_blocks(n), nseg = alias_segments(n);
  k_alias_count<<<unsigned(nblk), kAT, 0, st>>>(amp, n, s_hi, s_lo, sc.blk);
  k_alias_seg_reduce<<<unsigned(nseg), kSegT, 0, st>>>(sc.blk, nblk, sc.seg);
  k_alias_seg_top<<<1, kSegT, 0, st>>>(sc.seg, nseg, sc.tot);
  k_alias_seg_apply<<<unsigned(nseg), kSegT, 0, st>>>(sc.blk, nblk, sc.seg);
  static std::atomic<uint64_t> configured{0};  // devices whose opt-in is set (bit per device)
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 64 || !((configured.load() >> dev) & 1ull)) {
    e = cudaFuncSetAttribute(k_alias_place, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kPlaceSmem));
    if (e != cudaSuccess) return e;
    if (dev < 64) configured.fetch_or(1ull << dev);
  }
  k_alias_place<<<unsigned(nblk), kAT, kPlaceSmem, st>>>(amp, n, s_hi, s_lo, sc.blk, sc.tot, sc.keys, sc.qv,
                                                         sc.idx);
  const uint64_t nm = (N + kMItems - 1) / kMItems;
  k_alias_splits<<<unsigned((nm + 1 + 255) / 256), 256, 0, st>>>(sc.keys, sc.tot, n, nm + 1, sc.splits);
  k_alias_merge<<<unsigned(nm), kMT, 0, st>>>(sc.keys, sc.qv, sc.idx, sc.splits, sc.tot, n, table);
  count_launch(7);
  return cudaGetLastError();
}

cudaError_t launch_alias_sample(const uint64_t *table, int n, const double *u, uint64_t seed, int use_seed,
                                uint64_t shots, uint64_t *out, cudaStream_t st) {
  if (shots == 0) return cudaSuccess;
  const uint64_t grid = (shots + 255) / 256;
  if (grid > 0x7fffffffull) return cudaErrorInvalidValue;
  k_alias_sample<<<unsigned(grid), 256, 0, st>>>(table, n, u, seed, use_seed, shots, out);
  count_launch();
  return cudaGetLastError();
}

}  // namespace svgb
