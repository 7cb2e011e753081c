// sv_internal.h -- plan format shared by the host planner and the kernels.
//
// A circuit becomes a list of passes.  A pass is one HBM sweep of the state:
// every CTA owns a tile of 2^T amplitudes whose indices agree on all qubits
// outside the pass's tile set Q (|Q| = T, Q always holds the c lowest qubits so
// each global access is a run of 2^c contiguous amplitudes).  The CTA loads its
// tile into shared memory, applies the pass's ops in order, and stores it back.
//
// Ops act on tile-local bit positions (local bit j <-> physical qubit lq[j]):
//   OP_DENSE  a fused k-qubit block (k <= 5), complex64 2^k x 2^k matrix,
//             matrix bit m <-> local bit lb[m];
//   OP_PHASE  a product of diagonal gates whose terms each touch at most one
//             tile qubit (the others are fixed per CTA); phases are stored as
//             32-bit fractions of a turn so sums wrap exactly modulo 2*pi;
//   OP_RPHASE the register-stage form of a diagonal product (KIND_REG and
//             KIND_TC passes): terms may touch two tile qubits, and are
//             pre-classified by the stage's register bits (RegPhaseHdr); the
//             terms on tile qubits only are pre-summed per thread, those on
//             outer qubits are summed once per tile (RegPhaseSlot).
#pragma once

#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

namespace svgb {

// Kernels launched by this library in this process (all devices).
extern std::atomic<uint64_t> g_launches;
inline void count_launch(uint64_t k = 1) { g_launches.fetch_add(k, std::memory_order_relaxed); }

enum : uint8_t { OP_DENSE = 1, OP_PHASE = 2, OP_RPHASE = 3 };

constexpr int kMaxTile = 13;   // largest T (64 KiB of complex64 in shared memory)
constexpr int kMaxK = 5;       // largest fused block

enum : uint32_t { KIND_SMEM = 0, KIND_REG = 1, KIND_TC = 2 };


struct alignas(16) PlanPass {
  uint64_t outer_mask;  // physical qubits outside the tile (within n)
  uint64_t high_mask;   // tile qubits >= c (their ascending order = local bits c..T-1)
  uint64_t n_tiles;     // 2^(n-T)
  uint32_t T;           // tile qubits
  uint32_t c;           // low qubits (0..c-1) in every tile
  uint32_t n_ops;
  uint32_t ops_off;     // byte offset of OpRec[n_ops] from the plan base
  uint32_t kmax;        // largest dense k in this pass
  uint32_t n_phase_terms;
  uint32_t kind;        // KIND_SMEM: ops sweep the shared-memory tile one by one;
                        // KIND_REG: register stages (see StageRec)
  uint32_t R;           // KIND_REG: amplitudes per thread = 2^R
  uint32_t n_stages;
  uint32_t stages_off;  // byte offset of StageRec[n_stages]
  uint32_t data_bytes;  // bytes from ops_off to the end of this pass's records
  uint32_t w_off;       // KIND_REG / KIND_TC: byte offset of the pass's outer-term slot
                        // table (RegPhaseSlot), 0 when no phase op has outer terms
  uint32_t aux_off;     // batched plans, KIND_REG passes: byte offset of the pass's
                        // RegPassParams from the circuit's plan base (0 otherwise)
  uint32_t n_w;         // slots in the table at w_off
  int8_t lq[32];        // local bit -> physical qubit
};

// One register stage of a KIND_REG pass.  Thread t of the CTA holds the 2^R
// amplitudes with local index l = la[j] | dep(t, tb), j < 2^R: register bit i
// is local bit rb[i], thread-index bit i is local bit tb[i].  Ops of the stage
// act on registers only.  Between stages the tile is exchanged through shared
// memory at the XOR-swizzled index swz(l) = pa[j] ^ swz(dep(t, tb)).  The
// first stage loads from HBM and the last stores to HBM directly (their
// thread bits start with the low tile bits, so a warp touches contiguous runs).
struct alignas(16) StageRec {
  uint8_t rb[5];
  uint8_t tb[11];
  uint16_t pa[32];
  uint16_t la[32];
  uint32_t op_begin, op_end;
  uint32_t flags;       // bit 0: load from HBM, bit 1: store to HBM,
                        // bit 2: KIND_TC stage with a tensor-core product
  uint32_t b_off;       // KIND_TC: byte offset of the stage's 8 KB B_hi/B_lo image
  uint32_t xo[32];      // pa[j] * 8: byte offset of register amplitude j in the exchange buffer
};

// Tile-invariant address tables of a KIND_REG pass, passed to the kernel by
// value (its loops over j and k unroll, so every entry is a compile-time
// constant-bank operand).  A thread adds its own part once per CTA.
struct RegPassParams {
  uint32_t lo[32];      // first stage: la[j] * 8, byte offset in the natural-order tile
  uint64_t go[32];      // last stage: amplitude offset of la[j] from the tile base in HBM
  uint64_t ko[16];      // prefetch: amplitude offset of 16-byte chunk row k (chunks k*NT..)
  uint8_t oq[16];       // store: physical qubit written from local bit x (SWAPs folded in)
  uint32_t chk[4];      // the host's T, n_stages, data_bytes, ops_off of this pass: the kernel
                        // compares them with the device copy before using the records
};

// Columns of the shared-memory swizzle: local bit b < 4 maps to itself, local
// bit b >= 4 additionally flips the bank-pair bits swz_col(b) (distinct, not a
// single bit), so any 8 local bits include 4 whose bank-pair images are
// independent -- the lanes of a half-warp can always be chosen conflict-free.
// kSwz nibble i (bits 4i..4i+3) is the image of local bit 4 + i.
constexpr uint64_t kSwz = 0x1fedb7ca9653ull;
__host__ __device__ inline uint32_t swz_col(int b) {
  return b < 4 ? (1u << b) : uint32_t((kSwz >> (4 * (b - 4))) & 15u);
}
__host__ __device__ inline uint32_t swz(uint32_t l) {
  uint32_t x = l;
  for (int b = 4; b < 16; b++)
    if ((l >> b) & 1u) x ^= swz_col(b);
  return x;
}

// Load-buffer swizzle of tensor-core passes, at 16-byte granularity: local bit
// 0 stays in place (a 16-byte cp.async chunk holds local indices 2q and 2q + 1),
// bits 1..3 map to themselves, and a bit b >= 4 also flips bits 1..3 by
// swzl_col(b) (a nonzero 3-bit pattern, 3 bits per b in kSwzL), so a first stage
// whose registers hold low tile bits still reads the load buffer conflict-free:
// the planner gives its half-warp lanes bits with independent images.
constexpr uint64_t kSwzL = 0xae23f5711ull;  // b = 4..15: 1, 2, 4, 3, 5, 6, 7, 1, 2, 4, 3, 5
__host__ __device__ constexpr uint32_t swzl_col(int b) {
  return b < 4 ? (1u << b) : uint32_t(((kSwzL >> (3 * (b - 4))) & 7u) << 1);
}
__host__ __device__ constexpr uint32_t swzl(uint32_t l) {
  uint32_t x = l;
  for (int b = 4; b < 16; b++)
    if ((l >> b) & 1u) x ^= swzl_col(b);
  return x;
}

struct alignas(16) OpRec {
  uint8_t type;
  uint8_t k;
  uint8_t lb[5];        // DENSE: local bits, matrix bit m <-> lb[m]
  uint8_t rmask;        // DENSE in a KIND_REG pass: register positions (matrix bits in
                        // ascending register order)
  uint32_t data_off;    // DENSE: byte offset of the row-major matrix: float2 (re, im) per
                        // element, or in KIND_REG passes float4 (re, re, -im, im);
                        // PHASE: of PhaseTerm[]; RPHASE: of RegPhaseHdr + tables
  uint32_t count;       // PHASE: number of terms
};

struct alignas(16) PhaseTerm {
  uint64_t outer_mask;  // outer qubits that must all be 1 for the term to apply
  int32_t la;           // local bit that must be 1 (-1: none)
  uint32_t turn;        // phase as a fraction of 2*pi, scaled by 2^32
};

// OP_RPHASE record, relative to the stage holding it (register bits rb[0..R-1],
// thread bits tb[0..ntb-1], ntb = T - R).  The phase of register amplitude j of
// thread t is
//     2*pi/2^32 * ( a_0 + sum_{i: bit i of j} a_{1+i} ) + arg D[j]
// where class 0 holds the terms on no register bit and class 1+i those on
// register bit i (a term touches at most two qubits, so at most one register
// bit once the terms on register bits only are folded into D[j]), and a_k is
// the sum of the turns of class k's terms that apply to this thread in this
// tile (their outer qubits all 1 in the tile, their thread-local bits all 1 in
// t's local index):
//   * terms on tile qubits only: summed per thread by the planner, a table of
//     nt turns per class with such terms (bit k of pre_mask), after the header
//     in ascending k;
//   * terms on outer qubits: summed once per tile (the sum depends on the tile
//     only) into the pass's slots w_slot.. (RegPhaseSlot): slot 0 takes class
//     0's terms without a thread bit, slot 1 + i those on thread bit i (added
//     by the threads whose bit i is 1), slot 1 + ntb + r class 1+r's terms;
//     bit 0 of w_used marks slot 0 used, bit 1 any of slots 1..ntb, bit 2 + r
//     slot 1 + ntb + r.
// Sums are of 32-bit turn fractions modulo 2^32, so their order does not
// matter: every grouping gives the same a_k.
struct alignas(16) RegPhaseHdr {
  uint32_t pre_mask;    // classes with a per-thread table
  uint32_t w_used;      // outer-term slots in use (see above)
  uint32_t w_slot;      // first of this op's 1 + ntb + R slots
  uint32_t has_d;       // D differs from the identity
  uint32_t ntb;         // thread bits of the stage (T - R)
  uint32_t nt;          // threads of the stage (2^ntb): the tables' length
  uint32_t pad_[2];
  float2 d[32];         // register-only diagonal (2^R entries used)
};

// A pass's phase terms on outer qubits (KIND_REG and KIND_TC passes), at
// PlanPass.w_off: RegPhaseSlot[n_w] (each a range of the term array), then
// 2 x n_w uint32 of per-tile sums (a scratch area: the kernels write it in
// their shared-memory copy of the records, alternating halves tile by tile),
// then the terms.  rphase_w_sums / rphase_w_terms give the byte offsets of the
// last two from w_off.
struct alignas(8) RegPhaseSlot {
  uint32_t begin, end;  // term indices [begin, end)
};
struct alignas(16) RegPhaseOuter {
  uint64_t outer_mask;  // outer qubits that must all be 1 in the tile
  uint32_t turn;        // fraction of 2*pi, scaled by 2^32
  uint32_t pad_;
};
__host__ __device__ constexpr uint32_t rphase_w_sums(uint32_t n_w) { return (8u * n_w + 15u) & ~15u; }
__host__ __device__ constexpr uint32_t rphase_w_terms(uint32_t n_w) {
  return rphase_w_sums(n_w) + ((8u * n_w + 15u) & ~15u);
}

static_assert(sizeof(RegPhaseHdr) == 288, "RegPhaseHdr layout");
static_assert(sizeof(RegPhaseOuter) == 16, "RegPhaseOuter layout");
static_assert(sizeof(RegPhaseSlot) == 8, "RegPhaseSlot layout");
static_assert(sizeof(PlanPass) == 112, "PlanPass layout");
static_assert(sizeof(StageRec) == 288, "StageRec layout");
static_assert(sizeof(OpRec) == 16, "OpRec layout");
static_assert(sizeof(PhaseTerm) == 16, "PhaseTerm layout");

// Norm tracking across the tensor-core passes of one unitary circuit.  The
// tensor cores' float32 accumulation rounds toward zero, so every stage product
// shrinks the state by ~1e-7 of its norm, while a unitary circuit keeps
// ||psi||^2.  The circuit's first tensor-core pass sums |a|^2 of what it loads
// into in_sum; every tracked pass sums |a|^2 of what it stores into out_sum; a
// later pass scales what it loads by sqrt(*ref / *prev) (ref: the first pass's
// input sum, prev: the previous tracked pass's output sum).  So the drift of
// every pass but the last is undone as the next pass reads the state, and no
// extra pass over the state is needed.  All pointers are device doubles; null
// disables the corresponding step.
struct TcNorm {
  double *in_sum = nullptr;        // zeroed before the pass
  const double *ref = nullptr;     // with prev: the scale's numerator
  const double *prev = nullptr;    // the previous tracked pass's output sum
  double *out_sum = nullptr;       // zeroed before the pass
  double *clear = nullptr;         // set to zero by this pass (the next pass's out_sum)
};

// Launch one pass kernel (sv_apply.cu).  plan_dev/pass_off locate the PlanPass;
// host_pass is the same record on the host (for grid size and template choice).
// `norm` applies to tensor-core passes only (may be null).
cudaError_t launch_pass(float2 *amp, const uint8_t *plan_dev, uint32_t pass_off,
                        const PlanPass &host_pass, const RegPassParams *reg_params, int *err,
                        cudaStream_t stream, const TcNorm *norm = nullptr);
// Whether a tensor-core pass fits the kernel's shared memory.
bool tc_pass_fits(uint32_t T, uint32_t c, uint32_t n_stages, uint32_t data_bytes, uint32_t R);
// Whether a register-stage pass fits the persistent kernel's shared-memory tables.
bool reg_pass_fits(uint32_t T, uint32_t c, uint32_t R, uint32_t n_stages, uint32_t data_bytes);

// Measurement kernels (sv_measure.cu).
struct MeasureScratch {
  double *chunk = nullptr;   // 2^(n-6) sums of 64 amplitudes
  double *block = nullptr;   // 2^(n-12) inclusive prefix of 4096-amplitude block sums
  double *part = nullptr;    // per-CTA partials for reductions / scan carries
  uint64_t *counter = nullptr;
  size_t n_chunk = 0, n_block = 0, n_part = 0;
};

constexpr int kChunkBits = 6;   // 64 amplitudes
constexpr int kBlockBits = 12;  // 4096 amplitudes = 64 chunks

cudaError_t launch_reduce_pz(const float2 *amp, int n, uint64_t zmask, double *part,
                             size_t n_part, double *out2, cudaStream_t st);
// <X^x Z^z> with x_mask != 0 (Y on qubits in both masks), one read of the state:
// out2[0] = sum |psi|^2, out2[1] = half of <psi|P|psi> (see sv_measure.cu).
cudaError_t launch_reduce_pauli(const float2 *amp, int n, uint64_t x_mask, uint64_t z_mask, double *part,
                                size_t n_part, double *out2, cudaStream_t st);
// Builds the CDF; with ztotal_dev, the same read also writes
// sum p_i * (-1)^popcount(i & zmask) to ztotal_dev[0].
cudaError_t launch_build_cdf(const float2 *amp, int n, MeasureScratch &ms, double *total_dev,
                             cudaStream_t st, uint64_t zmask = 0, double *ztotal_dev = nullptr);
cudaError_t launch_sample(const float2 *amp, int n, const MeasureScratch &ms,
                          const double *total_dev, const double *u, uint64_t seed, int use_seed,
                          uint64_t shots, uint64_t *out, uint64_t *n_boundary, cudaStream_t st);
cudaError_t launch_probabilities(const float2 *amp, uint64_t offset, uint64_t count, double *out,
                                 cudaStream_t st);
cudaError_t launch_reset(float2 *amp, int n, uint64_t basis, cudaStream_t st);
// Partitioned blocks (sv_pblock.cu): out = a (x) b (a on the low qubits), and
// removal of qubit q known to be in |v>.
cudaError_t launch_kron(const float2 *a, int na, const float2 *b, int nb, float2 *out, cudaStream_t st);
cudaError_t launch_take(const float2 *psi, int n, int q, int v, float2 *out, cudaStream_t st);
// Collapse after a one-qubit measurement (see k_collapse).
cudaError_t launch_collapse(float2 *amp, int n, int q, int outcome, int to_zero, float scale,
                            cudaStream_t st);

size_t reduce_parts(int n);
// Amplitudes per reduction CTA (k_reduce_pz): reduce_parts(n) = ceil(2^n / kReduceCtaAmps).
constexpr uint64_t kReduceCtaAmps = 4096;
constexpr uint64_t reduce_parts_c(int n) { return ((uint64_t(1) << n) + kReduceCtaAmps - 1) / kReduceCtaAmps; }

// Walker alias table (sv_alias.cu).  Entry i of the table packs
// (own_i << 32) | alias_i: bucket i keeps own_i of its 2^31 units for outcome
// i and gives the rest to outcome alias_i.
constexpr uint64_t kAliasUnits = uint64_t(1) << 31;
struct AliasScratch {
  uint64_t *blk = nullptr;   // 3 per 4096-item block: light count, deficit sum, excess sum
  uint64_t *seg = nullptr;   // 3 per scan segment
  uint64_t *tot = nullptr;   // [0] light items, [1] total deficit, [2] total excess, [3] error
  uint64_t *keys = nullptr;  // N: deficit prefixes of light items, then excess prefixes of heavy ones
  uint32_t *qv = nullptr;    // N: Q of light items, by light rank
  uint32_t *idx = nullptr;   // N: item index of light items, then of heavy items
  uint64_t *splits = nullptr;  // merge-path split per merge CTA boundary (alias_splits(n))
};
size_t alias_blocks(int n);
size_t alias_segments(int n);
size_t alias_splits(int n);
// Queues the table build for weights |a_i|^2 * (s_hi + s_lo) (s = N / sum |a|^2).
cudaError_t launch_alias_build(const float2 *amp, int n, float s_hi, float s_lo, const AliasScratch &sc,
                               uint64_t *table, cudaStream_t st);
// Draws with uniforms u (or counter-based SplitMix64 from seed when use_seed).
cudaError_t launch_alias_sample(const uint64_t *table, int n, const double *u, uint64_t seed, int use_seed,
                                uint64_t shots, uint64_t *out, cudaStream_t st);

#ifdef __CUDACC__
// Counter-based SplitMix64 uniform for draw s of `seed`: 53 bits in [0, 1).
__device__ __forceinline__ double splitmix_uniform(uint64_t seed, uint64_t s) {
  uint64_t z = seed + (s + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return double(z >> 11) * (1.0 / 9007199254740992.0);
}
#endif

// Records the calling thread's sv_last_error() message (sv_capi.cu); returns code.
int set_last_error(int code, const char *fmt, ...);

}  // namespace svgb
