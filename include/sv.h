/*
 * sv.h -- C-ABI of the GB300 state-vector library (libsvgb.so).
 *
 * The library keeps a 2^n complex amplitude vector resident in GPU memory,
 * applies a circuit given as a flat gate IR, and returns amplitudes,
 * probabilities, measurement samples or Pauli-string expectation values.  This is
 * the "circuit IR in; samples, expectations or amplitudes out" interface of
 * the paper's state-vector backend (§III-A common IR, §II state-vector method,
 * §III-B end-of-circuit sampling and cached-state expectation values).
 *
 * Conventions (all functions):
 *  - Every function returns SV_OK (0) or a negative sv_status and never aborts.
 *    On failure sv_last_error() describes the cause.
 *  - Qubit q is bit q of the amplitude index (little-endian).  Amplitudes are
 *    complex64 stored interleaved (re, im) as two float32 -- 8 bytes each.
 *  - Work is queued asynchronously on the state's CUDA stream.  Functions that
 *    return host values (sv_norm, sv_expect_pauli, sv_sample* into host
 *    buffers, sv_get_amplitudes/sv_probabilities into host buffers) synchronise
 *    the stream before returning.
 *  - Pointers passed in are owned by the caller and only read/written during
 *    the call (device outputs: until the stream reaches that point).  A state
 *    is owned by the library unless created with sv_wrap.
 *  - A CUDA error marks the state as poisoned: later calls on it return
 *    SV_ERR_STATE; only sv_destroy is allowed.
 *  - No function is thread-safe on the same state; distinct states may be used
 *    from distinct threads.  sv_last_error() is per thread.
 */
#ifndef SVGB_SV_H
#define SVGB_SV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sv_state sv_state; /* opaque */

enum sv_dtype { SV_C64 = 1, SV_C128 = 2 /* not supported: SV_ERR_UNSUPPORTED */ };

enum sv_status {
  SV_OK = 0,
  SV_ERR_ARG = -1,         /* invalid argument or invalid IR */
  SV_ERR_OOM = -2,         /* device or pinned-host allocation failed */
  SV_ERR_CUDA = -3,        /* a CUDA call failed; the state is now poisoned */
  SV_ERR_UNSUPPORTED = -4, /* valid request this build does not implement */
  SV_ERR_TIMEOUT = -5,     /* a bounded device-side wait gave up */
  SV_ERR_STATE = -6        /* the state was poisoned by an earlier failure */
};

/*
 * Gate kinds of the IR, with OpenQASM 2 semantics (the paper's front end takes
 * Qiskit circuits and OpenQASM 2, §III-A):
 *   U3(θ,φ,λ) = [[cos θ/2, -e^{iλ} sin θ/2], [e^{iφ} sin θ/2, e^{i(φ+λ)} cos θ/2]]
 *   RX, RY, RZ(θ) = exp(-iθP/2); P(λ) = diag(1, e^{iλ}); H, X, Y, Z, S, SDG, T, TDG.
 *   CX(c,t): q[0] = control, q[1] = target.  CZ, CP(λ) = diag(1,1,1,e^{iλ}), SWAP.
 *   UNITARY: a dense 2^nq x 2^nq matrix (nq <= 5) given by `mat`.
 * For a gate on q[0..nq-1], bit m of the matrix row/column index refers to
 * qubit q[m] (q[0] is the least significant matrix bit).
 */
enum sv_gate_kind {
  SV_GATE_U3 = 1, SV_GATE_H, SV_GATE_X, SV_GATE_Y, SV_GATE_Z, SV_GATE_S, SV_GATE_SDG,
  SV_GATE_T, SV_GATE_TDG, SV_GATE_RX, SV_GATE_RY, SV_GATE_RZ, SV_GATE_P, SV_GATE_CX,
  SV_GATE_CZ, SV_GATE_CP, SV_GATE_SWAP, SV_GATE_UNITARY
};

/* One IR gate (56 bytes; plain data). */
typedef struct sv_gate {
  uint8_t kind;       /* sv_gate_kind */
  uint8_t nq;         /* number of qubits: 1 or 2 for named kinds, 1..5 for UNITARY */
  uint16_t reserved;  /* must be 0 */
  int32_t q[5];       /* target qubits, distinct, each in [0, n) */
  double p[3];        /* angles (radians) for U3 (θ,φ,λ), RX/RY/RZ/P/CP (p[0]) */
  const double *mat;  /* UNITARY only: host pointer to 2^nq x 2^nq complex128,
                         row-major, interleaved (re, im); read during the call */
} sv_gate;

/* Options of sv_apply_circuit.  Zero fields take the library default. */
typedef struct sv_opts {
  int32_t k_max;       /* fusion width: gates are fused into dense blocks of at most
                          k_max qubits (1..5; default 2).  Per pass, blocks wider
                          than 2 qubits are formed only when their estimated cost
                          is lower (the register kernels run 1-2-qubit blocks
                          fastest); with precision 1 or 2, up to min(k_max, 4).  A gate
                          wider than the width keeps a block of its own. */
  int32_t tile_qubits; /* T: qubits held by one CTA tile in shared memory per HBM
                          pass (5..13; default 12; clamped to n) */
  int32_t low_qubits;  /* c: low qubits every tile contains, so each global access
                          is a run of 2^c contiguous amplitudes (1..T; default 5) */
  int32_t precision;   /* 0 = FP32 CUDA cores for every block;
                          2 = 3xTF32 tensor cores (tcgen05) on every pass that fits:
                          all dense blocks of a register stage as one 16x16 complex
                          product (tiles of 11..13 qubits; smaller states use the
                          CUDA-core kernels);
                          1 = as 2, except that with kernel_variant 0 a pass runs on
                          the FP32 CUDA-core register kernel when the planner
                          estimates that faster: light passes (blocks of at most 2
                          qubits, no phase ops, few stages), from a per-pass model
                          of both kernels' measured times;
                          with 1 and 2, when every gate is unitary the tensor-core
                          passes track ||psi||^2
                          (the tensor cores' float32 accumulation rounds toward
                          zero, ~1e-7 of the norm per stage): the first tensor-core
                          pass sums it on load, each pass on store, and each later
                          pass rescales what it loads by sqrt(input / previous
                          output), so only the last pass's drift remains -- no
                          extra reads of the state */
  int32_t kernel_variant; /* 0 = amplitudes stay in registers across the ops of a
                          stage, shared memory only between stages (default): 32
                          amplitudes per thread when a pass's blocks have at most 2
                          qubits and T <= 12, else 16;
                          1 = every op sweeps the shared-memory tile;
                          2 = register stages with 16 amplitudes per thread; with
                          precision 1 or 2: blocks fused up to min(k_max, 5) qubits and
                          5-qubit stages (32 x 32 complex products, 32 amplitudes
                          per thread, T = 12 or 13) on every tensor-core pass whose
                          records fit (at most four 32 KB stage images).  Without
                          it, precisions 1 and 2 use 4-qubit stages, and 5-qubit stages
                          only for a pass holding a 5-qubit block (a 5-qubit
                          UNITARY gate) */
} sv_opts;

/* Statistics of the fusion + pass plan of a circuit (host-side only). */
typedef struct sv_plan_info {
  uint64_t n_gates;    /* IR gates */
  uint64_t n_blocks;   /* dense fused blocks after fusion */
  uint64_t n_phase;    /* diagonal phase ops (gates whose qubits leave the tile) */
  uint64_t n_passes;   /* HBM passes (one read + one write of the state each) */
  uint64_t hist_k[6];  /* hist_k[k] = dense blocks with k qubits */
  uint64_t flops;      /* useful real flops of the dense blocks over the whole state */
  uint64_t bytes;      /* algorithmic HBM bytes: n_passes * 2 * 2^n * 8 */
  uint64_t upload_bytes; /* size of the packed plan copied host -> device per apply */
  uint64_t n_stages;   /* register stages over all register-stage passes */
  uint64_t tc_stages;  /* stages applied as one 3xTF32 tensor-core product (precision 1, 2) */
  uint64_t passes_by_kind[3]; /* passes run by the shared-memory sweep kernel, the
                                 register-stage kernel and the tensor-core kernel */
} sv_plan_info;

/* ---- lifetime ------------------------------------------------------------ */

/* Allocate a 2^n_qubits complex64 state on the current CUDA device (cudaMalloc;
 * 8 * 2^n bytes) and set it to |0...0>.  n_qubits in [1, 36].  cuda_stream is a
 * cudaStream_t (NULL = legacy default stream).  *out receives the handle. */
int sv_create(int n_qubits, int dtype, void *cuda_stream, sv_state **out);

/* Wrap a caller-owned device buffer of 2^n_qubits complex64 amplitudes (e.g. a
 * torch tensor's storage, 16-byte aligned).  The contents are used as-is; the
 * buffer must outlive the handle and is never freed by the library. */
int sv_wrap(void *dev_ptr, int n_qubits, int dtype, void *cuda_stream, sv_state **out);

/* Free the handle, its scratch buffers and (if owned) the amplitudes.  Waits
 * for the state's stream.  NULL is accepted. */
int sv_destroy(sv_state *s);

/* Change the stream later work is queued on; that stream first waits for the
 * work already queued on the old one. */
int sv_set_stream(sv_state *s, void *cuda_stream);

/* Wait for all queued work on the state's stream. */
int sv_synchronize(sv_state *s);

/* Set the state to the basis vector |basis_index> (< 2^n). */
int sv_reset(sv_state *s, uint64_t basis_index);

/* Number of qubits of the state (or SV_ERR_ARG). */
int sv_num_qubits(const sv_state *s);

/* Device pointer of the amplitudes (2^n complex64). */
void *sv_device_ptr(sv_state *s);

/* ---- apply --------------------------------------------------------------- */

/*
 * Apply gates ir[0..n_gates-1] in order:  psi <- U_{G-1} ... U_0 psi.
 * The host validates the IR (kinds, qubits distinct and < n, finite angles),
 * fuses gates into dense blocks of at most k_max qubits, groups blocks into
 * HBM passes whose qubits fit one shared-memory tile, and launches one kernel
 * per pass on the state's stream.  opts may be NULL.  Returns SV_ERR_ARG for
 * an invalid IR (nothing is applied).  Asynchronous.
 */
int sv_apply_circuit(sv_state *s, const sv_gate *ir, size_t n_gates, const sv_opts *opts);

/* Fusion + pass-plan statistics for a circuit on n qubits (no GPU work). */
int sv_plan_stats(int n_qubits, const sv_gate *ir, size_t n_gates, const sv_opts *opts,
                  sv_plan_info *out);

/* ---- readout ------------------------------------------------------------- */

/* ||psi||^2: |a_i|^2 formed exactly from the float32 parts, accumulated with
 * compensated float32 sums per 64 amplitudes and double precision above. */
int sv_norm(sv_state *s, double *out_norm2);

/* out[j] = |a_{offset+j}|^2 in double precision, j < count.  out is a device
 * pointer if out_on_device, else host memory. */
int sv_probabilities(sv_state *s, double *out, uint64_t offset, uint64_t count, int out_on_device);

/* Copy amplitudes [offset, offset+count) (complex64, interleaved) to out. */
int sv_get_amplitudes(sv_state *s, void *out, uint64_t offset, uint64_t count, int out_on_device);

/* Overwrite amplitudes [offset, offset+count) from in (complex64). */
int sv_set_amplitudes(sv_state *s, const void *in, uint64_t offset, uint64_t count, int in_on_device);

/*
 * Measure all qubits `shots` times from the current state (end-of-circuit
 * sampling, §III-B).  With the CDF C_i = sum_{j<=i} |a_j|^2 (double precision)
 * and uniform u in [0,1), a draw returns x = min{ i : C_i > u * C_{N-1} }.
 * sv_sample draws u_s (s = 0..shots-1) on the device from `seed` with
 * counter-based SplitMix64: u_s = (mix64(seed + (s+1)*0x9E3779B97F4A7C15) >> 11) * 2^-53.
 * sv_sample_uniforms takes the uniforms from the caller.  out_bitstrings[s]
 * receives x for draw s, in draw order.  out_n_boundary (may be NULL) receives
 * how many draws fell within 1e-9 of a CDF boundary of this state.
 * Buffers are device pointers if on_device, else host memory.
 */
int sv_sample(sv_state *s, uint64_t shots, uint64_t seed, uint64_t *out_bitstrings,
              int on_device);
int sv_sample_uniforms(sv_state *s, const double *uniforms, uint64_t shots,
                       uint64_t *out_bitstrings, uint64_t *out_n_boundary, int on_device);

/*
 * End-of-circuit readout from one read of the state (§III-B: all shots drawn
 * from the final state, expectation values from the same cached state): the
 * FP64 CDF built for sampling also accumulates, per 4096-amplitude block,
 * sum_i |a_i|^2 (-1)^popcount(i & z_mask).  Draws are exactly those of
 * sv_sample_uniforms with the same uniforms (shots may be 0: readout only);
 * *out_expect = <Z_mask> = that sum / sum_i |a_i|^2 and *out_norm2 =
 * sum_i |a_i|^2 (the CDF total; equal to sv_norm's value up to the order of the
 * double-precision additions).  z_mask bits must be < n_qubits (0 gives 1).
 * Synchronises.  SV_ERR_ARG for a zero-norm state or null outputs.
 */
int sv_sample_expect_z(sv_state *s, const double *uniforms, uint64_t shots, uint64_t *out_bitstrings,
                       uint64_t *out_n_boundary, int on_device, uint64_t z_mask, double *out_expect,
                       double *out_norm2);

/*
 * Alias sampling (§III-C: shots drawn by alias sampling at O(1) work per shot;
 * Walker 1974).  sv_alias_build snapshots the current state's outcome
 * distribution into a Walker alias table held by the state (8 bytes per basis
 * state; later changes to the state do not touch it until the next build).
 * Every bucket holds C = 2^31 units; outcome i weighs
 * Q_i = round(|a_i|^2 * N / W * 2^31) units (W = sum |a|^2); light outcomes
 * (Q < C) are taken in index order, each filling its bucket from the current
 * heavy outcome (Q >= C, index order); a heavy outcome left with fewer than C
 * units keeps them and is filled by the next heavy one; the last heavy outcome
 * keeps a full bucket.  The build synchronises the state's stream and returns
 * SV_ERR_ARG when the state's total weight is zero or not finite,
 * SV_ERR_UNSUPPORTED past 32 qubits, SV_ERR_OOM without room for the table
 * (8 B per amplitude) and the build's scratch (16 B per amplitude, freed
 * before return).
 *
 * sv_alias_sample / sv_alias_sample_uniforms draw from the last table built
 * (SV_ERR_ARG if none): with uniform u in [0,1), x = u * N, i = floor(x),
 * f = x - i, the draw is i when f * 2^31 < own_i, else alias_i.  Uniforms come
 * from `seed` by the SplitMix64 rule of sv_sample, or from the caller.
 * out_bitstrings[s] receives draw s; device pointers if on_device, else host
 * memory.
 *
 * sv_alias_table copies entries [offset, offset+count) of the table; entry i
 * packs (own_i << 32) | alias_i.  sv_alias_release frees the table.
 */
int sv_alias_build(sv_state *s);
int sv_alias_sample(sv_state *s, uint64_t shots, uint64_t seed, uint64_t *out_bitstrings, int on_device);
int sv_alias_sample_uniforms(sv_state *s, const double *uniforms, uint64_t shots,
                             uint64_t *out_bitstrings, int on_device);
int sv_alias_table(sv_state *s, uint64_t *out, uint64_t offset, uint64_t count, int on_device);
int sv_alias_release(sv_state *s);

/*
 * Expectation of a Pauli string (cached-state expectation values, §III-B):
 * qubit q carries I, X, Z or Y when (bit q of x_mask, bit q of z_mask) is (0,0),
 * (1,0), (0,1) or (1,1); *out = <psi|P|psi> / ||psi||^2 (real: P is Hermitian).
 * With x_mask = 0, <Z_mask> = sum_i |a_i|^2 (-1)^popcount(i & z_mask) / ||psi||^2;
 * otherwise P = i^k X^x_mask Z^z_mask (k = popcount(x_mask & z_mask)) is summed
 * over index pairs (i, i ^ x_mask).  One read of the state, products split
 * error-free and summed in compensated float32 per thread and double across
 * threads.  Masks with bits at or above n_qubits: SV_ERR_ARG; a zero norm:
 * SV_ERR_ARG.  Synchronises the state's stream.
 */
int sv_expect_pauli(sv_state *s, uint64_t x_mask, uint64_t z_mask, double *out);

/*
 * Mid-circuit measurement and reset (§III-B: a circuit runs up to its first
 * measurement or reset, then the state is copied and each shot continues on
 * its own copy).
 *
 * sv_measure_qubit measures `qubit` with the caller's uniform u in [0,1):
 * with m_b the FP64 mass of the amplitudes whose bit `qubit` is b, the outcome
 * is 0 when u * (m_0 + m_1) < m_0, else 1; amplitudes of the other outcome are
 * set to 0 and the rest scaled by 1/sqrt(m_outcome) (the state ends normalised).
 * *outcome receives the bit, *prob (optional) m_outcome / (m_0 + m_1).
 * Synchronises (the decision needs the masses on the host); the collapse is
 * queued on the state's stream.  SV_ERR_ARG for a bad qubit, u outside [0,1)
 * or a zero state.
 *
 * sv_reset_qubit: the same measurement, then X on `qubit` when the outcome was
 * 1, so the qubit ends in |0>.
 *
 * sv_clone creates a new library-owned state (its own 2^n * 8-byte buffer, on
 * `cuda_stream`) holding a copy of src as of all work queued on src's stream;
 * the copy is queued on the new state's stream, and work queued on src's stream
 * afterwards (including sv_destroy(src)) waits for it.  SV_ERR_OOM when the
 * buffer cannot be allocated.
 */
int sv_measure_qubit(sv_state *s, int qubit, double u, int *outcome, double *prob);
int sv_reset_qubit(sv_state *s, int qubit, double u, int *outcome);
int sv_clone(sv_state *src, void *cuda_stream, sv_state **out);

/*
 * Partitioned blocks (§II p-block simulation; §III-E: registers merge when
 * their qubits first interact, communication qubits leave once measured).
 *
 * sv_merge creates a new (n_a + n_b)-qubit state a (x) b: a's qubits become
 * qubits 0..n_a-1 and b's become n_a..n_a+n_b-1, out[i_b * 2^n_a + i_a] =
 * b[i_b] * a[i_a].  Queued on `cuda_stream` after all work queued on a's and
 * b's streams; work queued on a's or b's stream afterwards waits for it; a and
 * b are unchanged and stay valid.  SV_ERR_ARG past 36
 * qubits or across devices, SV_ERR_OOM without room for the result.
 *
 * sv_take_qubit removes `qubit` from a register in which it is in a basis
 * state |v> (e.g. right after sv_measure_qubit / sv_reset_qubit): the new
 * (n-1)-qubit state holds psi[j with bit v inserted at `qubit`], the remaining
 * qubits renumbered downwards.  *value receives v.  The masses of both halves
 * are computed first (synchronises); if the smaller one exceeds tol times the
 * total (tol in [0, 0.5)) the qubit is entangled or in superposition and
 * SV_ERR_ARG is returned.  s is unchanged.
 */
int sv_merge(sv_state *a, sv_state *b, void *cuda_stream, sv_state **out);
int sv_take_qubit(sv_state *s, int qubit, double tol, int *value, sv_state **out);

/*
 * Allocation-free <Z_mask>, for callers that cannot allocate device memory
 * when they need the value: e.g. a process that reserved all free GPU memory
 * for resident state vectors up front, or a latency-critical loop that cannot
 * take cudaMalloc's implicit device-wide synchronisation.  (The paper has no
 * counterpart: this is a deployment variant of sv_expect_pauli.)
 *
 * amplitudes: device pointer to 2^n_qubits complex64 (16-byte aligned), read
 * only.  out: device pointer to 2 doubles, written with out[0] = <Z_mask> =
 * sum_i |a_i|^2 (-1)^popcount(i & z_mask) / sum_i |a_i|^2 and out[1] =
 * sum_i |a_i|^2, the same sums and order as sv_expect_pauli.  Queued on
 * cuda_stream (a cudaStream_t; NULL = legacy default stream); asynchronous.
 *
 * Limit: n_qubits <= 28 -- the scratch is a fixed 1 MiB array compiled into the
 * library, which every GPU that loads it holds until the process exits; larger
 * states return SV_ERR_ARG.  No cudaMalloc, cudaFree or other allocating call
 * is made.  Every call looks up the array's device address on the current
 * device (cudaGetSymbolAddress, which allocates nothing); the first call on a
 * device may load the library's device code there, so make it before any
 * stream capture.  A state whose norm is zero or not finite gives out[0] = NaN
 * (sv_expect_pauli returns SV_ERR_ARG for it).  All calls on a device share the one array,
 * which keeps the last call's contents; every slot a call reads is written
 * earlier in that same call, so nothing needs clearing, but calls whose work
 * overlaps on the GPU (e.g. queued on different streams) race -- serialise them.
 */
int sv_expect_z_static(const void *amplitudes, int n_qubits, uint64_t z_mask, double *out,
                       void *cuda_stream);

/* ---- batched circuits -----------------------------------------------------
 *
 * Many independent small circuits in one persistent kernel, captured once in
 * a CUDA graph (the paper's batch execution, §IV-B, where per-circuit launch
 * and transfer overheads make GPU simulation lose on small circuits, §II).
 * Each CTA runs whole circuits: a state of <= 13 qubits stays in shared
 * memory for the whole circuit; larger states (<= 24 qubits) live in a device
 * arena owned by the batch.  Every circuit starts in |0...0> and is measured
 * `shots[i]` times with counter-based SplitMix64 uniforms from `seeds[i]`
 * (the same rule and draws as sv_sample).  Gates are fused into blocks of at
 * most k_max <= 3 qubits; tile_qubits (<= 13) tiles the arena states.
 */
typedef struct sv_batch sv_batch;

/* Plan every circuit (host), allocate the plan, arena and sample buffers, and
 * capture the launch in a CUDA graph.  irs[i] / n_gates[i] / n_qubits[i]
 * describe circuit i (host memory, read during the call); shots[i] may be 0.
 * zmasks (may be NULL): zmasks[i] != 0 also computes <Z_zmasks[i]> of circuit
 * i (sv_batch_expectation).  keep_states != 0 also copies every final state to
 * the arena (for sv_batch_amplitudes).  Work is queued on cuda_stream (NULL =
 * legacy default stream). */
int sv_batch_create(size_t n_circ, const sv_gate *const *irs, const size_t *n_gates, const int *n_qubits,
                    const uint64_t *shots, const uint64_t *seeds, const uint64_t *zmasks, const sv_opts *opts,
                    int keep_states, void *cuda_stream, sv_batch **out);
/* Replay the captured graph (all circuits, all shots); asynchronous. */
int sv_batch_launch(sv_batch *b);
int sv_batch_synchronize(sv_batch *b);
/* Samples of circuit i (caller's order) after the last launch: shots[i]
 * uint64 into out (device pointer if on_device, else host; host copies sync). */
int sv_batch_samples(sv_batch *b, size_t circuit, uint64_t *out, int on_device);
/* out2[0] = <Z_zmask> of circuit i, out2[1] = its norm (host; synchronous). */
int sv_batch_expectation(sv_batch *b, size_t circuit, double *out2);
/* Final state of circuit i (2^n complex64 into host memory; synchronous).
 * States of <= 13 qubits are available only with keep_states. */
int sv_batch_amplitudes(sv_batch *b, size_t circuit, void *out);
/* Planned HBM passes over arena states and their algorithmic bytes. */
int sv_batch_stats(const sv_batch *b, uint64_t *n_passes, uint64_t *hbm_bytes);
int sv_batch_destroy(sv_batch *b);
/* One-shot: create, launch, copy every circuit's samples to out[i] (host
 * pointers; NULL skips), destroy. */
int sv_batch_run(const sv_gate *const *irs, const size_t *n_gates, const int *n_qubits, size_t n_circ,
                 const uint64_t *shots, const uint64_t *seeds, uint64_t *const *out, const sv_opts *opts);
/* Autotuner: times every (k_max in 1..3, tile_qubits in 10..13) batch of the
 * given circuits (typically a sample of a larger batch) over `reps` graph
 * launches after one warm-up, and returns the fastest options in *best (and
 * its time per launch in *best_ms, may be NULL). */
int sv_batch_autotune(size_t n_circ, const sv_gate *const *irs, const size_t *n_gates, const int *n_qubits,
                      const uint64_t *shots, const uint64_t *seeds, int reps, sv_opts *best, double *best_ms);

/* ---- profiling ----------------------------------------------------------- */

/* Per-kernel-kind launch records.  When enabled, the library brackets every
 * launch with CUDA events on the state's stream. */
typedef struct sv_kernel_stat {
  char name[32];       /* kernel kind */
  uint64_t launches;
  double ms;           /* summed event time */
  double bytes;        /* summed algorithmic HBM bytes */
} sv_kernel_stat;

int sv_profile_enable(sv_state *s, int on);
/* Synchronises; writes up to cap records; *n_out = number of kinds. Resets. */
int sv_profile_read(sv_state *s, sv_kernel_stat *out, int cap, int *n_out);

/* ---- errors ---------------------------------------------------------------*/

/* Message of the last failure on this thread ("" if none). */
const char *sv_last_error(void);

/* Library version string. */
const char *sv_version(void);

/* Number of CUDA kernels this library has launched in this process so far
 * (all states, all devices); a memset is not counted. */
uint64_t sv_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* SVGB_SV_H */
