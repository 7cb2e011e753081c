/*
 * sv_oracle.c -- the correctness oracle for the state-vector hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this library.  The CUDA
 * path never calls it, and it shares no code with the CUDA path.
 *
 * What it computes is the plain definition of exact state-vector simulation
 * (§II: the full 2^n complex amplitude vector), written out in complex128:
 *
 *   psi_out = U_G ... U_2 U_1 psi_in,
 *
 * each U_g being gate g's 2^k x 2^k matrix acting on its k target qubits and
 * the identity on every other qubit.  Gates are applied one at a time in
 * program order -- no fusion, no blocking, no reordering.
 *
 * Conventions (the paper ingests Qiskit circuits and OpenQASM 2, §III-A, and
 * is otherwise silent; these are the readings adopted):
 *   - qubit q is bit q of the amplitude index (little-endian);
 *   - for a gate on targets (t_0 .. t_{k-1}), bit m of the matrix row/column
 *     index refers to qubit t_m (t_0 is the least significant matrix bit);
 *     so for cx(c, t), c = t_0 and t = t_1;
 *   - gate matrices follow the OpenQASM 2 definitions (u3, cx, cp, ...).
 *
 * Measurement (§III-B: sampling of end-of-circuit measurements from the final
 * state; expectation values from the cached state):
 *   - p_i = |psi_i|^2, CDF C_i = sum_{j<=i} p_j accumulated sequentially in
 *     double precision;
 *   - a draw with uniform u in [0,1) picks x = min{ i : C_i > u * C_{N-1} }
 *     (strict), clamped to the last index with p_i > 0 if rounding leaves no
 *     such i;
 *   - <Z_mask> = sum_i p_i (-1)^popcount(i & mask) / C_{N-1}.
 *
 * Mid-circuit measurement of one qubit (§III-B: execution up to a
 * measurement or reset, then per-shot continuation from a copy of the state):
 *   - m_b = sum of p_i over indices whose bit q equals b (sequential double);
 *   - with uniform u, the outcome is 0 when u * (m_0 + m_1) < m_0, else 1
 *     (the same strict rule as the draw above, over the two outcomes);
 *   - the state collapses: amplitudes with bit q != outcome become 0, the rest
 *     are multiplied by 1 / sqrt(m_outcome);
 *   - a reset is that measurement followed by X on q when the outcome is 1.
 *
 * Partitioned blocks (§II p-block simulation; §III-E: registers merge when
 * they first interact and communication qubits leave after measurement):
 *   - merging registers A (n_a qubits) and B (n_b qubits) gives A (x) B with A
 *     on the low qubits: out[i_b * 2^n_a + i_a] = b[i_b] * a[i_a];
 *   - a qubit q known to be in the basis state |v> (e.g. just measured) leaves
 *     the register: out[j] = psi[j with bit v inserted at position q].
 *
 * Alias sampling (§III-C: shots are drawn by alias sampling, O(1) work per
 * shot, after Walker 1974).  One bucket per basis state, capacity C = 2^31
 * units; bucket i keeps own_i units for outcome i and gives the rest to
 * alias_i:
 *   - weights are quantised: q_i = p_i * (N / W) with W = sum_i p_i taken
 *     with Neumaier's compensated summation (so that W, and with it every
 *     Q_i, is fixed by the amplitudes to within a few ulps whatever their
 *     number or order), Q_i = q_i * 2^31 rounded to the nearest integer;
 *     everything after that is exact integer arithmetic;
 *   - items with Q_i < C are light, the others heavy, each list in index
 *     order; the light items are walked in order, each taking its deficit
 *     C - Q_i from the current heavy item; a heavy item whose remainder drops
 *     below C becomes a light bucket of that remainder, filled from the next
 *     heavy item; the last heavy item, and any never reached, keep a full
 *     bucket (own = C, alias = itself);
 *   - a draw with uniform u in [0,1): x = u * N, i = floor(x), f = x - i; it
 *     is i when f * 2^31 < own_i, else alias_i.
 *
 * Parity pinning: see tests/test_oracle_pins.py (closed forms for GHZ and QFT,
 * an explicit DFT matrix, Kronecker-product brute force for n <= 8, textbook
 * gate identities, norm preservation, circuit * inverse = |0...0>, sampler and
 * expectation closed forms).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef double _Complex cplx;

/* Gate kinds of the oracle's own IR (independent of the CUDA library's enum). */
enum {
  ORC_U3 = 1, ORC_H, ORC_X, ORC_Y, ORC_Z, ORC_S, ORC_SDG, ORC_T, ORC_TDG,
  ORC_RX, ORC_RY, ORC_RZ, ORC_P, ORC_CX, ORC_CZ, ORC_CP, ORC_SWAP, ORC_UNITARY
};

typedef struct {
  int32_t kind;
  int32_t nq;
  int32_t q[5];
  int32_t _pad;
  double p[3];
  const cplx *mat; /* ORC_UNITARY only: 2^nq x 2^nq row-major */
} orc_gate;

void orc_set_threads(int t) {
#ifdef _OPENMP
  omp_set_num_threads(t > 0 ? t : 1);
#else
  (void)t;
#endif
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/*
 * Gate matrix, row-major 2^k x 2^k, from the OpenQASM 2 definitions:
 *   u3(θ,φ,λ) = [[cos(θ/2), -e^{iλ} sin(θ/2)], [e^{iφ} sin(θ/2), e^{i(φ+λ)} cos(θ/2)]]
 *   rx(θ) = u3(θ,-π/2,π/2), ry(θ) = u3(θ,0,0), rz(φ) = diag(e^{-iφ/2}, e^{iφ/2}),
 *   p(λ) = diag(1, e^{iλ}), h = u3(π/2,0,π), x, y, z, s, sdg, t, tdg standard,
 *   cx (control t_0, target t_1), cz, cp(λ) = diag(1,1,1,e^{iλ}), swap.
 * Returns the number of qubits k, or -1 for an unknown kind.
 */
int orc_gate_matrix(const orc_gate *g, cplx *m) {
  const double *p = g->p;
  const double r2 = 1.0 / sqrt(2.0);
  int k;
  switch (g->kind) {
  case ORC_UNITARY:
    k = g->nq;
    memcpy(m, g->mat, sizeof(cplx) * (size_t)(1u << k) * (size_t)(1u << k));
    return k;
  case ORC_U3: {
    double c = cos(p[0] / 2.0), s = sin(p[0] / 2.0);
    m[0] = c;
    m[1] = -cexp(I * p[2]) * s;
    m[2] = cexp(I * p[1]) * s;
    m[3] = cexp(I * (p[1] + p[2])) * c;
    return 1;
  }
  case ORC_H: m[0] = r2; m[1] = r2; m[2] = r2; m[3] = -r2; return 1;
  case ORC_X: m[0] = 0; m[1] = 1; m[2] = 1; m[3] = 0; return 1;
  case ORC_Y: m[0] = 0; m[1] = -I; m[2] = I; m[3] = 0; return 1;
  case ORC_Z: m[0] = 1; m[1] = 0; m[2] = 0; m[3] = -1; return 1;
  case ORC_S: m[0] = 1; m[1] = 0; m[2] = 0; m[3] = I; return 1;
  case ORC_SDG: m[0] = 1; m[1] = 0; m[2] = 0; m[3] = -I; return 1;
  case ORC_T: m[0] = 1; m[1] = 0; m[2] = 0; m[3] = cexp(I * M_PI / 4.0); return 1;
  case ORC_TDG: m[0] = 1; m[1] = 0; m[2] = 0; m[3] = cexp(-I * M_PI / 4.0); return 1;
  case ORC_RX: {
    double c = cos(p[0] / 2.0), s = sin(p[0] / 2.0);
    m[0] = c; m[1] = -I * s; m[2] = -I * s; m[3] = c;
    return 1;
  }
  case ORC_RY: {
    double c = cos(p[0] / 2.0), s = sin(p[0] / 2.0);
    m[0] = c; m[1] = -s; m[2] = s; m[3] = c;
    return 1;
  }
  case ORC_RZ:
    m[0] = cexp(-I * p[0] / 2.0); m[1] = 0; m[2] = 0; m[3] = cexp(I * p[0] / 2.0);
    return 1;
  case ORC_P: m[0] = 1; m[1] = 0; m[2] = 0; m[3] = cexp(I * p[0]); return 1;
  case ORC_CX:
  case ORC_CZ:
  case ORC_CP:
  case ORC_SWAP:
    for (int i = 0; i < 16; i++) m[i] = 0;
    if (g->kind == ORC_CX) {
      /* index bit 0 = control (t_0), bit 1 = target (t_1) */
      m[0 * 4 + 0] = 1; m[2 * 4 + 2] = 1; m[1 * 4 + 3] = 1; m[3 * 4 + 1] = 1;
    } else if (g->kind == ORC_SWAP) {
      m[0 * 4 + 0] = 1; m[1 * 4 + 2] = 1; m[2 * 4 + 1] = 1; m[3 * 4 + 3] = 1;
    } else {
      m[0] = 1; m[5] = 1; m[10] = 1;
      m[15] = (g->kind == ORC_CZ) ? -1.0 : cexp(I * p[0]);
    }
    return 2;
  default:
    return -1;
  }
}

/*
 * Apply a k-qubit matrix M (2^k x 2^k row-major) on targets t[0..k-1]:
 * for every index i with all target bits clear, gather v_j = psi[i | bits(j)]
 * (bit m of j placed at qubit t_m), then psi[i | bits(r)] = sum_j M[r][j] v_j.
 */
void orc_apply_matrix(cplx *psi, int n, int k, const int32_t *t, const cplx *M) {
  const uint64_t N = 1ull << n;
  const int K = 1 << k;
  uint64_t tmask = 0;
  for (int m = 0; m < k; m++) tmask |= 1ull << t[m];
  uint64_t off[32];
  for (int j = 0; j < K; j++) {
    uint64_t o = 0;
    for (int m = 0; m < k; m++)
      if ((j >> m) & 1) o |= 1ull << t[m];
    off[j] = o;
  }
#pragma omp parallel for schedule(static)
  for (int64_t ii = 0; ii < (int64_t)N; ii++) {
    uint64_t i = (uint64_t)ii;
    if (i & tmask) continue;
    cplx v[32], w[32];
    for (int j = 0; j < K; j++) v[j] = psi[i | off[j]];
    for (int r = 0; r < K; r++) {
      cplx acc = 0;
      for (int j = 0; j < K; j++) acc += M[r * K + j] * v[j];
      w[r] = acc;
    }
    for (int r = 0; r < K; r++) psi[i | off[r]] = w[r];
  }
}

/* Check the IR: kinds known, 1 <= nq <= 5, qubits in range and distinct. */
int orc_validate(int n, const orc_gate *g, uint64_t ngates) {
  for (uint64_t a = 0; a < ngates; a++) {
    cplx m[1024];
    if (g[a].kind == ORC_UNITARY && (g[a].nq < 1 || g[a].nq > 5 || !g[a].mat)) return -1;
    int k = orc_gate_matrix(&g[a], m);
    if (k < 0) return -1;
    for (int x = 0; x < k; x++) {
      if (g[a].q[x] < 0 || g[a].q[x] >= n) return -1;
      for (int y = 0; y < x; y++)
        if (g[a].q[x] == g[a].q[y]) return -1;
    }
    for (int x = 0; x < 3; x++)
      if (!isfinite(g[a].p[x])) return -1;
  }
  return 0;
}

/* Run a circuit gate by gate, in order, on psi (2^n complex128). */
int orc_run(cplx *psi, int n, const orc_gate *g, uint64_t ngates) {
  if (orc_validate(n, g, ngates)) return -1;
  cplx m[1024];
  for (uint64_t a = 0; a < ngates; a++) {
    int k = orc_gate_matrix(&g[a], m);
    orc_apply_matrix(psi, n, k, g[a].q, m);
  }
  return 0;
}

/* ||psi||^2 summed sequentially in double precision. */
double orc_norm2(const cplx *psi, uint64_t N) {
  double s = 0.0;
  for (uint64_t i = 0; i < N; i++) {
    double re = creal(psi[i]), im = cimag(psi[i]);
    s += re * re + im * im;
  }
  return s;
}

/* p_i = |psi_i|^2 and the sequential double-precision CDF C_i. */
void orc_cdf(const cplx *psi, uint64_t N, double *C) {
  double s = 0.0;
  for (uint64_t i = 0; i < N; i++) {
    double re = creal(psi[i]), im = cimag(psi[i]);
    s += re * re + im * im;
    C[i] = s;
  }
}

/*
 * Inverse-CDF sampling: shot s takes t = u_s * C_{N-1} and returns
 * x = min{ i : C_i > t } (binary search over the non-decreasing C).  If no
 * such i exists (t rounded up to the total), x is the last index with
 * p_i > 0.  boundary[s] = 1 when t lies within eps of C_x or of C_{x-1}
 * (C_{-1} = 0); returns the number of such boundary draws.
 */
uint64_t orc_sample(const double *C, uint64_t N, const double *u, uint64_t S, double eps,
                    uint64_t *out, uint8_t *boundary) {
  const double total = C[N - 1];
  uint64_t last = N - 1;
  while (last > 0 && C[last] <= C[last - 1]) last--;
  uint64_t nb = 0;
  for (uint64_t s = 0; s < S; s++) {
    double t = u[s] * total;
    uint64_t lo = 0, hi = N; /* first index in [lo, hi) with C > t */
    while (lo < hi) {
      uint64_t mid = lo + (hi - lo) / 2;
      if (C[mid] > t) hi = mid; else lo = mid + 1;
    }
    uint64_t x = (lo < N) ? lo : last;
    double below = x ? C[x - 1] : 0.0;
    int b = (fabs(t - C[x]) < eps) || (fabs(t - below) < eps);
    out[s] = x;
    if (boundary) boundary[s] = (uint8_t)b;
    nb += (uint64_t)b;
  }
  return nb;
}

/* <Z_mask> = sum_i p_i (-1)^popcount(i & mask) / sum_i p_i (sequential). */
double orc_expect_z(const cplx *psi, uint64_t N, uint64_t zmask) {
  double num = 0.0, den = 0.0;
  for (uint64_t i = 0; i < N; i++) {
    double re = creal(psi[i]), im = cimag(psi[i]);
    double p = re * re + im * im;
    num += (__builtin_popcountll(i & zmask) & 1) ? -p : p;
    den += p;
  }
  return num / den;
}

/* Expectation of a Pauli string (cached-state expectation values, §III-B):
 * qubit q carries I, X, Z or Y when (bit q of x_mask, bit q of z_mask) is
 * (0,0), (1,0), (0,1) or (1,1).  The definition written out: phi = P psi by
 * applying each qubit's 2x2 Pauli matrix (X = [[0,1],[1,0]], Y = [[0,-i],[i,0]],
 * Z = [[1,0],[0,-1]]) with orc_apply_matrix, then <P> = <psi|phi> / <psi|psi>,
 * both sums sequential in complex128.  *out_re, *out_im receive <P> (the
 * imaginary part is 0 up to rounding: P is Hermitian).  Returns 0, or -1 when
 * the copy cannot be allocated. */
int orc_expect_pauli(const cplx *psi, int n, uint64_t x_mask, uint64_t z_mask, double *out_re,
                     double *out_im) {
  const uint64_t N = 1ull << n;
  cplx *phi = (cplx *)malloc(N * sizeof(cplx));
  if (!phi) return -1;
  memcpy(phi, psi, N * sizeof(cplx));
  const cplx X[4] = {0, 1, 1, 0};
  const cplx Y[4] = {0, -I, I, 0};
  const cplx Z[4] = {1, 0, 0, -1};
  for (int q = 0; q < n; q++) {
    const int xb = (int)((x_mask >> q) & 1u), zb = (int)((z_mask >> q) & 1u);
    const int32_t t = q;
    if (xb && zb) orc_apply_matrix(phi, n, 1, &t, Y);
    else if (xb) orc_apply_matrix(phi, n, 1, &t, X);
    else if (zb) orc_apply_matrix(phi, n, 1, &t, Z);
  }
  cplx num = 0;
  double den = 0.0;
  for (uint64_t i = 0; i < N; i++) {
    num += conj(psi[i]) * phi[i];
    den += creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
  }
  free(phi);
  *out_re = creal(num) / den;
  *out_im = cimag(num) / den;
  return 0;
}

/* Mid-circuit measurement of qubit q with uniform u: collapses psi in place and
 * returns the outcome; *prob = m_outcome / (m_0 + m_1). */
int orc_measure(cplx *psi, uint64_t N, int q, double u, double *prob) {
  const uint64_t bit = (uint64_t)1 << q;
  double m0 = 0.0, m1 = 0.0;
  for (uint64_t i = 0; i < N; i++) {
    double re = creal(psi[i]), im = cimag(psi[i]);
    double p = re * re + im * im;
    if (i & bit) m1 += p; else m0 += p;
  }
  const int outcome = (u * (m0 + m1) < m0) ? 0 : 1;
  const double m = outcome ? m1 : m0;
  const double scale = 1.0 / sqrt(m);
  for (uint64_t i = 0; i < N; i++) {
    if (((i & bit) != 0) == outcome) psi[i] *= scale;
    else psi[i] = 0.0;
  }
  if (prob) *prob = m / (m0 + m1);
  return outcome;
}

/* Reset of qubit q: measure with u, then flip q when the outcome was 1. */
int orc_reset_qubit(cplx *psi, uint64_t N, int q, double u) {
  const int outcome = orc_measure(psi, N, q, u, NULL);
  if (outcome) {
    const uint64_t bit = (uint64_t)1 << q;
    for (uint64_t i = 0; i < N; i++)
      if (i & bit) {
        cplx t = psi[i];
        psi[i] = psi[i ^ bit];
        psi[i ^ bit] = t;
      }
  }
  return outcome;
}

/* Merge of two registers: out (2^(na+nb) entries) = a (x) b, a on the low qubits. */
void orc_kron(const cplx *a, int na, const cplx *b, int nb, cplx *out) {
  const uint64_t Na = (uint64_t)1 << na, Nb = (uint64_t)1 << nb;
  for (uint64_t ib = 0; ib < Nb; ib++)
    for (uint64_t ia = 0; ia < Na; ia++) out[ib * Na + ia] = b[ib] * a[ia];
}

/* Qubit q in the basis state |v> leaves the n-qubit register: out has 2^(n-1) entries. */
void orc_take_qubit(const cplx *psi, int n, int q, int v, cplx *out) {
  const uint64_t half = (uint64_t)1 << (n - 1);
  const uint64_t low = ((uint64_t)1 << q) - 1;
  for (uint64_t j = 0; j < half; j++) {
    const uint64_t i = ((j & ~low) << 1) | (j & low) | ((uint64_t)v << q);
    out[j] = psi[i];
  }
}

/*
 * Walker alias table of p_i = |psi_i|^2 (see the header): Q (quantised
 * weights), own (units kept by bucket i) and alias (its other outcome).
 * Returns 0, or -1 when the state has no weight.
 */
int orc_alias_build(const cplx *psi, uint64_t N, uint64_t *Q, uint32_t *own, uint32_t *alias) {
  const uint64_t C = (uint64_t)1 << 31;
  double W = 0.0, comp = 0.0; /* Neumaier: comp collects the rounding error of each addition */
  for (uint64_t i = 0; i < N; i++) {
    double re = creal(psi[i]), im = cimag(psi[i]);
    double p = re * re + im * im;
    double t = W + p;
    if (fabs(W) >= fabs(p)) comp += (W - t) + p;
    else comp += (p - t) + W;
    W = t;
  }
  W += comp;
  if (!(W > 0.0)) return -1;
  const double scale = (double)N / W;
  uint64_t *light = (uint64_t *)malloc(N * sizeof(uint64_t));
  uint64_t *heavy = (uint64_t *)malloc(N * sizeof(uint64_t));
  uint64_t nl = 0, nh = 0;
  for (uint64_t i = 0; i < N; i++) {
    double re = creal(psi[i]), im = cimag(psi[i]);
    double p = re * re + im * im;
    Q[i] = (uint64_t)nearbyint(p * scale * 2147483648.0);
    if (Q[i] < C) light[nl++] = i;
    else heavy[nh++] = i;
  }
  if (nh == 0) {
    free(light);
    free(heavy);
    return -1;
  }
  uint64_t j = 0;
  uint64_t r = Q[heavy[0]]; /* units the current heavy item still holds */
  for (uint64_t k = 0; k < nl; k++) {
    const uint64_t i = light[k];
    own[i] = (uint32_t)Q[i];
    alias[i] = (uint32_t)heavy[j];
    r -= C - Q[i];
    while (r < C && j + 1 < nh) {
      /* heavy item j is used up: its bucket keeps r units, the next heavy fills the rest */
      own[heavy[j]] = (uint32_t)r;
      alias[heavy[j]] = (uint32_t)heavy[j + 1];
      r = Q[heavy[j + 1]] - (C - r);
      j++;
    }
  }
  for (uint64_t m = j; m < nh; m++) {
    own[heavy[m]] = (uint32_t)C;
    alias[heavy[m]] = (uint32_t)heavy[m];
  }
  free(light);
  free(heavy);
  return 0;
}

/* Draws from an alias table: out[s] for uniform u[s] (see the header). */
void orc_alias_sample(const uint32_t *own, const uint32_t *alias, uint64_t N, const double *u,
                      uint64_t S, uint64_t *out) {
  for (uint64_t s = 0; s < S; s++) {
    const double x = u[s] * (double)N;
    uint64_t i = (uint64_t)x;
    if (i >= N) i = N - 1;
    const double f = x - (double)i;
    out[s] = (f * 2147483648.0 < (double)own[i]) ? i : alias[i];
  }
}
