// Host interpreter of packed plans (register-stage, tensor-core and shared-memory
// passes), for tests/test_plan_semantics.py.  It plans a circuit with the
// library's planner (build_plan), then executes every pass the way the register
// and tensor-core kernels read their records -- the load's chunk rows
// (RegPassParams.ko), stage 0's offsets (lo), each stage's thread bits (tb) and
// swizzled exchange offsets (xo), the dense ops on register positions (rmask,
// (re, re, -im, im) matrices) or the stage's product with its real-embedded
// matrix B (D[m][n] = sum_k A[m][k] B[n][k], A = a thread's 16 amplitudes as
// (re, im) pairs), the register phase ops (classes, D), and the store (oq, go)
// -- in complex double, and compares the result with the circuit's gates applied
// one by one.  With a chunk size it plans incrementally (PlanBuilder, as the
// library streams its plans) and runs the chunks in order.
// Shared-memory passes run the way k_pass reads theirs.  Exit status 0 when
// every amplitude agrees within 1e-5, 2 otherwise.
#include "sv_plan.cpp"

#include <cstdio>
#include <random>

// Device-side helpers the planner links against.  The stage image here holds
// B (K x K, K = 2^(R+1)) as float pairs (hi = float(B), lo = float(B - hi)),
// [hi K x K | lo K x K] row-major in n: the interpreter checks what the planner
// computes and packs (stages, their matrices, offsets), not the tensor cores'
// operand layout, which the GPU self-test of the stage product covers.
namespace svgb {
bool tc_pass_fits(uint32_t T, uint32_t c, uint32_t n_stages, uint32_t data_bytes, uint32_t R) {
  // the kernel's limits: R = 4 with 11 <= T <= 13, R = 5 with 12 <= T <= 13;
  // shared memory = load + exchange buffers (8 B an amplitude each), the
  // per-thread stage tables, the pass's records
  if ((R != 4 && R != 5) || T < R + 7 || T > R + (R == 4 ? 9 : 8) || T < c + R || c < 1 || n_stages < 1 ||
      n_stages > 64 || data_bytes > 160u * 1024u)
    return false;
  const size_t L = size_t(1) << T, NT = L >> R;
  size_t o = 16 * L + size_t(n_stages) * NT * 4;
  o = (o + 15) & ~size_t(15);
  return o + data_bytes + 1024 <= 232448;
}
void tc_b_image(int R, const double *B, uint8_t *img) {
  const int K = 2 << R;
  float *f = reinterpret_cast<float *>(img);
  for (int i = 0; i < K * K; i++) {
    f[i] = float(B[i]);
    f[K * K + i] = float(B[i] - double(f[i]));
  }
}
bool reg_pass_fits(uint32_t, uint32_t, uint32_t, uint32_t, uint32_t) { return true; }
}  // namespace svgb

using namespace svgb;
using cdd = std::complex<double>;

static void apply_gate(std::vector<cdd> &psi, int n, const GateM &g) {
  const int K = 1 << g.k;
  uint64_t gm = g.mask;
  for (uint64_t i = 0; i < (uint64_t(1) << n); i++) {
    if (i & gm) continue;
    cdd v[32], w[32];
    for (int j = 0; j < K; j++) {
      uint64_t o = i;
      for (int x = 0; x < g.k; x++)
        if (j >> x & 1) o |= uint64_t(1) << g.q[x];
      v[j] = psi[o];
    }
    for (int r = 0; r < K; r++) {
      cdd a = 0;
      for (int j = 0; j < K; j++) a += cdd(g.m[r * K + j]) * v[j];
      w[r] = a;
    }
    for (int r = 0; r < K; r++) {
      uint64_t o = i;
      for (int x = 0; x < g.k; x++)
        if (r >> x & 1) o |= uint64_t(1) << g.q[x];
      psi[o] = w[r];
    }
  }
}

static uint32_t dep_bits(uint32_t j, uint32_t mask) {  // bit i of j -> i-th set bit of mask
  uint32_t out = 0;
  int i = 0;
  for (int p = 0; p < 32; p++)
    if (mask >> p & 1u) {
      if (j >> i & 1u) out |= 1u << p;
      i++;
    }
  return out;
}

static cdd turn_exp(uint32_t turn) {
  const double a = 2.0 * M_PI * double(int32_t(turn)) / 4294967296.0;
  return cdd(std::cos(a), std::sin(a));
}

// Register-stage passes (KIND_REG) and tensor-core passes (KIND_TC: the same
// records, with each stage's dense blocks folded into one product).
static int exec_reg_pass(std::vector<cdd> &amp, const Plan &plan, size_t p) {
  const PlanPass &hp = plan.passes[p];
  if (hp.kind != KIND_REG && hp.kind != KIND_TC) return 3;
  const uint8_t *base_ptr = plan.bytes.data();
  const RegPassParams &prm = plan.rparams[p];
  const uint32_t T = hp.T, c = hp.c, R = hp.R, NR = 1u << R, NT = 1u << (T - R), ns = hp.n_stages;
  const StageRec *stages = reinterpret_cast<const StageRec *>(base_ptr + hp.stages_off);
  const OpRec *ops = reinterpret_cast<const OpRec *>(base_ptr + hp.ops_off);
  const uint32_t cs = c - 1u, cmask = (1u << cs) - 1u;
  std::vector<uint32_t> tt(size_t(ns) * NT);
  for (uint32_t s = 0; s < ns; s++)
    for (uint32_t tid = 0; tid < NT; tid++) {
      uint32_t LB = 0;
      for (uint32_t i = 0; i < T - R; i++)
        if ((tid >> i) & 1u) LB |= 1u << stages[s].tb[i];
      tt[s * NT + tid] = LB | (swz(LB) << 16);
    }
  const uint32_t L = 1u << T;
  std::vector<cdd> buf(L), xbuf(L);
  std::vector<std::vector<cdd>> v(NT, std::vector<cdd>(NR));
  // the outer-term slots (RegPhaseSlot) of the pass's phase ops
  const uint32_t n_w = hp.n_w;
  std::vector<uint32_t> wsum(n_w);
  if (n_w && (hp.w_off < hp.ops_off || hp.w_off + rphase_w_terms(n_w) > hp.ops_off + hp.data_bytes)) return 6;
  const RegPhaseSlot *wsl = reinterpret_cast<const RegPhaseSlot *>(base_ptr + hp.w_off);
  const RegPhaseOuter *wt = reinterpret_cast<const RegPhaseOuter *>(base_ptr + hp.w_off + rphase_w_terms(n_w));
  for (uint64_t tile = 0; tile < hp.n_tiles; tile++) {
    const uint64_t base = pdep_host(tile, hp.outer_mask);
    // this tile's sums of each slot's terms whose outer qubits are all 1
    for (uint32_t sl = 0; sl < n_w; sl++) {
      uint32_t a = 0;
      for (uint32_t i = wsl[sl].begin; i < wsl[sl].end; i++) {
        if (hp.w_off + rphase_w_terms(n_w) + (i + 1) * sizeof(RegPhaseOuter) > hp.ops_off + hp.data_bytes) return 6;
        if ((base & wt[i].outer_mask) == wt[i].outer_mask) a += wt[i].turn;
      }
      wsum[sl] = a;
    }
    // load: 16-byte chunk rows into the natural-order tile (tensor-core passes:
    // chunk q at position swzl(2q), stage-0 reads at swzl(LB0) ^ lo[j] / 8)
    const bool tcp = hp.kind == KIND_TC;
    for (uint32_t tid = 0; tid < NT; tid++) {
      const uint64_t t_cp = pdep_host(tid >> cs, hp.high_mask) + (uint64_t(tid & cmask) << 1);
      for (uint32_t k = 0; k < NR / 2; k++) {
        const uint64_t g = base + t_cp + prm.ko[k];
        const uint32_t q = tid + k * NT;
        const uint32_t pos = tcp ? swzl(2 * q) : 2 * q;
        if (g + 1 >= amp.size() || pos + 1 >= L) return 4;
        buf[pos] = amp[g];
        buf[pos + 1] = amp[g + 1];
      }
    }
    for (uint32_t tid = 0; tid < NT; tid++) {
      const uint32_t LB0 = tt[tid] & 0xffffu;
      for (uint32_t j = 0; j < NR; j++) {
        const uint32_t pos = tcp ? (swzl(LB0) ^ (prm.lo[j] / 8)) : (LB0 + prm.lo[j] / 8);
        if (pos >= L) return 4;
        v[tid][j] = buf[pos];
      }
    }
    for (uint32_t s = 0; s < ns; s++) {
      const StageRec &st = stages[s];
      if (s > 0) {
        const StageRec &pv = stages[s - 1];
        for (uint32_t tid = 0; tid < NT; tid++) {
          const uint32_t PBp = (tt[(s - 1) * NT + tid] >> 16) * 8u;
          for (uint32_t j = 0; j < NR; j++) {
            const uint32_t a = (pv.xo[j] ^ PBp) / 8u;
            if (a >= L) return 4;
            xbuf[a] = v[tid][j];
          }
        }
        for (uint32_t tid = 0; tid < NT; tid++) {
          const uint32_t PB = (tt[s * NT + tid] >> 16) * 8u;
          for (uint32_t j = 0; j < NR; j++) v[tid][j] = xbuf[(st.xo[j] ^ PB) / 8u];
        }
      }
      if (hp.kind == KIND_TC && (st.flags & 4u)) {  // the stage product, before its phase ops
        if (NR != 16 && NR != 32) return 3;
        const uint32_t K = 2 * NR;
        const float *bf = reinterpret_cast<const float *>(base_ptr + st.b_off);
        for (uint32_t tid = 0; tid < NT; tid++) {
          double A[64], D[64];
          for (uint32_t j = 0; j < NR; j++) {
            A[2 * j] = v[tid][j].real();
            A[2 * j + 1] = v[tid][j].imag();
          }
          for (uint32_t nn = 0; nn < K; nn++) {
            double acc = 0;
            for (uint32_t k = 0; k < K; k++) acc += A[k] * (double(bf[nn * K + k]) + double(bf[K * K + nn * K + k]));
            D[nn] = acc;
          }
          for (uint32_t j = 0; j < NR; j++) v[tid][j] = cdd(D[2 * j], D[2 * j + 1]);
        }
      }
      for (uint32_t o = st.op_begin; o < st.op_end; o++) {
        const OpRec &op = ops[o];
        const uint8_t *d = base_ptr + op.data_off;
        for (uint32_t tid = 0; tid < NT; tid++) {
          std::vector<cdd> &x = v[tid];
          if (op.type == OP_DENSE) {
            const uint32_t M = op.rmask, K = 1u << op.k;
            const float *m = reinterpret_cast<const float *>(d);  // (re, re, -im, im) per element
            for (uint32_t g = 0; g < NR; g++) {
              if (g & M) continue;
              cdd in[32], out[32];
              for (uint32_t j = 0; j < K; j++) in[j] = x[g | dep_bits(j, M)];
              for (uint32_t r = 0; r < K; r++) {
                cdd acc = 0;
                for (uint32_t j = 0; j < K; j++) {
                  const float *e = m + 4 * (r * K + j);
                  acc += cdd(e[0], e[3]) * in[j];
                }
                out[r] = acc;
              }
              for (uint32_t r = 0; r < K; r++) x[g | dep_bits(r, M)] = out[r];
            }
          } else {
            // per-thread tables of the terms on tile qubits, plus the tile's
            // sums of the terms on outer qubits (slot w_slot + 0: no thread
            // bit, + 1 + i: thread bit i, + 1 + ntb + r: register bit r)
            const RegPhaseHdr *h = reinterpret_cast<const RegPhaseHdr *>(d);
            const uint32_t *pre = reinterpret_cast<const uint32_t *>(d + sizeof(RegPhaseHdr));
            if (h->nt != NT || h->ntb != T - R) return 6;
            if (h->w_used && h->w_slot + 1 + h->ntb + R > n_w) return 6;
            uint32_t a[6] = {0, 0, 0, 0, 0, 0};
            for (uint32_t k = 0; k <= R; k++)
              if ((h->pre_mask >> k) & 1u) a[k] = pre[uint32_t(__builtin_popcount(h->pre_mask & ((1u << k) - 1u))) * NT + tid];
            const uint32_t *w = wsum.data() + h->w_slot;
            if (h->w_used & 1u) a[0] += w[0];
            if (h->w_used & 2u)
              for (uint32_t i = 0; i < h->ntb; i++)
                if ((tid >> i) & 1u) a[0] += w[1 + i];
            for (uint32_t r = 0; r < R; r++)
              if ((h->w_used >> (2 + r)) & 1u) a[1 + r] += w[1 + h->ntb + r];
            cdd e[6];
            for (uint32_t k = 0; k <= R; k++) e[k] = turn_exp(a[k]);
            for (uint32_t j = 0; j < NR; j++) {
              cdd f = e[0];
              for (uint32_t i = 0; i < R; i++)
                if (j >> i & 1u) f *= e[1 + i];
              if (h->has_d) f *= cdd(h->d[j].x, h->d[j].y);
              x[j] *= f;
            }
          }
        }
      }
    }
    // store: local bit x of the last stage's thread part goes to qubit oq[x]
    for (uint32_t tid = 0; tid < NT; tid++) {
      const uint32_t LB = tt[(ns - 1) * NT + tid] & 0xffffu;
      uint64_t t_st = 0;
      for (uint32_t x = 0; x < T; x++)
        if ((LB >> x) & 1u) t_st |= uint64_t(1) << prm.oq[x];
      for (uint32_t j = 0; j < NR; j++) {
        const uint64_t g = base + t_st + prm.go[j];
        if (g >= amp.size()) return 4;
        amp[g] = v[tid][j];
      }
    }
  }
  return 0;
}

// KIND_SMEM passes (k_pass): the tile in natural order (local index l <-> HBM
// base + segoff(l >> c) + (l & low)), each op one sweep over it -- dense blocks
// on local bits lb with float2 (re, im) matrices, phase ops as per-tile sums of
// single-local-bit terms -- then stored back the same way.
static int exec_smem_pass(std::vector<cdd> &amp, const Plan &plan, size_t p) {
  const PlanPass &hp = plan.passes[p];
  const uint8_t *base_ptr = plan.bytes.data();
  const uint32_t T = hp.T, c = hp.c, L = 1u << T;
  const OpRec *ops = reinterpret_cast<const OpRec *>(base_ptr + hp.ops_off);
  std::vector<cdd> tile(L);
  for (uint64_t tid = 0; tid < hp.n_tiles; tid++) {
    const uint64_t base = pdep_host(tid, hp.outer_mask);
    auto gaddr = [&](uint32_t l) { return base + pdep_host(l >> c, hp.high_mask) + (l & ((1u << c) - 1u)); };
    for (uint32_t l = 0; l < L; l++) {
      if (gaddr(l) >= amp.size()) return 4;
      tile[l] = amp[gaddr(l)];
    }
    for (uint32_t o = 0; o < hp.n_ops; o++) {
      const OpRec &op = ops[o];
      if (op.type == OP_DENSE) {
        const float *m = reinterpret_cast<const float *>(base_ptr + op.data_off);  // (re, im) per element
        const uint32_t K = 1u << op.k;
        uint32_t gm = 0;
        for (uint32_t x = 0; x < op.k; x++) gm |= 1u << op.lb[x];
        for (uint32_t b = 0; b < L; b++) {
          if (b & gm) continue;
          cdd in[32], out[32];
          auto at = [&](uint32_t j) {
            uint32_t off = 0;
            for (uint32_t x = 0; x < op.k; x++)
              if (j >> x & 1u) off |= 1u << op.lb[x];
            return b | off;
          };
          for (uint32_t j = 0; j < K; j++) in[j] = tile[at(j)];
          for (uint32_t r = 0; r < K; r++) {
            cdd a = 0;
            for (uint32_t j = 0; j < K; j++) a += cdd(m[2 * (r * K + j)], m[2 * (r * K + j) + 1]) * in[j];
            out[r] = a;
          }
          for (uint32_t r = 0; r < K; r++) tile[at(r)] = out[r];
        }
      } else if (op.type == OP_PHASE) {
        const PhaseTerm *t = reinterpret_cast<const PhaseTerm *>(base_ptr + op.data_off);
        uint32_t acc[33] = {0};
        for (uint32_t i = 0; i < op.count; i++)
          if ((base & t[i].outer_mask) == t[i].outer_mask) acc[t[i].la + 1] += t[i].turn;
        for (uint32_t l = 0; l < L; l++) {
          uint32_t turn = acc[0];
          for (uint32_t j = 0; j < T; j++)
            if (l >> j & 1u) turn += acc[1 + j];
          tile[l] *= turn_exp(turn);
        }
      } else {
        return 5;
      }
    }
    for (uint32_t l = 0; l < L; l++) amp[gaddr(l)] = tile[l];
  }
  return 0;
}

int main(int argc, char **argv) {
  int n, ng;
  if (scanf("%d %d", &n, &ng) != 2) return 1;
  std::vector<sv_gate> ir(static_cast<size_t>(ng));
  std::vector<std::vector<double>> mats;  // UNITARY gates: the matrices after their parameters
  mats.reserve(static_cast<size_t>(ng));
  for (int i = 0; i < ng; i++) {
    sv_gate g{};
    int kind, nq;
    if (scanf("%d %d", &kind, &nq) != 2) return 1;
    g.kind = uint8_t(kind);
    g.nq = uint8_t(nq);
    for (int x = 0; x < nq; x++)
      if (scanf("%d", &g.q[x]) != 1) return 1;
    if (scanf("%lf %lf %lf", &g.p[0], &g.p[1], &g.p[2]) != 3) return 1;
    if (kind == SV_GATE_UNITARY) {
      mats.emplace_back(size_t(2) << (2 * nq));
      for (double &x : mats.back())
        if (scanf("%lf", &x) != 1) return 1;
      g.mat = mats.back().data();
    }
    ir[size_t(i)] = g;
  }
  sv_opts o{};
  o.k_max = argc > 1 ? atoi(argv[1]) : 2;
  o.tile_qubits = argc > 2 ? atoi(argv[2]) : 12;
  o.low_qubits = argc > 3 ? atoi(argv[3]) : 5;
  o.kernel_variant = argc > 4 ? atoi(argv[4]) : 0;
  // chunk > 0: plan incrementally, `chunk` passes at a time (as sv_apply_circuit
  // streams its plan), and run the chunks' passes in order
  const int chunk = argc > 5 ? atoi(argv[5]) : 0;
  o.precision = argc > 6 ? atoi(argv[6]) : 0;  // 1: tensor-core passes
  std::vector<Plan> plans;
  std::string err;
  if (chunk <= 0) {
    plans.emplace_back();
    if (!build_plan(n, ir.data(), size_t(ng), &o, plans.back(), err)) {
      printf("plan error: %s\n", err.c_str());
      return 1;
    }
  } else {
    PlanBuilder pb;
    if (!pb.init(n, ir.data(), size_t(ng), &o, err)) {
      printf("plan error: %s\n", err.c_str());
      return 1;
    }
    while (!pb.done()) {
      plans.emplace_back();
      if (!pb.next(plans.back(), size_t(chunk), err)) {
        printf("plan error: %s\n", err.c_str());
        return 1;
      }
    }
  }
  std::vector<GateM> gates;
  if (!convert_ir(n, ir.data(), size_t(ng), gates, err)) return 1;
  std::mt19937_64 rng(11);
  std::normal_distribution<double> nd;
  std::vector<cdd> a(size_t(1) << n), b;
  double nrm = 0;
  for (auto &x : a) {
    x = cdd(nd(rng), nd(rng));
    nrm += std::norm(x);
  }
  for (auto &x : a) x /= std::sqrt(nrm);
  b = a;
  for (auto &g : gates) apply_gate(a, n, g);
  size_t total = 0, n_tc = 0;
  for (const Plan &plan : plans)
    for (size_t p = 0; p < plan.passes.size(); p++, total++) {
      n_tc += plan.passes[p].kind == KIND_TC;
      const int rc = plan.passes[p].kind == KIND_SMEM ? exec_smem_pass(b, plan, p) : exec_reg_pass(b, plan, p);
      if (rc) {
        printf("pass %zu: %s\n", total, rc == 3 ? "unsupported pass" : rc == 5 ? "unknown op" : rc == 6 ? "bad phase record" : "index out of range");
        return rc;
      }
    }
  double e = 0;
  for (size_t i = 0; i < a.size(); i++) e = std::max(e, std::abs(a[i] - b[i]));
  printf("plans %zu passes %zu tensor-core %zu maxerr %.3e kinds:", plans.size(), total, n_tc, e);
  for (const Plan &plan : plans)
    for (const PlanPass &hp : plan.passes) printf(" %u", hp.kind);
  printf("\n");
  return e <= 1e-5 ? 0 : 2;
}
