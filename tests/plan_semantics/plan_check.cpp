// Host-only check of the planner's fusion (fuse_pass): the fused ops of one pass
// (dense blocks, phase terms, SWAP relabeling) applied to a random state must
// equal the gates applied one by one, and the shape-only forms of fuse_pass and
// fuse_stages (no matrices) must give the same ops.  Built and run by
// tests/test_plan_semantics.py.
#include "sv_plan.cpp"
#include <cstdio>
#include <random>
// device-side helpers the planner links against; not used by fuse_pass
namespace svgb {
bool tc_pass_fits(uint32_t, uint32_t, uint32_t, uint32_t, uint32_t) { return false; }
void tc_b_image(int, const double *, uint8_t *) {}
bool reg_pass_fits(uint32_t, uint32_t, uint32_t, uint32_t, uint32_t) { return true; }
}
using namespace svgb;
static void apply_k(std::vector<cd> &psi, int n, int k, const int *q, const std::vector<cd> &M) {
  const int K = 1 << k;
  uint64_t gm = 0;
  for (int x = 0; x < k; x++) gm |= 1ull << q[x];
  for (uint64_t i = 0; i < (1ull << n); i++) {
    if (i & gm) continue;
    cd v[32], w[32];
    for (int j = 0; j < K; j++) {
      uint64_t o = i;
      for (int x = 0; x < k; x++) if (j >> x & 1) o |= 1ull << q[x];
      v[j] = psi[o];
    }
    for (int r = 0; r < K; r++) { cd a = 0; for (int j = 0; j < K; j++) a += M[r * K + j] * v[j]; w[r] = a; }
    for (int r = 0; r < K; r++) {
      uint64_t o = i;
      for (int x = 0; x < k; x++) if (r >> x & 1) o |= 1ull << q[x];
      psi[o] = w[r];
    }
  }
}
int main(int argc, char **argv) {
  int n, ng;
  if (scanf("%d %d", &n, &ng) != 2) return 1;
  std::vector<sv_gate> ir(ng);
  for (int i = 0; i < ng; i++) {
    sv_gate g{}; int kind, nq;
    if (scanf("%d %d", &kind, &nq) != 2) return 1;
    g.kind = uint8_t(kind); g.nq = uint8_t(nq);
    for (int x = 0; x < nq; x++) if (scanf("%d", &g.q[x]) != 1) return 1;
    if (scanf("%lf %lf %lf", &g.p[0], &g.p[1], &g.p[2]) != 3) return 1;
    ir[i] = g;
  }
  const bool pairs = argc > 1 ? atoi(argv[1]) : 1;
  const int kmax = argc > 2 ? atoi(argv[2]) : 2;
  std::vector<GateM> gates;
  std::string err;
  if (!convert_ir(n, ir.data(), ng, gates, err)) { printf("err %s\n", err.c_str()); return 1; }
  uint64_t Q = (uint64_t(1) << n) - 1;
  int lpos[64];
  for (int q = 0; q < 64; q++) lpos[q] = q < n ? q : -1;
  std::vector<uint32_t> acc;
  for (size_t i = 0; i < gates.size(); i++) acc.push_back(uint32_t(i));
  std::vector<HostOp> ops;
  int rho[64];
  for (int q = 0; q < 64; q++) rho[q] = q;
  fuse_pass(gates, acc, Q, lpos, kmax, pairs, ops, pairs ? rho : nullptr);
  // The planner compares candidate fusions as shapes (no matrices) and builds
  // only the kept one: a shape fusion must give the same ops, qubits in the
  // same order, and the same phase terms.  Likewise the stage former.
  {
    std::vector<HostOp> shp;
    int rho_s[64];
    for (int q = 0; q < 64; q++) rho_s[q] = q;
    fuse_pass(gates, acc, Q, lpos, kmax, pairs, shp, pairs ? rho_s : nullptr, true);
    bool same = shp.size() == ops.size();
    for (size_t i = 0; same && i < ops.size(); i++) {
      same = shp[i].type == ops[i].type && shp[i].blk.qs == ops[i].blk.qs && shp[i].blk.mask == ops[i].blk.mask &&
             shp[i].blk.M.empty() && shp[i].terms.size() == ops[i].terms.size();
      for (size_t t = 0; same && t < ops[i].terms.size(); t++)
        same = shp[i].terms[t].outer == ops[i].terms[t].outer && shp[i].terms[t].la == ops[i].terms[t].la &&
               shp[i].terms[t].lb == ops[i].terms[t].lb && shp[i].terms[t].turn == ops[i].terms[t].turn;
    }
    for (int q = 0; same && q < 64; q++) same = !pairs || rho_s[q] == rho[q];
    std::vector<HostOp> st_full, st_shape;
    const bool f1 = fuse_stages(gates, acc, 4, st_full), f2 = fuse_stages(gates, acc, 4, st_shape, true);
    same = same && f1 == f2 && st_full.size() == st_shape.size();
    for (size_t i = 0; same && i < st_full.size(); i++)
      same = st_full[i].blk.qs == st_shape[i].blk.qs && st_shape[i].blk.M.empty() &&
             int(st_full[i].blk.M.size()) == (1 << (2 * st_full[i].blk.k()));
    if (!same) {
      printf("shape fusion differs from the full fusion\n");
      return 3;
    }
  }
  std::mt19937_64 rng(7);
  std::normal_distribution<double> nd;
  std::vector<cd> a(1ull << n), b;
  for (auto &x : a) x = cd(nd(rng), nd(rng));
  b = a;
  for (auto &g : gates) apply_k(a, n, g.k, g.q, g.m);
  int nd_ = 0, np_ = 0;
  for (auto &op : ops) {
    if (op.type == OP_DENSE) { apply_k(b, n, op.blk.k(), op.blk.qs.data(), op.blk.M); nd_++; }
    else {
      np_++;
      for (uint64_t i = 0; i < (1ull << n); i++) {
        double ph = 0;
        for (auto &t : op.terms) {
          bool on = (t.la < 0 || (i >> t.la & 1)) && (t.lb < 0 || (i >> t.lb & 1));
          if (on) ph += 2.0 * M_PI * double(t.turn) / 4294967296.0;
        }
        b[i] *= std::polar(1.0, ph);
      }
    }
  }
  // relabeling: qubit q's data sits at position rho[q]
  std::vector<cd> c(b.size());
  for (uint64_t i = 0; i < (1ull << n); i++) {
    uint64_t j = 0;
    for (int q = 0; q < n; q++) if (i >> q & 1) j |= 1ull << rho[q];
    c[i] = b[j];
  }
  double e = 0;
  for (size_t i = 0; i < a.size(); i++) e = std::max(e, std::abs(a[i] - c[i]));
  printf("blocks %d phase %d maxerr %.3e\n", nd_, np_, e);
  // phase terms are 32-bit fractions of a turn: each is off by at most pi * 2^-32
  // rad, a few dozen terms on amplitudes of modulus < 8 stay far below 1e-6
  return e < 1e-6 ? 0 : 2;
}
