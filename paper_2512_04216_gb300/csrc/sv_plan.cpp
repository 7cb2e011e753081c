// sv_plan.cpp -- host side of sv_apply_circuit: IR validation, gate matrices,
// pass planning and gate fusion.
//
// The method applies a circuit's gates one after another to the 2^n amplitude
// vector (§II, exact state-vector simulation).  Here the gate list is
// re-grouped, without changing the product it computes:
//
//  1. Pass planning.  Scan the unapplied gates in program order and accept a
//     gate into the current pass when (a) no earlier unaccepted gate shares a
//     qubit with it, and (b) its qubits fit the pass's tile set Q (at most T
//     qubits, always including the c lowest).  Diagonal gates need not fit Q:
//     their effect on a tile depends on outer qubits only through a per-tile
//     constant.  A rejected gate blocks its qubits for the rest of the scan, so
//     every accepted gate commutes with every rejected gate before it.  Two
//     choices of Q are tried per pass and the one accepting more non-diagonal
//     gates is kept: growing Q in scan order (first come, first served), and
//     growing Q one qubit or one two-qubit gate at a time by the most gates a
//     scan of the next unapplied gates then accepts per added qubit.
//  2. Fusion.  Within a pass, gates are merged into dense blocks of at most
//     k_max qubits (open blocks on disjoint qubit sets; a gate merges the open
//     blocks it touches when the union fits, else those blocks are emitted and
//     the gate opens a new one).  Block matrices are built in complex128 and
//     stored as complex64.  Diagonal gates with at most one tile qubit become
//     phase terms instead; in passes that run on register stages, so do
//     diagonal gates on two tile qubits (a controlled phase between two tile
//     qubits costs one term of a phase op instead of a 4x4 block), unless an
//     open block already holds their qubits or can take them while no phase op
//     is being collected.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/sv.h"
#include "sv_internal.h"
#include "sv_plan.h"
#include "sv_tc.h"

namespace svgb {

using cd = std::complex<double>;

static inline int popc(uint64_t x) { return __builtin_popcountll(x); }
static inline int ctz(uint64_t x) { return __builtin_ctzll(x); }

// ---------------------------------------------------------------------------
// gate matrices (OpenQASM 2 definitions, see include/sv.h)
// ---------------------------------------------------------------------------

static bool gate_matrix(const sv_gate &g, GateM &out, std::string &err) {
  const double *p = g.p;
  const cd I(0.0, 1.0);
  out.diag = false;
  auto one = [&](cd a, cd b, cd c, cd d) {
    out.k = 1;
    out.m = {a, b, c, d};
  };
  switch (g.kind) {
    case SV_GATE_U3: {
      double ct = std::cos(0.5 * p[0]), st = std::sin(0.5 * p[0]);
      one(ct, -std::exp(I * p[2]) * st, std::exp(I * p[1]) * st, std::exp(I * (p[1] + p[2])) * ct);
      break;
    }
    case SV_GATE_H: {
      double r = std::sqrt(0.5);
      one(r, r, r, -r);
      break;
    }
    case SV_GATE_X: one(0.0, 1.0, 1.0, 0.0); break;
    case SV_GATE_Y: one(0.0, -I, I, 0.0); break;
    case SV_GATE_Z: one(1.0, 0.0, 0.0, -1.0); out.diag = true; break;
    case SV_GATE_S: one(1.0, 0.0, 0.0, I); out.diag = true; break;
    case SV_GATE_SDG: one(1.0, 0.0, 0.0, -I); out.diag = true; break;
    case SV_GATE_T: one(1.0, 0.0, 0.0, std::polar(1.0, M_PI / 4)); out.diag = true; break;
    case SV_GATE_TDG: one(1.0, 0.0, 0.0, std::polar(1.0, -M_PI / 4)); out.diag = true; break;
    case SV_GATE_RX: {
      double ct = std::cos(0.5 * p[0]), st = std::sin(0.5 * p[0]);
      one(ct, -I * st, -I * st, ct);
      break;
    }
    case SV_GATE_RY: {
      double ct = std::cos(0.5 * p[0]), st = std::sin(0.5 * p[0]);
      one(ct, -st, st, ct);
      break;
    }
    case SV_GATE_RZ:
      one(std::polar(1.0, -0.5 * p[0]), 0.0, 0.0, std::polar(1.0, 0.5 * p[0]));
      out.diag = true;
      break;
    case SV_GATE_P: one(1.0, 0.0, 0.0, std::polar(1.0, p[0])); out.diag = true; break;
    case SV_GATE_CX:
    case SV_GATE_CZ:
    case SV_GATE_CP:
    case SV_GATE_SWAP: {
      out.k = 2;
      out.m.assign(16, 0.0);
      auto at = [&](int r, int c) -> cd & { return out.m[r * 4 + c]; };
      if (g.kind == SV_GATE_CX) {
        // index bit 0 = control q[0], bit 1 = target q[1]
        at(0, 0) = 1.0; at(2, 2) = 1.0; at(1, 3) = 1.0; at(3, 1) = 1.0;
      } else if (g.kind == SV_GATE_SWAP) {
        at(0, 0) = 1.0; at(1, 2) = 1.0; at(2, 1) = 1.0; at(3, 3) = 1.0;
        out.swap = true;
      } else {
        at(0, 0) = 1.0; at(1, 1) = 1.0; at(2, 2) = 1.0;
        at(3, 3) = (g.kind == SV_GATE_CZ) ? cd(-1.0) : std::polar(1.0, p[0]);
        out.diag = true;
      }
      break;
    }
    case SV_GATE_UNITARY: {
      if (g.nq < 1 || g.nq > 5 || g.mat == nullptr) {
        err = "UNITARY gate needs 1 <= nq <= 5 and a matrix";
        return false;
      }
      out.k = g.nq;
      size_t K = size_t(1) << g.nq;
      out.m.resize(K * K);
      for (size_t i = 0; i < K * K; i++) {
        out.m[i] = cd(g.mat[2 * i], g.mat[2 * i + 1]);
        if (!std::isfinite(g.mat[2 * i]) || !std::isfinite(g.mat[2 * i + 1])) {
          err = "UNITARY matrix has a non-finite entry";
          return false;
        }
      }
      // max |(U^dagger U - I)_ij|: sv_apply_circuit restores the norm after a
      // tensor-core apply only when every gate is unitary
      double dev = 0.0;
      for (size_t a = 0; a < K; a++)
        for (size_t b = 0; b < K; b++) {
          cd x = (a == b) ? cd(-1.0) : cd(0.0);
          for (size_t r = 0; r < K; r++) x += std::conj(out.m[r * K + a]) * out.m[r * K + b];
          dev = std::max(dev, std::abs(x));
        }
      out.unitary = dev <= 1e-6;
      break;
    }
    default:
      err = "unknown gate kind " + std::to_string(int(g.kind));
      return false;
  }
  if (g.kind != SV_GATE_UNITARY && g.nq != out.k) {
    err = "gate kind " + std::to_string(int(g.kind)) + " takes " + std::to_string(out.k) +
          " qubit(s), nq = " + std::to_string(int(g.nq));
    return false;
  }
  for (int x = 0; x < out.k; x++) out.q[x] = g.q[x];
  return true;
}

bool convert_ir(int n, const sv_gate *ir, size_t ng, std::vector<GateM> &gates, std::string &err) {
  gates.resize(ng);
  for (size_t a = 0; a < ng; a++) {
    const sv_gate &g = ir[a];
    if (g.reserved != 0) {
      err = "gate " + std::to_string(a) + ": reserved field must be 0";
      return false;
    }
    for (int x = 0; x < 3; x++)
      if (!std::isfinite(g.p[x])) {
        err = "gate " + std::to_string(a) + ": non-finite parameter";
        return false;
      }
    if (!gate_matrix(g, gates[a], err)) {
      err = "gate " + std::to_string(a) + ": " + err;
      return false;
    }
    uint64_t mask = 0;
    for (int x = 0; x < gates[a].k; x++) {
      int q = gates[a].q[x];
      if (q < 0 || q >= n) {
        err = "gate " + std::to_string(a) + ": qubit " + std::to_string(q) + " out of range [0," +
              std::to_string(n) + ")";
        return false;
      }
      if (mask >> q & 1) {
        err = "gate " + std::to_string(a) + ": repeated qubit " + std::to_string(q);
        return false;
      }
      mask |= uint64_t(1) << q;
    }
    gates[a].mask = mask;
  }
  return true;
}

// ---------------------------------------------------------------------------
// fusion helpers
// ---------------------------------------------------------------------------

// A fused block.  A block without a matrix (M empty) is a shape only: the
// planner fuses the candidate forms of a pass as shapes (qubits and order, all
// that its choices read) and multiplies out the matrices of the form it keeps.
struct Block {
  uint64_t mask = 0;
  std::vector<int> qs;   // matrix bit m <-> physical qubit qs[m]
  std::vector<cd> M;     // 2^k x 2^k row-major (empty: a shape only)
  int k() const { return int(qs.size()); }
};

// M <- G (on block bits pos[0..kg-1]) * M, column by column (nothing for a shape).
static void apply_to_block(Block &b, const GateM &g) {
  if (b.M.empty()) return;
  const int k = b.k();
  const int K = 1 << k, KG = 1 << g.k;
  int pos[5];
  for (int x = 0; x < g.k; x++) {
    auto it = std::find(b.qs.begin(), b.qs.end(), g.q[x]);
    pos[x] = int(it - b.qs.begin());
  }
  int gmask = 0;
  for (int x = 0; x < g.k; x++) gmask |= 1 << pos[x];
  int off[32];
  for (int j = 0; j < KG; j++) {
    int o = 0;
    for (int x = 0; x < g.k; x++)
      if (j >> x & 1) o |= 1 << pos[x];
    off[j] = o;
  }
  cd v[32], w[32];
  for (int col = 0; col < K; col++) {
    for (int r0 = 0; r0 < K; r0++) {
      if (r0 & gmask) continue;
      for (int j = 0; j < KG; j++) v[j] = b.M[(r0 | off[j]) * K + col];
      for (int r = 0; r < KG; r++) {
        cd acc = 0.0;
        for (int j = 0; j < KG; j++) acc += g.m[r * KG + j] * v[j];
        w[r] = acc;
      }
      for (int r = 0; r < KG; r++) b.M[(r0 | off[r]) * K + col] = w[r];
    }
  }
}

// Tensor product of disjoint blocks: qs = a.qs ++ b.qs (a on the low matrix bits);
// a shape if either is one.
static Block kron_blocks(const Block &a, const Block &b) {
  Block c;
  c.mask = a.mask | b.mask;
  c.qs = a.qs;
  c.qs.insert(c.qs.end(), b.qs.begin(), b.qs.end());
  if (a.M.empty() || b.M.empty()) return c;
  const int KA = 1 << a.k(), KB = 1 << b.k(), K = KA * KB;
  c.M.assign(size_t(K) * K, 0.0);
  for (int rb = 0; rb < KB; rb++)
    for (int ra = 0; ra < KA; ra++)
      for (int jb = 0; jb < KB; jb++)
        for (int ja = 0; ja < KA; ja++)
          c.M[(rb * KA + ra) * K + (jb * KA + ja)] = a.M[ra * KA + ja] * b.M[rb * KB + jb];
  return c;
}

static Block identity_block(bool shape = false) {
  Block b;
  if (!shape) b.M = {cd(1.0)};
  return b;
}

// The one-qubit identity block on qubit q (a shape when `shape`).
static Block qubit_block(int q, bool shape) {
  Block one;
  one.mask = uint64_t(1) << q;
  one.qs = {q};
  if (!shape) one.M = {cd(1.0), cd(0.0), cd(0.0), cd(1.0)};
  return one;
}

static uint32_t to_turn(double phi) {
  double f = phi / (2.0 * M_PI);
  f -= std::floor(f);
  double s = std::nearbyint(f * 4294967296.0);
  return uint32_t(uint64_t(s) & 0xffffffffu);
}

struct HostTerm {
  uint64_t outer;  // outer qubits required to be 1
  int la;          // local bit required to be 1 (-1 none)
  int lb;          // second local bit required to be 1 (-1 none; la < lb)
  uint32_t turn;
};

struct HostOp {
  uint8_t type;
  Block blk;                   // DENSE
  std::vector<HostTerm> terms; // PHASE
};

// Decompose a diagonal 1- or 2-qubit gate into phase terms (constant, per-qubit,
// pair) and append them.  lpos[q] = local bit of q or -1.
static void diag_terms(const GateM &g, const int *lpos, std::vector<HostTerm> &out) {
  double ph[4];
  const int K = 1 << g.k;
  for (int j = 0; j < K; j++) ph[j] = std::arg(g.m[j * K + j]);
  // coefficient of the product of the index bits in subset S (Mobius inversion)
  for (int S = 0; S < K; S++) {
    double a = 0.0;
    for (int T = 0; T < K; T++)
      if ((T & S) == T) a += ((popc(uint64_t(S ^ T)) & 1) ? -1.0 : 1.0) * ph[T];
    uint32_t turn = to_turn(a);
    if (turn == 0) continue;
    HostTerm t{0, -1, -1, turn};
    for (int x = 0; x < g.k; x++)
      if (S >> x & 1) {
        const int q = g.q[x];
        if (lpos[q] < 0) t.outer |= uint64_t(1) << q;
        else if (t.la < 0) t.la = lpos[q];
        else t.lb = lpos[q];
      }
    if (t.lb >= 0 && t.lb < t.la) std::swap(t.la, t.lb);
    out.push_back(t);
  }
}

static void merge_terms(std::vector<HostTerm> &terms) {
  std::sort(terms.begin(), terms.end(), [](const HostTerm &a, const HostTerm &b) {
    if (a.la != b.la) return a.la < b.la;
    if (a.lb != b.lb) return a.lb < b.lb;
    return a.outer < b.outer;
  });
  std::vector<HostTerm> out;
  for (auto &t : terms) {
    if (!out.empty() && out.back().la == t.la && out.back().lb == t.lb && out.back().outer == t.outer)
      out.back().turn += t.turn;
    else
      out.push_back(t);
  }
  out.erase(std::remove_if(out.begin(), out.end(), [](const HostTerm &t) { return t.turn == 0; }),
            out.end());
  terms.swap(out);
}

// ---------------------------------------------------------------------------
// planning
// ---------------------------------------------------------------------------

// With `rho` (relabeling), a SWAP of two tile qubits emits nothing: rho[q] is
// the qubit whose loaded position now holds qubit q's data, and later gates act
// on those positions; the caller stores qubit q's data from local bit
// lpos[rho[q]].  Without it, SWAPs are ordinary 4x4 blocks.
static void fuse_pass(const std::vector<GateM> &gates, const std::vector<uint32_t> &acc,
                      uint64_t Q, const int *lpos, int kmax, bool pairs, std::vector<HostOp> &ops,
                      int *rho = nullptr, bool shape = false) {
  std::vector<Block> open;
  std::vector<HostTerm> pending;
  uint64_t pending_local = 0;

  auto emit_block = [&](Block &&b) {
    HostOp op;
    op.type = OP_DENSE;
    op.blk = std::move(b);
    ops.push_back(std::move(op));
  };
  auto close_touching = [&](uint64_t m) {
    for (size_t i = 0; i < open.size();) {
      if (open[i].mask & m) {
        emit_block(std::move(open[i]));
        open.erase(open.begin() + i);
      } else {
        i++;
      }
    }
  };
  auto flush_phase = [&]() {
    if (pending.empty()) {
      pending_local = 0;
      return;
    }
    // register passes leave blocks open past the diagonal gates they queue:
    // the blocks holding the phase's qubits come first
    if (pairs) close_touching(pending_local);
    merge_terms(pending);
    if (!pending.empty()) {
      HostOp op;
      op.type = OP_PHASE;
      op.terms.swap(pending);
      ops.push_back(std::move(op));
    }
    pending.clear();
    pending_local = 0;
  };

  GateM renamed;
  for (uint32_t gi : acc) {
    const GateM *gp = &gates[gi];
    if (rho) {
      if (gp->swap) {
        std::swap(rho[gp->q[0]], rho[gp->q[1]]);
        continue;
      }
      bool moved = false;
      for (int x = 0; x < gp->k; x++) moved |= rho[gp->q[x]] != gp->q[x];
      if (moved) {
        renamed = *gp;
        renamed.mask = 0;
        for (int x = 0; x < gp->k; x++) {
          renamed.q[x] = rho[gp->q[x]];
          renamed.mask |= uint64_t(1) << renamed.q[x];
        }
        gp = &renamed;
      }
    }
    const GateM &g = *gp;
    const uint64_t local = g.mask & Q;
    const bool outer = (g.mask & ~Q) != 0;
    bool to_phase = false;
    if (g.diag && popc(local) <= (pairs ? 2 : 1)) {
      to_phase = true;
      if (!outer) {
        // a local diagonal gate: absorb it into an open block that holds its
        // qubits; with no phase op being collected, also into open blocks that
        // can take it within k_max (a new phase op costs more than a wider
        // block) -- in register passes even when that only adds its other
        // qubit to a block (e.g. a controlled phase next to a Hadamard)
        uint64_t U = local;
        for (auto &b : open)
          if (b.mask & local) U |= b.mask;
        bool inside = false;
        for (auto &b : open)
          if ((b.mask & local) == local) inside = true;
        const bool grows = pairs ? (U != local || std::any_of(open.begin(), open.end(), [&](const Block &b) {
                                     return (b.mask & local) != 0;
                                   }))
                                 : (U & ~local) != 0;
        if (inside || (pending.empty() && grows && popc(U) <= kmax)) to_phase = false;
      }
    }
    if (to_phase) {
      // register passes keep the touching blocks open (a later gate may still
      // join them; the flush emits them before the phase op)
      if (!pairs) close_touching(local);
      diag_terms(g, lpos, pending);
      pending_local |= local;
      continue;
    }
    if (pending_local & g.mask) flush_phase();
    uint64_t U = g.mask;
    for (auto &b : open)
      if (b.mask & g.mask) U |= b.mask;
    Block nb;
    if (popc(U) <= kmax) {
      nb = identity_block(shape);
      for (size_t i = 0; i < open.size();) {
        if (open[i].mask & g.mask) {
          nb = kron_blocks(nb, open[i]);
          open.erase(open.begin() + i);
        } else {
          i++;
        }
      }
    } else {
      close_touching(g.mask);
      nb = identity_block(shape);
    }
    // append the gate's new qubits, then multiply the gate in
    for (int x = 0; x < g.k; x++) {
      if (!(nb.mask >> g.q[x] & 1)) nb = kron_blocks(nb, qubit_block(g.q[x], shape));
    }
    apply_to_block(nb, g);
    open.push_back(std::move(nb));
  }
  for (auto &b : open) emit_block(std::move(b));
  open.clear();
  flush_phase();
}

// Tensor-core passes whose gates are all non-diagonal and at most kmax wide:
// every stage is one product over at most kmax qubits, so the ops are built
// stage by stage.  A stage's qubit set S starts as the first remaining gate's
// qubits and grows one qubit at a time, each time by the qubit that lets the
// most remaining gates into the stage (two-qubit and wider gates weigh 4, one-
// qubit gates 1): a scan in program order admits a gate when its qubits lie in
// S and no earlier gate left out touches them, so the stage's gates may move
// ahead of the ones left out only where they share no qubit.  The admitted
// gates are multiplied into one block over S.  False (ops untouched) when the
// pass has a diagonal or a wider gate.
static bool fuse_stages(const std::vector<GateM> &gates, const std::vector<uint32_t> &acc, int kmax,
                        std::vector<HostOp> &ops, bool shape = false) {
  for (uint32_t gi : acc)
    if (gates[gi].diag || gates[gi].k > kmax) return false;
  std::vector<uint32_t> rem = acc, in, out;
  auto scan = [&](uint64_t S, std::vector<uint32_t> *a, std::vector<uint32_t> *r) {
    uint64_t blocked = 0;
    int score = 0;
    for (uint32_t gi : rem) {
      const GateM &g = gates[gi];
      if (!(g.mask & blocked) && (g.mask & ~S) == 0) {
        score += g.k >= 2 ? 4 : 1;
        if (a) a->push_back(gi);
      } else {
        blocked |= g.mask;
        if (r) r->push_back(gi);
      }
    }
    return score;
  };
  std::vector<HostOp> built;
  while (!rem.empty()) {
    uint64_t S = gates[rem[0]].mask;
    while (popc(S) < kmax) {
      uint64_t cand = 0;
      for (uint32_t gi : rem) cand |= gates[gi].mask;
      cand &= ~S;
      if (!cand) break;
      int best = -1;
      uint64_t bq = 0;
      for (uint64_t cq = cand; cq; cq &= cq - 1) {
        const uint64_t q = cq & (~cq + 1);
        const int sc = scan(S | q, nullptr, nullptr);
        if (sc > best) {
          best = sc;
          bq = q;
        }
      }
      S |= bq;
    }
    in.clear();
    out.clear();
    scan(S, &in, &out);
    Block b = identity_block(shape);
    for (uint64_t cq = S; cq; cq &= cq - 1) b = kron_blocks(b, qubit_block(ctz(cq), shape));
    for (uint32_t gi : in) apply_to_block(b, gates[gi]);
    HostOp op;
    op.type = OP_DENSE;
    op.blk = std::move(b);
    built.push_back(std::move(op));
    rem.swap(out);
  }
  ops.swap(built);
  return true;
}

static void put_bytes(std::vector<uint8_t> &buf, const void *p, size_t n) {
  const uint8_t *b = static_cast<const uint8_t *>(p);
  buf.insert(buf.end(), b, b + n);
}
static void align16(std::vector<uint8_t> &buf) {
  while (buf.size() % 16) buf.push_back(0);
}

// Register stages hold 2^Rb amplitudes per thread (Rb = 4 or 5 register
// bits); the persistent kernels take Rb + 5 <= T <= 13 with at least Rb
// non-low tile bits.
static bool T_reg_ok(int T, int c, int Rb) { return T - Rb >= 5 && T <= kMaxTile && T - c >= Rb; }

// The outer-term slots of one register or tensor-core pass (RegPhaseSlot):
// slot s collects the terms whose sum the kernels form once per tile.
struct WSlots {
  std::vector<std::vector<RegPhaseOuter>> slot;
  size_t terms = 0;
};

// Bytes a phase op adds to a pass's records at most: its record, its per-thread
// tables and its slots (entry, two sums, terms), with alignment.
static size_t rphase_bytes_max(const std::vector<HostTerm> &terms, int T, int Rb) {
  const size_t nt = size_t(1) << (T - Rb), nslot = size_t(1 + (T - Rb) + Rb);
  return sizeof(RegPhaseHdr) + size_t(Rb + 1) * nt * 4 + nslot * 16 + terms.size() * sizeof(RegPhaseOuter) + 64;
}

// Appends the OP_RPHASE record of a phase op placed in a register stage whose
// register bits are R (register index i <-> i-th lowest bit of R) and whose
// thread bit i is local bit tb[i] (i < ntb); its outer terms go to new slots
// of `ws`.  Returns the number of terms.  Terms on register bits only fold into
// D; a term touches at most two qubits (diagonal gates have one or two), so a
// term on an outer qubit has at most one more bit, a register or a thread bit.
static uint32_t put_rphase(const std::vector<HostTerm> &terms, uint32_t R, const uint8_t *tb, int ntb,
                           WSlots &ws, std::vector<uint8_t> &buf) {
  RegPhaseHdr h{};
  const int Rb = popc(uint64_t(R));
  const uint32_t nt = 1u << ntb;
  h.ntb = uint32_t(ntb);
  h.nt = nt;
  int tbi[32];
  for (int b = 0; b < 32; b++) tbi[b] = -1;
  for (int i = 0; i < ntb; i++) tbi[tb[i]] = i;
  // LB(t): the local index bits of thread t
  std::vector<uint32_t> LB(nt, 0);
  for (uint32_t t = 0; t < nt; t++)
    for (int i = 0; i < ntb; i++)
      if ((t >> i) & 1u) LB[t] |= 1u << tb[i];
  uint32_t dturn[32] = {0};
  std::vector<uint32_t> pre[6];
  const uint32_t nslot = uint32_t(1 + ntb + Rb);
  std::vector<std::vector<RegPhaseOuter>> sl(nslot);
  for (const HostTerm &t : terms) {
    uint32_t tmask = 0, jm = 0;
    int nreg = 0, reg0 = -1;
    for (int b : {t.la, t.lb}) {
      if (b < 0) continue;
      if ((R >> b) & 1u) {
        const int i = popc(uint64_t(R & ((1u << b) - 1u)));
        jm |= 1u << i;
        if (reg0 < 0) reg0 = i;
        nreg++;
      } else {
        tmask |= 1u << b;
      }
    }
    if (tmask == 0 && t.outer == 0) {
      for (int j = 0; j < (1 << Rb); j++)
        if ((uint32_t(j) & jm) == jm) dturn[j] += t.turn;
      continue;
    }
    const int k = nreg ? 1 + reg0 : 0;
    if (t.outer == 0) {
      if (pre[k].empty()) pre[k].assign(nt, 0u);
      for (uint32_t x = 0; x < nt; x++)
        if ((LB[x] & tmask) == tmask) pre[k][x] += t.turn;
    } else {
      const uint32_t s = k ? uint32_t(1 + ntb + (k - 1)) : (tmask ? uint32_t(1 + tbi[ctz(uint64_t(tmask))]) : 0u);
      sl[s].push_back(RegPhaseOuter{t.outer, t.turn, 0});
    }
  }
  for (int k = 0; k <= Rb; k++)
    if (!pre[k].empty()) h.pre_mask |= 1u << k;
  bool any = false;
  for (uint32_t s = 0; s < nslot; s++) {
    if (sl[s].empty()) continue;
    any = true;
    h.w_used |= s == 0 ? 1u : (s <= uint32_t(ntb) ? 2u : 1u << (2 + (s - 1 - ntb)));
  }
  if (any) {
    h.w_slot = uint32_t(ws.slot.size());
    for (auto &v : sl) {
      ws.terms += v.size();
      ws.slot.push_back(std::move(v));
    }
  }
  for (int j = 0; j < 32; j++) {
    if (dturn[j]) h.has_d = 1;
    const double a = 2.0 * M_PI * double(dturn[j]) / 4294967296.0;
    h.d[j] = make_float2(float(std::cos(a)), float(std::sin(a)));
  }
  put_bytes(buf, &h, sizeof(h));
  for (int k = 0; k <= Rb; k++)
    if (!pre[k].empty()) put_bytes(buf, pre[k].data(), pre[k].size() * 4);
  return uint32_t(terms.size());
}

// Appends a pass's slot table (RegPhaseSlot[n], the per-tile sums' scratch,
// the terms) and records it in the pass header; nothing when no slot is used.
static void put_wslots(const WSlots &ws, PlanPass &hp, std::vector<uint8_t> &buf) {
  if (ws.slot.empty()) return;
  align16(buf);
  const uint32_t n = uint32_t(ws.slot.size());
  const size_t at = buf.size();
  hp.w_off = uint32_t(at);
  hp.n_w = n;
  std::vector<RegPhaseSlot> tab(n);
  uint32_t b = 0;
  for (uint32_t s = 0; s < n; s++) {
    tab[s].begin = b;
    b += uint32_t(ws.slot[s].size());
    tab[s].end = b;
  }
  buf.resize(at + rphase_w_terms(n), 0);
  std::memcpy(buf.data() + at, tab.data(), n * sizeof(RegPhaseSlot));
  for (const auto &v : ws.slot)
    if (!v.empty()) put_bytes(buf, v.data(), v.size() * sizeof(RegPhaseOuter));
}

// ---------------------------------------------------------------------------
// register stages (KIND_REG passes)
// ---------------------------------------------------------------------------

struct HStage {
  uint32_t R = 0;        // local bits held in registers
  std::vector<int> ops;  // op indices (program order within the stage)
};

// Greedy, in op order: a stage takes every op whose earlier unplaced ops do not
// share a bit with it and whose bits fit the stage's Rb register bits.  Phase
// ops need no register bits.  The first stage of a register pass avoids the c
// low bits (it loads with the low bits on the lanes); that of a tensor-core pass
// may hold any (its load buffer is swizzled, see swzl).  The last stage stores whatever bits it
// holds: no store-only stage is appended (it would cost a whole-tile exchange
// through shared memory, more than the partly filled 32-byte sectors of a store
// whose lanes skip some low bits, which L2 merges before they reach DRAM),
// except for a single-stage pass whose SWAPs relabel the store's low qubits.
// With `tc` the dense ops of a stage become one product applied before the
// stage's phase ops, so a dense op that touches a bit of an accepted phase op
// waits for a later stage.
// `store_low` (default: the c low bits) is the set of local bits that the store
// puts on the lanes; it differs from the load's low bits when SWAPs relabel qubits
// (`store_natural` false: the store lanes are not local bits 0..c-1 in order, so a
// single stage cannot both load and store).
static void assign_stages(const std::vector<HostOp> &ops, const std::vector<uint32_t> &omask, int T,
                          int c, int Rb, std::vector<HStage> &st, bool tc = false, uint32_t store_low = 0,
                          bool store_natural = true) {
  const uint32_t all = (T >= 32) ? ~0u : ((1u << T) - 1u), low = (1u << c) - 1u;
  if (!store_low) store_low = low;
  std::vector<int> rem(ops.size());
  for (size_t i = 0; i < ops.size(); i++) rem[i] = int(i);
  bool first = true;
  while (!rem.empty()) {
    const uint32_t allowed = (first && !tc) ? (all & ~low) : all;
    HStage s;
    uint32_t blocked = 0;
    uint32_t phase_bits = 0;  // tc: bits of accepted phase ops (applied after the stage's product)
    std::vector<int> rest;
    for (int o : rem) {
      const uint32_t M = omask[o];
      if ((M & blocked) || (tc && ops[o].type == OP_DENSE && (M & phase_bits))) {
        blocked |= M;
        rest.push_back(o);
        continue;
      }
      if (ops[o].type == OP_PHASE) {
        s.ops.push_back(o);
        phase_bits |= M;
      } else if ((M & ~s.R) == 0) {
        s.ops.push_back(o);
      } else if ((M & ~allowed) == 0 && popc(uint64_t(s.R | M)) <= Rb) {
        s.R |= M;
        s.ops.push_back(o);
      } else {
        blocked |= M;
        rest.push_back(o);
      }
    }
    st.push_back(std::move(s));
    rem.swap(rest);
    first = false;
  }
  if (st.empty()) st.push_back(HStage{});
  (void)store_low;
  if (st.size() == 1 && !store_natural && !tc) st.push_back(HStage{});
  for (size_t i = 0; i < st.size(); i++) {
    uint32_t allowed = all;
    if (i == 0 && !tc) allowed &= ~low;
    for (int b = T - 1; b >= 0 && popc(uint64_t(st[i].R)) < Rb; b--)
      if (((allowed >> b) & 1u) && !((st[i].R >> b) & 1u)) st[i].R |= 1u << b;
  }
}

// `store_lanes` (store stages of relabeled passes): the local bits that hold
// output qubits 0..c-1, in that order, to be put on the lanes.
static StageRec make_stage(const HStage &hs, int T, int c, int Rb, bool load, bool store,
                           const std::vector<int> *store_lanes = nullptr, bool tc = false) {
  StageRec sr{};
  int nr = 0;
  for (int b = 0; b < T; b++)
    if ((hs.R >> b) & 1u) sr.rb[nr++] = uint8_t(b);
  std::vector<int> rest;
  for (int b = 0; b < T; b++)
    if (!((hs.R >> b) & 1u)) rest.push_back(b);
  std::vector<int> tb;
  bool lanes_free = store_lanes != nullptr;  // no store lane held in registers
  if (store_lanes)
    for (int b : *store_lanes) lanes_free &= !((hs.R >> b) & 1u);
  if (store && !load && lanes_free) {
    tb = *store_lanes;  // output qubits 0..c-1 on the lanes, then the rest ascending
    for (int b : rest)
      if (std::find(tb.begin(), tb.end(), b) == tb.end()) tb.push_back(b);
  } else if (load && tc) {
    // tensor-core passes read their first stage from the swizzled load buffer:
    // four half-warp lane bits with independent images under swzl, lowest first
    uint32_t basis[4] = {0, 0, 0, 0};
    std::vector<int> lanes, others;
    for (int b : rest) {
      uint32_t v = swzl_col(b);
      for (int i = 3; i >= 0; i--)
        if ((v >> i) & 1u) {
          if (basis[i]) {
            v ^= basis[i];
          } else {
            basis[i] = v;
            break;
          }
        }
      if (v && lanes.size() < 4) lanes.push_back(b);
      else others.push_back(b);
    }
    tb = lanes;
    std::sort(others.begin(), others.end());
    tb.insert(tb.end(), others.begin(), others.end());
  } else if (load) {
    tb = rest;  // ascending: the low tile bits sit on the lanes
  } else if (store) {
    // the lowest bits not held in registers on the lanes, for the store; a bit
    // whose swizzle image depends on the half-warp's earlier lane bits waits,
    // so the exchange read into this stage stays conflict-free (register
    // passes keep the c low bits out of their store stage, and get them in order)
    uint32_t basis[4] = {0, 0, 0, 0};
    std::vector<int> lanes, others;
    for (int b : rest) {
      uint32_t v = swz_col(b);
      for (int i = 3; i >= 0; i--)
        if ((v >> i) & 1u) {
          if (basis[i]) {
            v ^= basis[i];
          } else {
            basis[i] = v;
            break;
          }
        }
      if (v && lanes.size() < 4) lanes.push_back(b);
      else others.push_back(b);
    }
    tb = lanes;
    std::sort(others.begin(), others.end());
    tb.insert(tb.end(), others.begin(), others.end());
  } else {
    // four lane bits whose swizzle images are independent (one half-warp of
    // 8-byte accesses then hits 16 distinct bank pairs), then the others
    uint32_t basis[4] = {0, 0, 0, 0};
    std::vector<int> lanes, others;
    for (int b : rest) {
      uint32_t v = swz_col(b);
      for (int i = 3; i >= 0; i--)
        if ((v >> i) & 1u) {
          if (basis[i]) {
            v ^= basis[i];
          } else {
            basis[i] = v;
            break;
          }
        }
      if (v && lanes.size() < 4) lanes.push_back(b);
      else others.push_back(b);
    }
    tb = lanes;
    tb.insert(tb.end(), others.begin(), others.end());
  }
  for (size_t i = 0; i < tb.size() && i < 11; i++) sr.tb[i] = uint8_t(tb[i]);
  for (int j = 0; j < (1 << Rb); j++) {
    uint32_t l = 0;
    for (int i = 0; i < Rb; i++)
      if ((j >> i) & 1) l |= 1u << sr.rb[i];
    sr.la[j] = uint16_t(l);
    sr.pa[j] = uint16_t(swz(l));
    sr.xo[j] = uint32_t(swz(l)) * 8u;
  }
  sr.flags = (load ? 1u : 0u) | (store ? 2u : 0u);
  (void)c;
  return sr;
}

// U <- G * U for an NU x NU stage matrix U (NU = 16 or 32), G a k-qubit matrix
// on bit positions pos[].
static void apply_on_positions(std::vector<cd> &U, int NU, const std::vector<cd> &G, int k, const int *pos) {
  const int KG = 1 << k;
  int gmask = 0;
  for (int x = 0; x < k; x++) gmask |= 1 << pos[x];
  int off[32];
  for (int j = 0; j < KG; j++) {
    int o = 0;
    for (int x = 0; x < k; x++)
      if ((j >> x) & 1) o |= 1 << pos[x];
    off[j] = o;
  }
  cd v[32], w[32];
  for (int col = 0; col < NU; col++)
    for (int r0 = 0; r0 < NU; r0++) {
      if (r0 & gmask) continue;
      for (int j = 0; j < KG; j++) v[j] = U[size_t(r0 | off[j]) * NU + col];
      for (int r = 0; r < KG; r++) {
        cd a = 0.0;
        for (int j = 0; j < KG; j++) a += G[size_t(r) * KG + j] * v[j];
        w[r] = a;
      }
      for (int r = 0; r < KG; r++) U[size_t(r0 | off[r]) * NU + col] = w[r];
    }
}

// Packs a tensor-core pass (records after the PlanPass headers); false when
// it does not fit, leaving buf untouched.
static RegPassParams reg_params(const PlanPass &hp, const StageRec &first, const StageRec &last,
                                const int *outq);

// `outq`: local bit -> physical qubit of the store; `rp` receives the kernel's
// address tables and record checks.  Rb: register qubits of a stage (4: 16x16
// complex products, 5: 32x32).
static bool pack_tc_pass(const std::vector<HostOp> &ops, const std::vector<uint32_t> &omask, const int *lpos,
                         int T, int c, const int *outq, PlanPass &hp, std::vector<uint8_t> &buf,
                         RegPassParams &rp, sv_plan_info &info, int Rb) {
  const int NU = 1 << Rb, K = 2 * NU;
  std::vector<HStage> stages;
  assign_stages(ops, omask, T, c, Rb, stages, true);
  size_t nphase = 0, terms_bytes = 0, nmma = 0;
  for (auto &st : stages) {
    bool mma = false;
    for (int o : st.ops) {
      if (ops[o].type == OP_PHASE) {
        nphase++;
        terms_bytes += rphase_bytes_max(ops[o].terms, T, Rb);
      } else {
        mma = true;
      }
    }
    nmma += mma;
  }
  const size_t est = nphase * sizeof(OpRec) + terms_bytes + 16 * nphase + stages.size() * sizeof(StageRec) + 16 +
                     nmma * tc_b_image_bytes(Rb) + 16;
  if (stages.size() > 64 ||
      !tc_pass_fits(uint32_t(T), uint32_t(c), uint32_t(stages.size()), uint32_t(est), uint32_t(Rb)))
    return false;

  align16(buf);
  hp.ops_off = uint32_t(buf.size());
  const size_t ops_at = buf.size();
  buf.resize(buf.size() + nphase * sizeof(OpRec), 0);
  std::vector<OpRec> recs;
  std::vector<StageRec> srecs;
  std::vector<std::vector<double>> bmats;  // per MMA stage: B[n][k], K x K
  uint32_t nterms = 0;
  WSlots ws;
  for (size_t si = 0; si < stages.size(); si++) {
    const HStage &st = stages[si];
    StageRec sr = make_stage(st, T, c, Rb, si == 0, si + 1 == stages.size(), nullptr, true);
    sr.op_begin = uint32_t(recs.size());
    std::vector<cd> U(size_t(NU) * NU, 0.0);
    for (int d = 0; d < NU; d++) U[size_t(d) * (NU + 1)] = 1.0;
    bool mma = false;
    for (int o : st.ops) {
      const HostOp &op = ops[o];
      if (op.type == OP_PHASE) {
        OpRec r{};
        r.type = OP_RPHASE;
        align16(buf);
        r.data_off = uint32_t(buf.size());
        r.count = put_rphase(op.terms, st.R, sr.tb, T - Rb, ws, buf);
        nterms += r.count;
        info.n_phase++;
        recs.push_back(r);
      } else {
        const int k = op.blk.k();
        int pos[5];
        for (int m = 0; m < k; m++) pos[m] = popc(uint64_t(st.R & ((1u << lpos[op.blk.qs[m]]) - 1u)));
        apply_on_positions(U, NU, op.blk.M, k, pos);
        mma = true;
        info.n_blocks++;
        info.hist_k[k]++;
      }
    }
    sr.op_end = uint32_t(recs.size());
    if (mma) {
      sr.flags |= 4u;
      std::vector<double> B(size_t(K) * K);
      for (int r = 0; r < NU; r++)
        for (int j = 0; j < NU; j++) {
          const cd u = U[size_t(r) * NU + j];
          B[size_t(2 * r) * K + 2 * j] = u.real();
          B[size_t(2 * r) * K + 2 * j + 1] = -u.imag();
          B[size_t(2 * r + 1) * K + 2 * j] = u.imag();
          B[size_t(2 * r + 1) * K + 2 * j + 1] = u.real();
        }
      bmats.push_back(std::move(B));
    }
    srecs.push_back(sr);
  }
  std::memcpy(buf.data() + ops_at, recs.data(), recs.size() * sizeof(OpRec));
  align16(buf);
  hp.stages_off = uint32_t(buf.size());
  const size_t stage_at = buf.size();
  buf.resize(buf.size() + srecs.size() * sizeof(StageRec), 0);
  align16(buf);
  size_t bi = 0;
  std::vector<uint8_t> img(tc_b_image_bytes(Rb));
  for (auto &sr : srecs) {
    if (sr.flags & 4u) {
      sr.b_off = uint32_t(buf.size());
      tc_b_image(Rb, bmats[bi++].data(), img.data());
      put_bytes(buf, img.data(), img.size());
    }
  }
  std::memcpy(buf.data() + stage_at, srecs.data(), srecs.size() * sizeof(StageRec));
  put_wslots(ws, hp, buf);
  align16(buf);
  hp.data_bytes = uint32_t(buf.size() - hp.ops_off);
  hp.n_ops = uint32_t(recs.size());
  hp.n_stages = uint32_t(srecs.size());
  hp.n_phase_terms = nterms;
  hp.kind = KIND_TC;
  hp.R = uint32_t(Rb);
  rp = reg_params(hp, srecs.front(), srecs.back(), outq);
  rp.chk[0] = hp.T;
  rp.chk[1] = hp.n_stages;
  rp.chk[2] = hp.data_bytes;
  rp.chk[3] = hp.ops_off;
  info.n_stages += srecs.size();
  info.tc_stages += nmma;
  return true;
}

static uint64_t pdep_host(uint64_t x, uint64_t mask) {
  uint64_t out = 0;
  for (int b = 0; b < 64 && x; b++)
    if ((mask >> b) & 1) {
      if (x & 1) out |= uint64_t(1) << b;
      x >>= 1;
    }
  return out;
}

// Address tables of a KIND_REG pass (see RegPassParams).
static RegPassParams reg_params(const PlanPass &hp, const StageRec &first, const StageRec &last,
                                const int *outq) {
  RegPassParams p{};
  const uint32_t c = hp.c, cs = c - 1u;
  const uint32_t NT = 1u << (hp.T - hp.R);
  for (uint32_t x = 0; x < hp.T; x++) p.oq[x] = uint8_t(outq[x]);
  for (int j = 0; j < (1 << hp.R); j++) {
    // tensor-core passes: the load buffer is swizzled (swzl); the kernel xors
    // the thread's part in
    p.lo[j] = (hp.kind == KIND_TC ? swzl(first.la[j]) : uint32_t(first.la[j])) * 8u;
    const uint32_t l = last.la[j];
    uint64_t g = 0;
    for (uint32_t x = 0; x < hp.T; x++)
      if ((l >> x) & 1u) g |= uint64_t(1) << outq[x];
    p.go[j] = g;
  }
  for (uint32_t k = 0; k < (1u << (hp.R - 1)); k++) p.ko[k] = pdep_host(uint64_t(k) * (NT >> cs), hp.high_mask);
  return p;
}

// Accepted / rejected split of `rem` for a fixed tile set Q.
static void scan_fixed(const std::vector<GateM> &gates, const std::vector<uint32_t> &rem, uint64_t Q,
                       std::vector<uint32_t> &acc, std::vector<uint32_t> &rest) {
  uint64_t blocked = 0;
  acc.clear();
  rest.clear();
  for (uint32_t gi : rem) {
    const GateM &g = gates[gi];
    if (!(g.mask & blocked) && (g.diag || (g.mask & ~Q) == 0)) {
      acc.push_back(gi);
    } else {
      blocked |= g.mask;
      rest.push_back(gi);
    }
  }
}

// Non-diagonal gates among the first `limit` of `rem` that a fixed Q accepts.
static int count_fixed(const std::vector<GateM> &gates, const std::vector<uint32_t> &rem, size_t limit,
                       uint64_t Q) {
  uint64_t blocked = 0;
  int cnt = 0;
  for (size_t i = 0; i < limit; i++) {
    const GateM &g = gates[rem[i]];
    if (!(g.mask & blocked) && (g.diag || (g.mask & ~Q) == 0)) {
      cnt += !g.diag;
    } else {
      blocked |= g.mask;
    }
  }
  return cnt;
}

// Tile set grown by look-ahead: start from the low qubits and the first
// unapplied gate, then add single qubits, or the two outside qubits of a gate
// in the look-ahead window, scored by how many non-diagonal gates a scan of the
// window then accepts per added qubit.  With one set (beam_width 1) the set
// whose scan of all remaining gates accepts the most non-diagonal gates is
// taken, also from a beam of the beam_width best partial sets grown in step
// (one greedy choice often shuts out a better completion).  For tensor-core
// passes (stage_rank) the beam's complete sets are ranked instead by those
// gates per unit of estimated pass time, 3 + the tensor-core stages of the
// pass's gates fused as shapes (the constant gave the shortest estimated step
// on random 28- to 34-qubit circuits): fewer stages can be worth a pass more.
static uint64_t lookahead_tile(const std::vector<GateM> &gates, const std::vector<uint32_t> &rem, int n,
                               int T, uint64_t lowmask, size_t beam_width, bool stage_rank) {
  constexpr size_t kWindow = 96;
  const size_t W = std::min(rem.size(), kWindow);
  uint64_t Q0 = lowmask;
  for (uint32_t gi : rem)
    if (!gates[gi].diag) {
      if (popc(Q0 | gates[gi].mask) <= T) Q0 |= gates[gi].mask;
      break;
    }
  std::vector<uint64_t> beam = {Q0}, done, cand;
  std::vector<std::pair<double, uint64_t>> grown;
  while (!beam.empty()) {
    grown.clear();
    for (uint64_t Q : beam) {
      if (popc(Q) >= T) {
        done.push_back(Q);
        continue;
      }
      cand.clear();
      for (int q = 0; q < n; q++)
        if (!((Q >> q) & 1)) cand.push_back(uint64_t(1) << q);
      if (popc(Q) + 2 <= T)
        for (size_t i = 0; i < W; i++) {
          const uint64_t m = gates[rem[i]].mask & ~Q;
          if (popc(m) == 2) cand.push_back(m);
        }
      if (cand.empty()) {
        done.push_back(Q);
        continue;
      }
      for (uint64_t m : cand) grown.push_back({double(count_fixed(gates, rem, W, Q | m)) / popc(m), Q | m});
    }
    // best first; equal scores in mask order, so the plan is deterministic
    std::sort(grown.begin(), grown.end(), [](const std::pair<double, uint64_t> &a,
                                             const std::pair<double, uint64_t> &b) {
      return a.first > b.first || (a.first == b.first && a.second < b.second);
    });
    beam.clear();
    for (const auto &g : grown) {
      if (std::find(beam.begin(), beam.end(), g.second) == beam.end()) beam.push_back(g.second);
      if (beam.size() >= beam_width) break;
    }
  }
  uint64_t best = Q0;
  int best_n = -1;
  double best_r = -1.0;
  for (uint64_t Q : done) {
    const int k = count_fixed(gates, rem, rem.size(), Q);
    if (stage_rank) {
      std::vector<uint32_t> acc, rest;
      scan_fixed(gates, rem, Q, acc, rest);
      int lpos[64];
      for (int q = 0; q < 64; q++) lpos[q] = -1;
      int j = 0;
      for (int q = 0; q < n; q++)
        if (Q >> q & 1) lpos[q] = j++;
      std::vector<HostOp> ops;
      if (!fuse_stages(gates, acc, 4, ops, true)) fuse_pass(gates, acc, Q, lpos, 4, true, ops, nullptr, true);
      std::vector<uint32_t> om(ops.size(), 0);
      for (size_t i = 0; i < ops.size(); i++) {
        if (ops[i].type == OP_DENSE) {
          for (int q : ops[i].blk.qs) om[i] |= 1u << lpos[q];
        } else {
          for (auto &t : ops[i].terms) {
            if (t.la >= 0) om[i] |= 1u << t.la;
            if (t.lb >= 0) om[i] |= 1u << t.lb;
          }
        }
      }
      std::vector<HStage> st;
      assign_stages(ops, om, T, ctz(~lowmask), 4, st, true);
      const double r = double(k) / (3.0 + double(st.size()));
      if (r > best_r) {
        best_r = r;
        best = Q;
      }
      continue;
    }
    if (k > best_n) {
      best_n = k;
      best = Q;
    }
  }
  return best;
}

bool PlanBuilder::init(int n, const sv_gate *ir, size_t ng, const sv_opts *opts_in, std::string &err) {
  sv_opts o{};
  if (opts_in) o = *opts_in;
  int kmax = o.k_max ? o.k_max : 2;
  int T = o.tile_qubits ? o.tile_qubits : 12;
  int c = o.low_qubits ? o.low_qubits : 5;
  if (kmax < 1 || kmax > kMaxK) {
    err = "k_max must be in [1,5]";
    return false;
  }
  if (T < 1 || T > kMaxTile) {
    err = "tile_qubits must be in [1," + std::to_string(kMaxTile) + "]";
    return false;
  }
  if (o.precision < 0 || o.precision > 2) {
    err = "precision must be 0, 1 or 2";
    return false;
  }
  // kernel_variant: 0 = register stages where possible (32 amplitudes per
  // thread when the pass's blocks have at most 2 qubits and T <= 12, else 16),
  // 1 = shared-memory sweeps, 2 = register stages with 16 amplitudes per thread;
  // with precision 1 or 2, variant 2 fuses up to 5 qubits and gives every
  // tensor-core pass 5-qubit stages (32 amplitudes a thread)
  const bool o_smem = (o.kernel_variant == 1);
  if (o.kernel_variant < 0 || o.kernel_variant > 2) {
    err = "kernel_variant must be 0, 1 or 2";
    return false;
  }
  const bool o_r5 = (o.kernel_variant == 0);
  if (T > n) T = n;
  if (c > T) c = T;
  // a pass must be able to take any single gate (up to 5 qubits) next to the c low qubits
  int widest = 1;
  std::vector<GateM> &gates = gates_;
  gates.clear();
  if (!convert_ir(n, ir, ng, gates, err)) return false;
  for (auto &g : gates) widest = std::max(widest, g.k);
  if (T < n && T - c < widest) c = std::max(1, T - widest);
  if (T < n && T - c < widest) {
    err = "tile_qubits too small for a " + std::to_string(widest) + "-qubit gate";
    return false;
  }
  kmax = std::min(kmax, T);  // a wider UNITARY still gets a block of its own

  n_ = n;
  kmax_ = kmax;
  T_ = T;
  c_ = c;
  o_ = o;
  o_smem_ = o_smem;
  o_r5_ = o_r5;
  ng_ = ng;
  nmask_ = (n >= 64) ? ~uint64_t(0) : ((uint64_t(1) << n) - 1);
  lowmask_ = (uint64_t(1) << c) - 1;
  remaining_.resize(ng);
  for (size_t i = 0; i < ng; i++) remaining_[i] = uint32_t(i);
  return true;
}

bool PlanBuilder::next(Plan &plan, size_t max_passes, std::string &err) {
  const int n = n_, T = T_, c = c_;
  int kmax = kmax_;
  const sv_opts &o = o_;
  const bool o_smem = o_smem_, o_r5 = o_r5_;
  const std::vector<GateM> &gates = gates_;
  std::vector<uint32_t> &remaining = remaining_;
  plan = Plan();
  plan.n = n;
  plan.info.n_gates = first_ ? ng_ : 0;
  first_ = false;
  const uint64_t nmask = nmask_;
  const uint64_t lowmask = lowmask_;

  struct PassH {
    uint64_t Q;
    std::vector<HostOp> ops;
    std::vector<uint32_t> acc;  // accepted gates (program order)
    int lq[32];
    bool pairs;                 // fused with two-local-qubit phase terms
    int kfuse;                  // fusion width used
    bool relabeled;             // SWAPs folded into the store mapping
    int rho[64];                // qubit q's data ends at the loaded position of rho[q]
    // precision 1: the same gates fused for the CUDA-core register kernel (blocks
    // of <= 2 qubits, SWAPs folded into the store), for the per-pass choice
    bool has_alt = false;
    std::vector<HostOp> alt_ops;
    bool alt_pairs = false;
    int alt_rho[64];
  };
  std::vector<PassH> passes;

  while (!remaining.empty() && passes.size() < max_passes) {
    uint64_t Q = lowmask, blocked = 0;
    std::vector<uint32_t> acc, rest;
    acc.reserve(remaining.size());
    for (uint32_t gi : remaining) {
      const GateM &g = gates[gi];
      if (g.mask & blocked) {
        blocked |= g.mask;
        rest.push_back(gi);
        continue;
      }
      if (g.diag || (g.mask & ~Q) == 0) {
        acc.push_back(gi);
      } else if (popc(Q | g.mask) <= T) {
        Q |= g.mask;
        acc.push_back(gi);
      } else {
        blocked |= g.mask;
        rest.push_back(gi);
      }
    }
    if (acc.empty()) {
      err = "internal: pass planner made no progress";
      return false;
    }
    // fill the tile set up to T qubits with the lowest unused qubits
    for (int q = 0; q < n && popc(Q) < T; q++) Q |= uint64_t(1) << q;
    // rescan with the full tile set, and compare with the look-ahead tile set
    if (T < n) {
      auto nondiag = [&](const std::vector<uint32_t> &a) {
        size_t k = 0;
        for (uint32_t gi : a) k += !gates[gi].diag;
        return k;
      };
      std::vector<uint32_t> acc2, rest2;
      scan_fixed(gates, remaining, Q, acc2, rest2);
      if (nondiag(acc2) >= nondiag(acc)) {
        acc.swap(acc2);
        rest.swap(rest2);
      }
      // a beam of 8 partial tile sets from 27 qubits up: there a pass takes more
      // GPU time than planning it with the beam (~0.4 ms a pass on the host)
      uint64_t Ql = lookahead_tile(gates, remaining, n, T, lowmask, n >= 27 ? 8 : 1, n >= 27 && o.precision >= 1);
      for (int q = 0; q < n && popc(Ql) < T; q++) Ql |= uint64_t(1) << q;
      scan_fixed(gates, remaining, Ql, acc2, rest2);
      if (nondiag(acc2) > nondiag(acc)) {
        acc.swap(acc2);
        rest.swap(rest2);
        Q = Ql;
      }
    }
    PassH ph;
    ph.Q = Q;
    int lpos[64];
    for (int q = 0; q < 64; q++) lpos[q] = -1;
    int j = 0;
    for (int q = 0; q < n; q++)
      if (Q >> q & 1) {
        lpos[q] = j;
        ph.lq[j] = q;
        j++;
      }
    // two-local-qubit phase terms only where the pass can run on register stages
    int wmax = 1;
    for (uint32_t gi : acc) wmax = std::max(wmax, gates[gi].k);
    auto pairs_ok = [&](int k) { return !o_smem && k <= 4 && wmax <= 4 && T_reg_ok(popc(Q), c, 4); };
    // Fusion width: blocks of <= 2 qubits run on the 32-amplitude register
    // kernel (paired FMAs, 4 * 2^k FMA per amplitude); wider blocks cost 2^k more
    // each and run on slower kernels, so k_max > 2 is used for a pass only when
    // the wider fusion's estimated cost is lower.  Tensor-core stages take up to
    // 4 qubits at one cost.  A gate wider than the width keeps a block of its own.
    auto est = [](const std::vector<HostOp> &ops) {
      double w = 0.0;
      int kx = 0;
      for (const HostOp &op : ops) {
        if (op.type == OP_DENSE) {
          w += double(1 << op.blk.k());
          kx = std::max(kx, op.blk.k());
        } else {
          w += 4.0;
        }
      }
      return w * (kx <= 2 ? 1.0 : (kx <= 4 ? 1.3 : 4.0));
    };
    int kf = (o.precision >= 1) ? std::min(kmax, o.kernel_variant == 2 ? 5 : 4) : std::min(kmax, 2);
    // SWAPs of tile qubits become a relabeling of the store (register passes only)
    ph.relabeled = !o_smem && o.precision == 0;
    for (int q = 0; q < 64; q++) ph.rho[q] = q;
    ph.pairs = pairs_ok(kf);
    // The candidate forms are compared as shapes (qubits only); only the kept
    // form's matrices are multiplied out.
    bool staged_form = false;
    if (o.precision >= 1 && kf == 4 && !o_smem) {
      // tensor-core stages: the look-ahead stage former when it needs fewer stages
      auto n_stages = [&](const std::vector<HostOp> &ops) {
        std::vector<uint32_t> om(ops.size(), 0);
        for (size_t i = 0; i < ops.size(); i++) {
          if (ops[i].type == OP_DENSE) {
            for (int q : ops[i].blk.qs) om[i] |= 1u << lpos[q];
          } else {
            for (auto &t : ops[i].terms) {
              if (t.la >= 0) om[i] |= 1u << t.la;
              if (t.lb >= 0) om[i] |= 1u << t.lb;
            }
          }
        }
        std::vector<HStage> st;
        assign_stages(ops, om, popc(Q), c, 4, st, true);
        return st.size();
      };
      std::vector<HostOp> blocks, staged;
      fuse_pass(gates, acc, Q, lpos, kf, ph.pairs, blocks, nullptr, true);
      staged_form = fuse_stages(gates, acc, 4, staged, true) && n_stages(staged) < n_stages(blocks);
    }
    if (o.precision == 0 && kmax > kf) {
      // the wider fusion when its estimated cost is lower
      std::vector<HostOp> narrow, wide;
      const bool pw = pairs_ok(kmax);
      int rho_n[64], rho_w[64];
      for (int q = 0; q < 64; q++) rho_n[q] = rho_w[q] = q;
      fuse_pass(gates, acc, Q, lpos, kf, ph.pairs, narrow, ph.relabeled ? rho_n : nullptr, true);
      fuse_pass(gates, acc, Q, lpos, kmax, pw, wide, ph.relabeled ? rho_w : nullptr, true);
      if (est(wide) < est(narrow)) {
        ph.pairs = pw;
        kf = kmax;
      }
    }
    if (staged_form)
      fuse_stages(gates, acc, 4, ph.ops);
    else
      fuse_pass(gates, acc, Q, lpos, kf, ph.pairs, ph.ops, ph.relabeled ? ph.rho : nullptr);
    if (o.precision == 1 && o_r5) {
      // the CUDA-core form, as a shape: multiplied out if the pass goes there
      ph.has_alt = true;
      for (int q = 0; q < 64; q++) ph.alt_rho[q] = q;
      ph.alt_pairs = pairs_ok(std::min(kmax, 2));
      fuse_pass(gates, acc, Q, lpos, std::min(kmax, 2), ph.alt_pairs, ph.alt_ops, ph.alt_rho, true);
    }
    ph.kfuse = kf;
    ph.acc = std::move(acc);
    passes.push_back(std::move(ph));
    remaining.swap(rest);
  }

  // ---- pack -----------------------------------------------------------------
  std::vector<uint8_t> &buf = plan.bytes;
  const size_t P = passes.size();
  buf.resize(P * sizeof(PlanPass), 0);
  plan.passes.resize(P);
  plan.pass_offs.resize(P);
  plan.rparams.assign(P, RegPassParams{});
  const double amps = std::ldexp(1.0, n);
  for (size_t p = 0; p < P; p++) {
    PassH &ph = passes[p];
    PlanPass hp{};
    hp.outer_mask = nmask & ~ph.Q;
    hp.high_mask = ph.Q & ~lowmask;
    hp.T = uint32_t(popc(ph.Q));
    hp.c = uint32_t(c);
    hp.n_tiles = uint64_t(1) << (n - int(hp.T));
    hp.n_ops = uint32_t(ph.ops.size());
    for (int x = 0; x < 32; x++) hp.lq[x] = int8_t(x < int(hp.T) ? ph.lq[x] : -1);
    int lpos[64];
    for (int q = 0; q < 64; q++) lpos[q] = -1;
    for (int x = 0; x < int(hp.T); x++) lpos[ph.lq[x]] = x;

    // local-bit masks of the ops
    size_t nops = 0;
    std::vector<uint32_t> omask;
    uint32_t kmx = 0;
    auto op_masks = [&]() {
      nops = ph.ops.size();
      omask.assign(nops, 0);
      kmx = 0;
      for (size_t i = 0; i < nops; i++) {
        const HostOp &op = ph.ops[i];
        if (op.type == OP_DENSE) {
          for (int q : op.blk.qs) omask[i] |= 1u << lpos[q];
          kmx = std::max<uint32_t>(kmx, uint32_t(op.blk.k()));
        } else {
          for (auto &t : op.terms) {
            if (t.la >= 0) omask[i] |= 1u << t.la;
            if (t.lb >= 0) omask[i] |= 1u << t.lb;
          }
        }
      }
    };
    op_masks();
    // register stages when every block fits the registers of one thread
    const int T_ = int(hp.T);
    // store mapping: local bit x is written to physical qubit outq[x]; SWAPs folded
    // into the pass leave qubit q's data at local bit lpos[rho[q]]
    int outq[32];
    std::vector<int> store_lanes(size_t(c), 0);
    uint32_t store_low = 0;
    bool store_natural = true;
    auto store_map = [&]() {
      for (int x = 0; x < 32; x++) outq[x] = x < T_ ? ph.lq[x] : -1;
      if (ph.relabeled)
        for (int x = 0; x < T_; x++) outq[lpos[ph.rho[ph.lq[x]]]] = ph.lq[x];
      store_lanes.assign(size_t(c), 0);
      store_low = 0;
      for (int x = 0; x < T_; x++)
        if (outq[x] < c) {
          store_lanes[size_t(outq[x])] = x;
          store_low |= 1u << x;
        }
      store_natural = true;
      for (int q = 0; q < c; q++) store_natural &= store_lanes[size_t(q)] == q;
    };
    store_map();
    // Precision 1: a pass runs on the tensor cores unless the CUDA-core register
    // kernel (32 amplitudes a thread, blocks of <= 2 qubits, no phase ops) is
    // estimated faster.  Times in units of one HBM pass, fitted to both kernels'
    // measured passes on a 34-qubit state: tensor cores 0.66 + 0.47 per stage +
    // 0.36 per phase op; CUDA cores max(1.05, 0.30 + 0.10 per stage + 0.0075 per
    // block flop per amplitude).  Light passes (few stages of one- and two-qubit
    // blocks, SWAPs folded into the store) go to the CUDA cores.
    if (ph.has_alt && kmx <= 4 && T_reg_ok(T_, c, 5)) {
      std::vector<HStage> st;
      assign_stages(ph.ops, omask, T_, c, 4, st, true);
      size_t nph = 0;
      for (auto &op : ph.ops) nph += op.type == OP_PHASE;
      const double t_tc = 0.66 + 0.47 * double(st.size()) + 0.36 * double(nph);
      std::swap(ph.ops, ph.alt_ops);
      std::swap(ph.pairs, ph.alt_pairs);
      std::swap(ph.rho, ph.alt_rho);
      ph.relabeled = true;
      op_masks();
      store_map();
      bool light = kmx <= 2;
      double flop = 0.0;
      for (auto &op : ph.ops) {
        if (op.type == OP_PHASE) light = false;
        else flop += 8.0 * double(1 << op.blk.k());
      }
      bool use_cc = false;
      if (light) {
        st.clear();
        assign_stages(ph.ops, omask, T_, c, 5, st, false, store_low, store_natural);
        const double t_cc = std::max(1.05, 0.30 + 0.10 * double(st.size()) + 0.0075 * flop);
        use_cc = t_cc < t_tc - 0.05;
      }
      if (!use_cc) {
        std::swap(ph.ops, ph.alt_ops);
        std::swap(ph.pairs, ph.alt_pairs);
        std::swap(ph.rho, ph.alt_rho);
        ph.relabeled = false;
        op_masks();
        store_map();
      } else {
        ph.kfuse = std::min(kmax, 2);
        int rho[64];
        for (int q = 0; q < 64; q++) rho[q] = q;
        ph.ops.clear();
        fuse_pass(gates, ph.acc, ph.Q, lpos, ph.kfuse, ph.pairs, ph.ops, rho);
      }
      hp.n_ops = uint32_t(nops);
    }
    // tensor-core stages (precision 1) when the pass fits the TC kernel: 4-qubit
    // stages, or 5-qubit stages for a pass holding a 5-qubit block (or all
    // passes with kernel variant 2), else 4-qubit ones if those fit
    const int Rtc = (kmx == 5 || o.kernel_variant == 2) ? 5 : 4;
    if (o.precision >= 1 && kmx <= 5 && !ph.relabeled &&
        (pack_tc_pass(ph.ops, omask, lpos, int(hp.T), c, outq, hp, buf, plan.rparams[p], plan.info, Rtc) ||
         (Rtc == 5 && kmx <= 4 &&
          pack_tc_pass(ph.ops, omask, lpos, int(hp.T), c, outq, hp, buf, plan.rparams[p], plan.info, 4)))) {
      hp.kmax = kmx;
      for (auto &op : ph.ops)
        if (op.type == OP_DENSE) plan.info.flops += uint64_t(amps * 8.0 * double(1 << op.blk.k()));
      std::memcpy(buf.data() + p * sizeof(PlanPass), &hp, sizeof(hp));
      plan.passes[p] = hp;
      plan.pass_offs[p] = uint32_t(p * sizeof(PlanPass));
      continue;
    }
    // register stages hold 2^Rb amplitudes per thread (blocks up to 4
    // qubits); passes with 5-qubit blocks use the shared-memory kernel
    const int Rb = (o_r5 && kmx <= 2 && T_reg_ok(T_, c, 5)) ? 5 : 4;
    const bool use_reg = !o_smem && kmx <= 4 && T_reg_ok(T_, c, Rb);
    std::vector<HStage> stages;
    std::vector<int> order;
    bool reg = use_reg;
    if (reg) {
      assign_stages(ph.ops, omask, T_, c, Rb, stages, false, store_low, store_natural);
      // bytes of this pass's records as packed below (16-byte aligned pieces)
      size_t est = nops * sizeof(OpRec) + stages.size() * sizeof(StageRec) + 16;
      for (auto &op : ph.ops)
        est += op.type == OP_DENSE ? ((size_t(16) << (2 * op.blk.k())) + 15) / 16 * 16
                                   : rphase_bytes_max(op.terms, T_, Rb);
      if (!reg_pass_fits(uint32_t(T_), uint32_t(c), uint32_t(Rb), uint32_t(stages.size()), uint32_t(est))) {
        reg = false;
        stages.clear();
      }
    }
    if (!reg && (ph.pairs || ph.relabeled)) {
      // the shared-memory kernel takes phase terms with one tile qubit only and
      // stores in the loaded order
      ph.ops.clear();
      fuse_pass(gates, ph.acc, ph.Q, lpos, ph.kfuse, false, ph.ops);
      ph.pairs = false;
      ph.relabeled = false;
      op_masks();
      hp.n_ops = uint32_t(nops);
    }
    if (reg) {
      for (auto &st : stages) order.insert(order.end(), st.ops.begin(), st.ops.end());
    } else {
      for (size_t i = 0; i < nops; i++) order.push_back(int(i));
    }
    std::vector<int> stage_of(nops, -1);
    for (size_t si = 0; si < stages.size(); si++)
      for (int o : stages[si].ops) stage_of[o] = int(si);
    std::vector<StageRec> srecs;
    for (size_t si = 0; si < stages.size(); si++)
      srecs.push_back(make_stage(stages[si], T_, c, Rb, si == 0, si + 1 == stages.size(),
                                 store_natural ? nullptr : &store_lanes));
    WSlots ws;

    align16(buf);
    hp.ops_off = uint32_t(buf.size());
    const size_t ops_at = buf.size();
    buf.resize(buf.size() + nops * sizeof(OpRec), 0);
    std::vector<OpRec> recs(nops);
    uint32_t nterms = 0;
    for (size_t oi = 0; oi < nops; oi++) {
      HostOp &op = ph.ops[order[oi]];
      OpRec r{};
      r.type = op.type;
      align16(buf);
      r.data_off = uint32_t(buf.size());
      if (op.type == OP_DENSE) {
        const int k = op.blk.k();
        r.k = uint8_t(k);
        for (int m = 0; m < k; m++) r.lb[m] = uint8_t(lpos[op.blk.qs[m]]);
        const int K = 1 << k;
        // matrix bit order: block order, or ascending register position
        int perm[5];
        for (int m = 0; m < k; m++) perm[m] = m;
        if (reg) {
          const HStage &st = stages[stage_of[order[oi]]];
          int pos[5];
          for (int m = 0; m < k; m++) pos[m] = popc(st.R & ((1u << r.lb[m]) - 1u));
          std::sort(perm, perm + k, [&](int a, int b) { return pos[a] < pos[b]; });
          for (int m = 0; m < k; m++) r.rmask |= uint8_t(1u << pos[m]);
        }
        // new index bit i <- old matrix bit perm[i]
        auto old_index = [&](int x) {
          int o = 0;
          for (int i = 0; i < k; i++)
            if (x >> i & 1) o |= 1 << perm[i];
          return o;
        };
        for (int rr = 0; rr < K; rr++)
          for (int cc = 0; cc < K; cc++) {
            const cd e = op.blk.M[size_t(old_index(rr)) * K + old_index(cc)];
            if (reg) {
              // register stages: (re, re, -im, im), the operands of two paired FMAs
              const float a = float(e.real()), b = float(e.imag());
              float f[4] = {a, a, -b, b};
              put_bytes(buf, f, sizeof(f));
            } else {
              float f[2] = {float(e.real()), float(e.imag())};
              put_bytes(buf, f, sizeof(f));
            }
          }
        plan.info.n_blocks++;
        plan.info.hist_k[k]++;
        plan.info.flops += uint64_t(amps * 8.0 * K);
      } else if (reg) {
        r.type = OP_RPHASE;
        const int si = stage_of[order[oi]];
        r.count = put_rphase(op.terms, stages[si].R, srecs[si].tb, T_ - Rb, ws, buf);
        nterms += r.count;
        plan.info.n_phase++;
      } else {
        r.count = uint32_t(op.terms.size());
        for (auto &t : op.terms) {
          PhaseTerm pt{};
          pt.outer_mask = t.outer;
          pt.la = t.la;
          pt.turn = t.turn;
          put_bytes(buf, &pt, sizeof(pt));
        }
        nterms += r.count;
        plan.info.n_phase++;
      }
      recs[oi] = r;
    }
    std::memcpy(buf.data() + ops_at, recs.data(), recs.size() * sizeof(OpRec));
    hp.kmax = kmx;
    hp.n_phase_terms = nterms;
    hp.kind = reg ? KIND_REG : KIND_SMEM;
    if (reg) {
      hp.R = uint32_t(Rb);
      hp.n_stages = uint32_t(stages.size());
      align16(buf);
      hp.stages_off = uint32_t(buf.size());
      uint32_t ob = 0;
      StageRec first{}, last{};
      for (size_t si = 0; si < stages.size(); si++) {
        StageRec sr = srecs[si];
        sr.op_begin = ob;
        ob += uint32_t(stages[si].ops.size());
        sr.op_end = ob;
        put_bytes(buf, &sr, sizeof(sr));
        if (si == 0) first = sr;
        if (si + 1 == stages.size()) last = sr;
      }
      plan.rparams[p] = reg_params(hp, first, last, outq);
      plan.info.n_stages += stages.size();
      put_wslots(ws, hp, buf);
    }
    align16(buf);
    hp.data_bytes = uint32_t(buf.size() - hp.ops_off);
    if (reg) {
      // the kernel checks its device copy of the records against these
      RegPassParams &rp = plan.rparams[p];
      rp.chk[0] = hp.T;
      rp.chk[1] = hp.n_stages;
      rp.chk[2] = hp.data_bytes;
      rp.chk[3] = hp.ops_off;
    }
    std::memcpy(buf.data() + p * sizeof(PlanPass), &hp, sizeof(hp));
    plan.passes[p] = hp;
    plan.pass_offs[p] = uint32_t(p * sizeof(PlanPass));
  }
  align16(buf);
  for (auto &hp : plan.passes) plan.info.passes_by_kind[hp.kind < 3 ? hp.kind : 0]++;
  plan.info.n_passes = P;
  plan.info.bytes = uint64_t(double(P) * 16.0 * amps);
  plan.info.upload_bytes = buf.size();
  plan.precision = o.precision;
  return true;
}

bool build_plan(int n, const sv_gate *ir, size_t ng, const sv_opts *opts, Plan &plan, std::string &err) {
  PlanBuilder b;
  if (!b.init(n, ir, ng, opts, err)) return false;
  return b.next(plan, SIZE_MAX, err);
}

}  // namespace svgb
