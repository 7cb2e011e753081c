// sv_plan.h -- host planner interface (sv_plan.cpp).
#pragma once

#include <complex>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/sv.h"
#include "sv_internal.h"

namespace svgb {

struct GateM {
  int k = 0;
  int q[5] = {0, 0, 0, 0, 0};
  uint64_t mask = 0;
  bool diag = false;
  bool swap = false;  // SWAP gate (a pure exchange of two qubits)
  bool unitary = true;  // false for a UNITARY matrix with max |U^dagger U - I| > 1e-6
  std::vector<std::complex<double>> m;  // 2^k x 2^k row-major
};

struct Plan {
  int n = 0;
  int precision = 0;
  std::vector<uint8_t> bytes;        // packed PlanPass[P], OpRec[], matrices, terms
  std::vector<PlanPass> passes;      // host copies
  std::vector<uint32_t> pass_offs;   // byte offset of each PlanPass
  std::vector<RegPassParams> rparams;  // KIND_REG passes: kernel address tables
  sv_plan_info info{};
};

bool convert_ir(int n, const sv_gate *ir, size_t ng, std::vector<GateM> &gates, std::string &err);
bool build_plan(int n, const sv_gate *ir, size_t ng, const sv_opts *opts, Plan &plan,
                std::string &err);

// Incremental planner: init() validates and converts the IR; each next() plans up
// to max_passes further passes and packs them as a standalone Plan, so a caller
// can launch the first passes while later ones are still being planned.
class PlanBuilder {
 public:
  bool init(int n, const sv_gate *ir, size_t ng, const sv_opts *opts, std::string &err);
  bool done() const { return remaining_.empty(); }
  // Every gate of the circuit is unitary (named gates; UNITARY matrices within 1e-6).
  bool unitary() const {
    for (const GateM &g : gates_)
      if (!g.unitary) return false;
    return true;
  }
  bool next(Plan &plan, size_t max_passes, std::string &err);

 private:
  int n_ = 0, kmax_ = 2, T_ = 12, c_ = 5;
  sv_opts o_{};
  bool o_smem_ = false, o_r5_ = false, first_ = true;
  uint64_t nmask_ = 0, lowmask_ = 0;
  size_t ng_ = 0;
  std::vector<GateM> gates_;
  std::vector<uint32_t> remaining_;
};

}  // namespace svgb
