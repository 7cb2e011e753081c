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

}  // namespace svgb
