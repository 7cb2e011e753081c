"""Plant plausible mistakes in a copy of the oracle (CPU only) and check that
the pins catch every one of them: a pin set that a dropped term, a wrong sign,
a swapped index or a transposed operand slips through would not pin anything.
"""
import os
import subprocess

import pytest

import oracle
from oracle import build as obuild
from tests import oracle_pins as P

MUTANTS = {
    "u3_sign": ("m[1] = -cexp(I * p[2]) * s;", "m[1] = cexp(I * p[2]) * s;"),
    "u3_phase": ("m[3] = cexp(I * (p[1] + p[2])) * c;", "m[3] = cexp(I * (p[1] - p[2])) * c;"),
    "u3_swap_phi_lambda": ("m[2] = cexp(I * p[1]) * s;", "m[2] = cexp(I * p[2]) * s;"),
    "rz_sign": ("m[0] = cexp(-I * p[0] / 2.0); m[1] = 0;", "m[0] = cexp(I * p[0] / 2.0); m[1] = 0;"),
    "y_sign": ("m[0] = 0; m[1] = -I; m[2] = I;", "m[0] = 0; m[1] = I; m[2] = -I;"),
    "target_bit_order": ("if ((j >> m) & 1) o |= 1ull << t[m];", "if ((j >> m) & 1) o |= 1ull << t[k - 1 - m];"),
    "cx_control_target": ("m[0 * 4 + 0] = 1; m[2 * 4 + 2] = 1; m[1 * 4 + 3] = 1; m[3 * 4 + 1] = 1;",
                          "m[0 * 4 + 0] = 1; m[1 * 4 + 1] = 1; m[2 * 4 + 3] = 1; m[3 * 4 + 2] = 1;"),
    "matrix_transposed": ("acc += M[r * K + j] * v[j];", "acc += M[j * K + r] * v[j];"),
    "dropped_last_column": ("for (int j = 0; j < K; j++) acc += M", "for (int j = 0; j < K - 1; j++) acc += M"),
    "sampler_not_strict": ("if (C[mid] > t) hi = mid;", "if (C[mid] >= t) hi = mid;"),
    "sampler_unnormalised": ("double t = u[s] * total;", "double t = u[s];"),
    "sampler_no_lower_boundary": ("int b = (fabs(t - C[x]) < eps) || (fabs(t - below) < eps);",
                                  "int b = (fabs(t - C[x]) < eps);"),
    "cdf_drops_imag": ("s += re * re + im * im;\n    C[i] = s;", "s += re * re;\n    C[i] = s;"),
    "expect_sign": ("num += (__builtin_popcountll(i & zmask) & 1) ? -p : p;",
                    "num += (__builtin_popcountll(i & zmask) & 1) ? p : -p;"),
    "expect_unnormalised": ("return num / den;", "return num;"),
    "validate_allows_duplicates": ("if (g[a].q[x] == g[a].q[y]) return -1;", "(void)y;"),
    "measure_rule_flipped": ("const int outcome = (u * (m0 + m1) < m0) ? 0 : 1;",
                             "const int outcome = (u * (m0 + m1) < m0) ? 1 : 0;"),
    "measure_not_renormalised": ("const double scale = 1.0 / sqrt(m);", "const double scale = 1.0;"),
    "measure_wrong_qubit": ("int orc_measure(cplx *psi, uint64_t N, int q, double u, double *prob) {\n  const uint64_t bit = (uint64_t)1 << q;",
                            "int orc_measure(cplx *psi, uint64_t N, int q, double u, double *prob) {\n  const uint64_t bit = (uint64_t)1 << (q ^ 1);"),
    "reset_no_flip": ("  if (outcome) {\n    const uint64_t bit", "  if (0) {\n    const uint64_t bit"),
    "kron_operands_swapped": ("out[ib * Na + ia] = b[ib] * a[ia];", "out[ia * Nb + ib] = b[ib] * a[ia];"),
    "take_wrong_half": ("| ((uint64_t)v << q);", "| ((uint64_t)(1 - v) << q);"),
    "alias_lights_to_last_heavy": ("alias[i] = (uint32_t)heavy[j];", "alias[i] = (uint32_t)heavy[nh - 1];"),
    "alias_drops_carried_deficit": ("r = Q[heavy[j + 1]] - (C - r);", "r = Q[heavy[j + 1]];"),
    "alias_light_threshold": ("if (Q[i] < C) light[nl++] = i;", "if (Q[i] <= C) light[nl++] = i;"),
    "alias_unscaled": ("nearbyint(p * scale * 2147483648.0)", "nearbyint(p * 2147483648.0)"),
    "alias_coin_flipped": ("(f * 2147483648.0 < (double)own[i]) ? i : alias[i]",
                           "(f * 2147483648.0 < (double)own[i]) ? alias[i] : i"),
    "alias_converted_keeps_full": ("own[heavy[j]] = (uint32_t)r;", "own[heavy[j]] = (uint32_t)C;"),
    "alias_plain_running_sum": ("  W += comp;", "  (void)comp;"),
    "pauli_y_sign": ("const cplx Y[4] = {0, -I, I, 0};", "const cplx Y[4] = {0, I, -I, 0};"),
    "pauli_x_as_z": ("else if (xb) orc_apply_matrix(phi, n, 1, &t, X);", "else if (xb) orc_apply_matrix(phi, n, 1, &t, Z);"),
    "pauli_no_conjugate": ("num += conj(psi[i]) * phi[i];", "num += psi[i] * phi[i];"),
    "pauli_unnormalised": ("*out_re = creal(num) / den;", "*out_re = creal(num);"),
}


def _build_mutant(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(obuild.SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique/not found"
    path = os.path.join(str(tmp_path), f"{name}.c")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    so = os.path.join(str(tmp_path), f"lib{name}.so")
    subprocess.run(["gcc", "-O1", "-std=gnu99", "-fPIC", "-shared", "-o", so, path, "-lm"], check=True)
    return oracle.Oracle(so)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    o = _build_mutant(tmp_path, name)
    caught = []
    for pin in P.ALL_PINS:
        try:
            pin(o)
        except (AssertionError, ValueError) as e:
            # a ValueError is the oracle rejecting a valid input: also a catch
            caught.append(f"{pin.__name__}: {str(e)[:60]}")
    assert caught, f"mutant {name} passed every pin"
