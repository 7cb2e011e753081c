"""The runtime model's interpolation and regression pieces against closed forms
and scipy's monotone cubic interpolant (CPU only)."""
import numpy as np
import pytest

from paper_2512_04216_gb300 import costmodel as CM


def test_pchip_reproduces_knots_and_cubics_of_lines():
    x = np.array([10.0, 12, 15, 16, 20])
    y = 3.0 * x - 7.0
    f = CM.pchip(x, y)
    assert np.allclose(f(x), y, atol=1e-12)
    t = np.linspace(10, 20, 57)
    assert np.allclose(f(t), 3.0 * t - 7.0, atol=1e-12)  # a line is reproduced exactly


def test_pchip_is_monotone_on_monotone_data():
    rng = np.random.default_rng(3)
    x = np.cumsum(rng.uniform(0.5, 2.0, 9))
    y = np.cumsum(rng.uniform(0.0, 3.0, 9))
    t = np.linspace(x[0], x[-1], 2001)
    v = CM.pchip(x, y)(t)
    assert np.all(np.diff(v) >= -1e-12)


def test_pchip_matches_scipy():
    interp = pytest.importorskip("scipy.interpolate")
    rng = np.random.default_rng(5)
    for _ in range(5):
        x = np.cumsum(rng.uniform(0.3, 2.0, 8))
        y = rng.normal(size=8)
        t = np.linspace(x[0], x[-1], 501)
        want = interp.PchipInterpolator(x, y)(t)
        assert np.allclose(CM.pchip(x, y)(t), want, atol=1e-10)


def test_linear_fit_recovers_coefficients():
    S = np.array([1, 10, 100, 1000, 1e5])
    c1, c2 = CM.linear_fit(S, 0.25 + 3e-6 * S)
    assert abs(c1 - 0.25) < 1e-12 and abs(c2 - 3e-6) < 1e-15


def test_model_curves_interpolate_in_log_space():
    m = CM.CostModel(ns=[10, 20, 30], c_pass=[1e-3, 1e-3 * 2 ** 10, 1e-3 * 2 ** 20], c_flop=1e-12, c_fix=0.05,
                     c_shot1=[0.1, 0.2, 0.4], c_shot2=1e-5)
    # 2^n growth is exact in log space
    assert abs(m.apply_ms(25, 1, 0.0) - (0.05 + 1e-3 * 2 ** 15)) < 1e-9
    assert abs(m.apply_ms(20, 2, 1e9) - (0.05 + 2 * 1e-3 * 2 ** 10 + 1e-3)) < 1e-9
    assert abs(m.shots_ms(20, 1000) - (0.2 + 1e-2)) < 1e-12
    assert CM.CostModel.from_json(m.to_json()) == m


def test_dense_gate_count_skips_diagonal_gates():
    """The host term counts the gates the planner multiplies into blocks: every
    non-diagonal gate; z, s, sdg, t, tdg, rz, p, cz and cp only add phase terms."""
    capi = pytest.importorskip("paper_2512_04216_gb300.capi")
    import workloads as W
    n = 10
    qft = W.qft(n)
    ir, keep = capi.to_ir(qft)
    assert CM.CostModel.dense_gates(ir, len(qft)) == n + n // 2  # H on every qubit, the final SWAPs
    rl = W.random_layered(n, 3, 1)
    ir, keep = capi.to_ir(rl)
    assert CM.CostModel.dense_gates(ir, len(rl)) == len(rl)
    mixed = [("z", (0,), ()), ("s", (1,), ()), ("sdg", (2,), ()), ("t", (3,), ()), ("tdg", (4,), ()),
             ("rz", (5,), (0.3,)), ("p", (6,), (0.2,)), ("cz", (0, 1), ()), ("cp", (2, 3), (0.1,)),
             ("x", (0,), ()), ("y", (1,), ()), ("rx", (2,), (0.4,)), ("swap", (3, 4), ())]
    ir, keep = capi.to_ir(mixed)
    assert CM.CostModel.dense_gates(ir, len(mixed)) == 4
    m = CM.CostModel(ns=[10, 20], c_pass=[1.0, 2.0], c_flop=0.0, c_fix=0.5, c_gate=0.01, c_phase=1e-6)
    assert abs(m.apply_ms(10, 3, 0.0, 100) - (0.5 + 1.0 + 3 * 1.0)) < 1e-12
    assert abs(m.apply_ms(10, 3, 0.0, 100, 2.0 * 1024) - (0.5 + 1.0 + 3 * 1.0 + 1e-6 * 2048)) < 1e-12
    st = {"flops": 123.0, "n_phase": 3}
    assert CM.CostModel.eff_flops(10, st) == 123.0 and CM.CostModel.phase_amps(10, st) == 3 * 1024
