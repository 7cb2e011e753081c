"""Tensor-core (tcgen05, 3xTF32) path: the stage product against an FP64
product, and whole circuits with precision=2 (every pass that fits on the
tensor cores) and precision=1 (the planner's per-pass choice between the
tensor-core and the CUDA-core register kernel) against the complex128 oracle.

Tolerances: the split-TF32 product keeps about float32 accuracy -- per element
|d - d_fp64| <= 2e-6 * (sum_k |a_mk| |b_nk|), versus ~1e-3 for one plain TF32
product; whole circuits use the complex64 bar of the other GPU tests
(per-amplitude abs error <= 1e-5, fidelity >= 1 - 1e-6).
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

AMP_TOL = 1e-5
FID_TOL = 1e-6


@pytest.fixture(scope="module")
def sv():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    import paper_2512_04216_gb300 as P
    return P


def test_tc_product_matches_fp64(sv):
    rng = np.random.default_rng(0)
    for scale in (1.0, 1e-3, 37.0):
        a = (rng.standard_normal((128, 32)) * scale).astype(np.float32)
        b = rng.standard_normal((32, 32))
        d = sv.capi.sv_tc_selftest(a, b)
        want = a.astype(np.float64) @ b.T
        bound = np.abs(a.astype(np.float64)) @ np.abs(b).T
        err = np.abs(d - want)
        assert np.all(err <= 2e-6 * bound + 1e-30), float(np.max(err / bound))
        # the split matters: one plain TF32 product would be ~1e-3 off
        assert float(np.max(err / bound)) < 1e-5


def test_tc_product_unitary_embedding(sv):
    # the real embedding of a complex 16x16 unitary maps rows of 16 complex
    # amplitudes (interleaved re, im) to the rows of U psi
    rng = np.random.default_rng(1)
    z = rng.standard_normal((16, 16)) + 1j * rng.standard_normal((16, 16))
    U, _ = np.linalg.qr(z)
    B = np.zeros((32, 32))
    B[0::2, 0::2] = U.real
    B[0::2, 1::2] = -U.imag
    B[1::2, 0::2] = U.imag
    B[1::2, 1::2] = U.real
    psi = rng.standard_normal((128, 16)) + 1j * rng.standard_normal((128, 16))
    a = np.empty((128, 32), dtype=np.float32)
    a[:, 0::2] = psi.real
    a[:, 1::2] = psi.imag
    d = sv.capi.sv_tc_selftest(a, B)
    out = d[:, 0::2] + 1j * d[:, 1::2]
    want = psi.astype(np.complex64).astype(np.complex128) @ U.T
    assert np.max(np.abs(out - want)) < 1e-5


def _run(P, n, circ, psi0=None, precision=2, **opts):
    s = P.StateVector(n)
    if psi0 is not None:
        s.set_amplitudes(psi0)
    s.apply(circ, precision=precision, **opts)
    g = s.amplitudes().astype(np.complex128)
    s.close()
    return g


def _compare(g, ref, what):
    err = float(np.max(np.abs(g - ref)))
    fid = oracle.fidelity(ref, g)
    assert err <= AMP_TOL, f"{what}: max abs err {err:.3e}"
    assert fid >= 1 - FID_TOL, f"{what}: fidelity {fid!r}"


@pytest.mark.parametrize("T", [11, 12, 13])
@pytest.mark.parametrize("k_max", [2, 4])
def test_tc_random_layered(sv, T, k_max):
    n = 16
    circ = W.random_layered(n, 14, 21)
    info = sv.capi.sv_plan_stats(n, circ, sv.capi.make_opts(k_max, T, 5, 2))
    assert info["tc_stages"] > 0
    _compare(_run(sv, n, circ, k_max=k_max, tile_qubits=T), oracle.run(n, circ), f"T={T} k={k_max}")


def test_tc_config1_small(sv):
    n, d = 12, 20
    c = W.random_layered(n, d, 1)
    _compare(_run(sv, n, c, tile_qubits=11, k_max=4), oracle.run(n, c), "n=12 d=20 T=11")


@pytest.mark.parametrize("n", [11, 13, 15])
def test_tc_gate_soup(sv, n):
    rng = np.random.default_rng(n)
    circ = W.random_gate_soup(n, 200, seed=700 + n)
    for k in (3, 4):
        qs = tuple(int(q) for q in rng.choice(n, size=k, replace=False))
        z = rng.standard_normal((1 << k, 1 << k)) + 1j * rng.standard_normal((1 << k, 1 << k))
        u, _ = np.linalg.qr(z)
        circ.insert(len(circ) // 3, ("unitary", qs, (u,)))
    psi0 = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    psi0 = (psi0 / np.linalg.norm(psi0)).astype(np.complex64)
    ref = oracle.run(n, circ, psi0.astype(np.complex128))
    _compare(_run(sv, n, circ, psi0, k_max=4, tile_qubits=min(n, 12)), ref, f"soup n={n}")


def test_tc_qft_closed_form(sv):
    for n in (14, 18):
        x = W.basis_index(n, 5)
        s = sv.StateVector(n, basis_index=x)
        s.apply(W.qft(n), precision=2, k_max=4)
        g = s.amplitudes().astype(np.complex128)
        s.close()
        y = np.arange(1 << n)
        _compare(g, np.exp(2j * np.pi * ((x * y) % (1 << n)) / (1 << n)) / math.sqrt(1 << n), f"QFT {n}")


def test_tc_mirror_28(sv):
    n = 28
    c = W.random_layered(n, 40, 2)
    s = sv.StateVector(n)
    s.apply(c + W.inverse(c), precision=2, k_max=4)
    a0 = s.amplitudes(0, 1)[0]
    norm2 = s.norm2()
    # fidelity with |0...0>: |a_0|^2 / ||psi||^2
    assert abs(a0) ** 2 / norm2 >= 1 - FID_TOL, (abs(a0) ** 2, norm2)
    # The tensor cores' float32 accumulation rounds toward zero (~1e-7 of norm
    # per stage product, ~500 products here); the passes of a unitary circuit
    # track the norm and each pass undoes the previous pass's drift as it loads,
    # so only the last pass's drift remains and the norm holds to the CUDA-core
    # path's bar.
    assert abs(norm2 - 1) < 1e-5, norm2
    s.close()


def test_tc_non_unitary_matrix_not_renormalised(sv):
    # A UNITARY gate whose matrix is not unitary (here 0.9 x a unitary) changes
    # the norm; a pass holding it must not have its tile norms restored, so the
    # result follows the oracle's exact action, norm included.
    n = 14
    rng = np.random.default_rng(5)
    z = rng.standard_normal((8, 8)) + 1j * rng.standard_normal((8, 8))
    u, _ = np.linalg.qr(z)
    circ = W.random_layered(n, 6, 31)
    circ.insert(len(circ) // 2, ("unitary", (1, 6, 9), (0.9 * u,)))
    ref = oracle.run(n, circ)
    g = _run(sv, n, circ, k_max=4, tile_qubits=12)
    assert abs(oracle.norm2(g) - 0.81) < 1e-5
    _compare(g, ref, "0.9 x unitary")


def test_tc_norm_tracking_keeps_input_norm(sv):
    # The passes of a unitary circuit undo each pass's norm drift against the
    # norm the circuit started from, which need not be 1: a state of norm^2
    # 0.64 keeps 0.64 (relative 1e-5) through ~40 tensor-core passes, and the
    # amplitudes still match the oracle's exact unitary action.
    n = 18
    rng = np.random.default_rng(9)
    psi0 = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    psi0 = (0.8 * psi0 / np.linalg.norm(psi0)).astype(np.complex64)
    circ = W.random_layered(n, 40, 17)
    info = sv.capi.sv_plan_stats(n, circ, sv.capi.make_opts(4, 11, 5, 2))
    assert info["passes_by_kind"][2] >= 20
    g = _run(sv, n, circ, psi0=psi0, k_max=4, tile_qubits=11)
    n0 = oracle.norm2(psi0.astype(np.complex128))
    assert abs(oracle.norm2(g) / n0 - 1) < 1e-5, (oracle.norm2(g), n0)
    ref = oracle.run(n, circ, psi0.astype(np.complex128))
    err = float(np.max(np.abs(g - ref)))
    assert err <= AMP_TOL, err


def test_tc_product_r5_matches_fp64(sv):
    # the 5-qubit stage product: 128 x 64 times 64 x 64 (16 MMAs of N = 128 and 64)
    rng = np.random.default_rng(3)
    for scale in (1.0, 1e-3):
        a = (rng.standard_normal((128, 64)) * scale).astype(np.float32)
        b = rng.standard_normal((64, 64))
        d = sv.capi.sv_tc_selftest_r(5, a, b)
        want = a.astype(np.float64) @ b.T
        bound = np.abs(a.astype(np.float64)) @ np.abs(b).T
        err = np.abs(d - want)
        assert np.all(err <= 2e-6 * bound + 1e-30), float(np.max(err / bound))
    # r = 4 through the same entry point equals sv_tc_selftest
    a4 = rng.standard_normal((128, 32)).astype(np.float32)
    b4 = rng.standard_normal((32, 32))
    assert np.array_equal(sv.capi.sv_tc_selftest_r(4, a4, b4), sv.capi.sv_tc_selftest(a4, b4))


@pytest.mark.parametrize("T", [12, 13])
def test_tc_five_qubit_stages(sv, T):
    # kernel variant 2: blocks fused up to 5 qubits and 5-qubit stages (32 x 32
    # complex products) on every tensor-core pass that fits
    n = 16
    circ = W.random_layered(n, 12, 23)
    info = sv.capi.sv_plan_stats(n, circ, sv.capi.make_opts(5, T, 5, 2, 2))
    assert info["tc_stages"] > 0 and info["hist_k"][5] > 0
    _compare(_run(sv, n, circ, k_max=5, tile_qubits=T, kernel_variant=2), oracle.run(n, circ), f"R=5 T={T}")


@pytest.mark.parametrize("depth", [1, 2])
def test_tc_five_qubit_unitaries(sv, depth):
    # 5-qubit UNITARY gates: a pass holding such a block takes 5-qubit
    # tensor-core stages when its records fit (at most four 32 KB stage
    # images), else the shared-memory kernel; depth 1 plans both passes as
    # 5-qubit tensor-core passes, depth 2 one of each
    n = 14
    rng = np.random.default_rng(8)
    circ = W.random_layered(n, depth, 41)
    for _ in range(2):
        qs = tuple(int(x) for x in rng.choice(n, 5, replace=False))
        z = rng.standard_normal((32, 32)) + 1j * rng.standard_normal((32, 32))
        u, _ = np.linalg.qr(z)
        circ.insert(int(rng.integers(0, len(circ) + 1)), ("unitary", qs, (u,)))
    info = sv.capi.sv_plan_stats(n, circ, sv.capi.make_opts(4, 12, 5, 2))
    assert info["tc_stages"] > 0 and info["hist_k"][5] == 2
    _compare(_run(sv, n, circ, k_max=4, tile_qubits=12), oracle.run(n, circ), "5-qubit unitaries")


def test_mixed_precision_plan(sv):
    # precision 1: the planner puts light passes (one- and two-qubit blocks, no
    # phase ops) on the CUDA-core register kernel and the rest on the tensor
    # cores; the mixed plan tracks the norm across its tensor-core passes only
    n = 20
    circ = W.random_layered(n, 40, 3) + W.qft(n)
    info = sv.capi.sv_plan_stats(n, circ, sv.capi.make_opts(5, 12, 5, 1))
    assert info["passes_by_kind"][1] > 0 and info["passes_by_kind"][2] > 0, info["passes_by_kind"]
    g = _run(sv, n, circ, precision=1, k_max=5, tile_qubits=12)
    _compare(g, oracle.run(n, circ), "mixed n=20")
    assert abs(oracle.norm2(g) - 1) < 1e-5
