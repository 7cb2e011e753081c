"""CUDA path vs the complex128 oracle, through the C-ABI (GPU required).

Tolerances (complex64 state, float32 arithmetic in the kernels):
  per-amplitude |a_gpu - a_oracle| <= 1e-5 and fidelity >= 1 - 1e-6;
  sampled bitstrings identical to the oracle's draws on the same state except
  draws within 1e-9 of a CDF boundary (counted); norms and expectations of the
  same complex64 state agree with the oracle's double sums to 1e-12.
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
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2512_04216_gb300 as P
    return P


def _run_gpu(P, n, circ, psi0=None, **opts):
    s = P.StateVector(n)
    if psi0 is not None:
        s.set_amplitudes(psi0)
    s.apply(circ, **opts)
    out = s.amplitudes().astype(np.complex128)
    return s, out


def _compare(gpu, ref, what=""):
    err = float(np.max(np.abs(gpu - ref)))
    fid = oracle.fidelity(ref, gpu)
    assert err <= AMP_TOL, f"{what}: max abs err {err:.3e}"
    assert fid >= 1 - FID_TOL, f"{what}: fidelity {fid!r}"
    return err, fid


def test_small_random_layered_default(sv):
    n, d = 12, 20
    c = W.random_layered(n, d, 1)
    s, g = _run_gpu(sv, n, c)
    _compare(g, oracle.run(n, c), "n=12 d=20")
    s.close()


@pytest.mark.parametrize("variant", [0, 1, 2])
@pytest.mark.parametrize("k_max", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("T,c", [(6, 1), (8, 3), (9, 5), (10, 5), (12, 5), (13, 4), (13, 5)])
def test_random_layered_plans(sv, k_max, T, c, variant):
    n, d = 15, 12
    circ = W.random_layered(n, d, 7)
    s, g = _run_gpu(sv, n, circ, k_max=k_max, tile_qubits=T, low_qubits=c, kernel_variant=variant)
    _compare(g, oracle.run(n, circ), f"k={k_max} T={T} c={c} variant={variant}")
    s.close()


@pytest.mark.parametrize("n", [1, 2, 3, 5, 6, 8, 11, 13, 15])
def test_gate_soup_every_kind(sv, n):
    rng = np.random.default_rng(n)
    circ = W.random_gate_soup(n, 150, seed=300 + n)
    for k in range(3, min(n, 5) + 1):
        qs = tuple(int(q) for q in rng.choice(n, size=k, replace=False))
        a = rng.standard_normal((1 << k, 1 << k)) + 1j * rng.standard_normal((1 << k, 1 << k))
        u, _ = np.linalg.qr(a)
        circ.insert(len(circ) // 2, ("unitary", qs, (u,)))
    psi0 = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    psi0 /= np.linalg.norm(psi0)
    for opts in [dict(), dict(kernel_variant=1), dict(k_max=4, tile_qubits=min(n, 11), low_qubits=3),
                 dict(k_max=5, tile_qubits=min(n, 10), low_qubits=1),
                 dict(k_max=1, tile_qubits=min(n, 7), low_qubits=2)]:
        s, g = _run_gpu(sv, n, circ, psi0.astype(np.complex64), **opts)
        ref = oracle.run(n, circ, psi0.astype(np.complex64).astype(np.complex128))
        _compare(g, ref, f"soup n={n} {opts}")
        s.close()


def test_diagonal_gates_outside_tile(sv):
    # controlled phases whose qubits leave the tile become per-tile phase ops
    n = 16
    rng = np.random.default_rng(3)
    circ = [("h", (q,), ()) for q in range(n)]
    for _ in range(200):
        a, b = (int(x) for x in rng.choice(n, 2, replace=False))
        kind = ["cp", "cz", "rz", "p", "t", "sdg", "z"][int(rng.integers(7))]
        if kind in ("cp",):
            circ.append((kind, (a, b), (float(rng.uniform(-4, 4)),)))
        elif kind == "cz":
            circ.append((kind, (a, b), ()))
        elif kind in ("rz", "p"):
            circ.append((kind, (a,), (float(rng.uniform(-4, 4)),)))
        else:
            circ.append((kind, (a,), ()))
    circ += [("u3", (q,), (0.3 * q, 0.1, -0.2)) for q in range(n)]
    for opts in (dict(tile_qubits=8, low_qubits=3), dict(tile_qubits=12), dict(tile_qubits=10, k_max=3)):
        s, g = _run_gpu(sv, n, circ, **opts)
        _compare(g, oracle.run(n, circ), f"diagonal {opts}")
        s.close()


@pytest.mark.parametrize("n", [11, 15])
def test_interleaved_diagonals(sv, n):
    """Diagonal gates on two tile qubits between dense gates (the QFT pattern):
    register-stage passes turn them into phase ops whose terms split by the
    stage's register bits; every kernel path must agree with the oracle."""
    rng = np.random.default_rng(40 + n)
    circ = []
    for _ in range(8):
        for q in rng.choice(n, 3, replace=False):
            circ.append(("u3", (int(q),), tuple(float(x) for x in rng.uniform(-3, 3, 3))))
        for _ in range(24):
            a, b = (int(x) for x in rng.choice(n, 2, replace=False))
            kind = ["cp", "cz", "rz", "p", "t", "s", "cx", "h"][int(rng.integers(8))]
            if kind == "cp":
                circ.append((kind, (a, b), (float(rng.uniform(-4, 4)),)))
            elif kind in ("cz", "cx"):
                circ.append((kind, (a, b), ()))
            elif kind in ("rz", "p"):
                circ.append((kind, (a,), (float(rng.uniform(-4, 4)),)))
            else:
                circ.append((kind, (a,), ()))
    ref = oracle.run(n, circ)
    for opts in (dict(), dict(kernel_variant=2), dict(tile_qubits=13),
                 dict(tile_qubits=9, low_qubits=4), dict(tile_qubits=13, k_max=1),
                 dict(tile_qubits=10, k_max=3), dict(tile_qubits=12, k_max=4),
                 dict(tile_qubits=11, precision=1), dict(tile_qubits=13, precision=1, k_max=2),
                 dict(kernel_variant=1)):
        s, g = _run_gpu(sv, n, circ, **opts)
        _compare(g, ref, f"interleaved n={n} {opts}")
        s.close()


def test_ghz_and_qft_closed_forms(sv):
    n = 14
    s, g = _run_gpu(sv, n, W.ghz(n))
    want = np.zeros(1 << n)
    want[0] = want[-1] = 1 / math.sqrt(2)
    _compare(g, want, "GHZ")
    s.close()
    for n in (10, 16):
        x = W.basis_index(n, 99)
        s = sv.StateVector(n, basis_index=x)
        s.apply(W.qft(n))
        g = s.amplitudes().astype(np.complex128)
        y = np.arange(1 << n)
        _compare(g, np.exp(2j * np.pi * ((x * y) % (1 << n)) / (1 << n)) / math.sqrt(1 << n), f"QFT {n}")
        s.close()


def test_norm_expect_probabilities(sv):
    n = 13
    c = W.random_layered(n, 10, 5)
    s, g = _run_gpu(sv, n, c)
    assert abs(s.norm2() - oracle.norm2(g)) < 1e-12
    for m in (1, 6, (1 << n) - 1, 0b1010101):
        assert abs(s.expect_z(m) - oracle.expect_z(g, m)) < 1e-12
    p = s.probabilities()
    assert np.array_equal(p, np.abs(g) ** 2) or np.max(np.abs(p - np.abs(g) ** 2)) < 1e-18
    p2 = s.probabilities(offset=100, count=37)
    assert np.allclose(p2, p[100:137], rtol=0, atol=0)
    s.close()


@pytest.mark.parametrize("n", [3, 6, 12, 13, 17])
def test_sampler_parity(sv, n):
    c = W.random_layered(n, 8, 11 + n)
    s, g = _run_gpu(sv, n, c)
    u = W.shot_uniforms(1234 + n, 4096)
    x_gpu, nb_gpu = s.sample_uniforms(u)
    # (i) oracle sampler on the GPU's own final state: identical except boundary draws
    x_or, bnd, nb_or = oracle.sample(g, u)
    diff = x_gpu.astype(np.int64) != x_or.astype(np.int64)
    assert np.all(bnd[diff] == 1), f"{int(diff.sum())} mismatches, boundary {nb_or}"
    # (ii) against the oracle's own complex128 state: mismatches only within delta
    ref = oracle.run(n, c)
    C_gpu, C_ref = oracle.cdf(g), oracle.cdf(ref)
    delta = float(np.max(np.abs(C_gpu - C_ref))) + 1e-9
    _, _, _ = oracle.sample_cdf(C_ref, u, eps=delta)
    x_ref, bnd_ref, _ = oracle.sample_cdf(C_ref, u, eps=delta)
    diff2 = x_gpu.astype(np.int64) != x_ref.astype(np.int64)
    assert np.all(bnd_ref[diff2] == 1), f"{int(diff2.sum())} mismatches beyond delta={delta:.2e}"
    s.close()


def test_sample_seed_matches_uniforms(sv):
    n = 11
    s, g = _run_gpu(sv, n, W.random_layered(n, 6, 4))
    x_seed = s.sample(3000, seed=77)
    x_u, _ = s.sample_uniforms(W.shot_uniforms(77, 3000))
    assert np.array_equal(x_seed, x_u)
    s.close()


def test_sampler_edge_states(sv):
    n = 9
    for idx in (0, 5, (1 << n) - 1):
        s = sv.StateVector(n, basis_index=idx)
        x, nb = s.sample_uniforms(W.shot_uniforms(3, 500))
        assert np.all(x == idx)
        s.close()
    s = sv.StateVector(n)
    s.apply(W.ghz(n))
    x, _ = s.sample_uniforms(W.shot_uniforms(4, 20000))
    assert set(np.unique(x).tolist()) <= {0, (1 << n) - 1}
    assert abs(np.mean(x == 0) - 0.5) < 0.02
    # zero shots, hand-worked fixture (index 1 has zero probability)
    assert s.sample_uniforms(np.zeros(0))[0].shape == (0,)
    s.close()
    s = sv.StateVector(2)
    s.set_amplitudes(np.array([0.5, 0, 0.5, math.sqrt(0.5)], dtype=np.complex64))
    from tests.oracle_pins import load_sampler_golden
    amps, rows = load_sampler_golden()
    x, _ = s.sample_uniforms(np.array([r[0] for r in rows]))
    x_or, b_or, _ = oracle.sample(s.amplitudes().astype(np.complex128), np.array([r[0] for r in rows]))
    ok = (x.astype(np.int64) == x_or.astype(np.int64)) | (b_or == 1)
    assert np.all(ok)
    assert 1 not in x.tolist()
    s.close()


def test_invalid_ir_leaves_state_usable(sv):
    n = 6
    s = sv.StateVector(n)
    with pytest.raises(sv.capi.SvError) as e:
        s.apply([("h", (0,), ()), ("cx", (0, 9), ())])
    assert e.value.code == sv.capi.SV_ERR_ARG
    s.apply(W.ghz(n))
    g = s.amplitudes()
    assert abs(abs(g[0]) ** 2 - 0.5) < 1e-6
    with pytest.raises(sv.capi.SvError):
        s.expect_z(1 << n)
    s.close()


def test_many_states_on_streams(sv):
    import torch
    states = []
    circs = []
    for i in range(6):
        st = torch.cuda.Stream()
        n = 8 + 2 * i
        s = sv.StateVector(n, stream=st)
        c = W.random_layered(n, 6, 50 + i)
        s.apply(c)
        states.append(s)
        circs.append((n, c))
    for s, (n, c) in zip(states, circs):
        _compare(s.amplitudes().astype(np.complex128), oracle.run(n, c), f"stream n={n}")
        s.close()


def test_large_mirror_and_qft_28(sv):
    """28 qubits (2 GiB), in the plan options the benchmark times (k_max 5,
    12 tile qubits, 5 low qubits, register kernels): C.C^-1 returns |0> and the
    QFT of a basis state matches its closed form on sampled indices."""
    n = 28
    opts = dict(k_max=5, tile_qubits=12, low_qubits=5, kernel_variant=0, precision=0)
    c = W.random_layered(n, 40, 2)
    s = sv.StateVector(n)
    s.apply(c + W.inverse(c), **opts)
    a0 = s.amplitudes(0, 1)[0]
    norm2 = s.norm2()
    assert abs(a0) ** 2 / norm2 >= 1 - FID_TOL, (abs(a0) ** 2, norm2)
    assert abs(norm2 - 1) < 1e-5, norm2
    x = W.basis_index(n, 2)
    s.reset(x)
    s.apply(W.qft(n), **opts)
    rng = np.random.default_rng(0)
    idx = np.unique(rng.integers(0, 1 << n, 1 << 14))
    amps = s.amplitudes()
    y = idx.astype(np.int64)
    want = np.exp(2j * np.pi * ((x * y) % (1 << n)) / (1 << n)) / math.sqrt(1 << n)
    assert np.max(np.abs(amps[idx] - want)) < 1e-6
    s.close()


@pytest.mark.parametrize("n", [3, 12, 17, 24])
def test_fused_readout_matches_separate_calls_and_oracle(sv, n):
    # sv_sample_expect_z: the draws of sv_sample_uniforms, and <Z_mask> and the
    # norm from the same read of the state, against the oracle's double sums.
    c = W.random_layered(n, 8, 40 + n)
    s, g = _run_gpu(sv, n, c)
    u = W.shot_uniforms(50 + n, 4096)
    x1, nb1 = s.sample_uniforms(u)
    for mask in (0, 1, (1 << n) - 1, 0b1011 & ((1 << n) - 1)):
        x2, nb2, e, n2 = s.sample_expect_z(u, mask)
        assert np.array_equal(x1, x2) and nb1 == nb2
        assert abs(e - oracle.expect_z(g, mask)) < 1e-12, (n, mask)
        assert abs(n2 - oracle.norm2(g)) < 1e-12
        assert abs(n2 - s.norm2()) < 1e-12
    assert abs(s.expect_z(0) - 1.0) < 1e-12  # Z_0 is the identity
    _, nb0, e0, n0 = s.sample_expect_z(np.empty(0), 0b11 & ((1 << n) - 1))  # readout only
    assert nb0 == 0 and abs(e0 - oracle.expect_z(g, 0b11 & ((1 << n) - 1))) < 1e-12
    with pytest.raises(sv.capi.SvError):
        s.sample_expect_z(u, 1 << n)
    s.close()
