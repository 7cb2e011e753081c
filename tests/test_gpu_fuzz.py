"""Randomised parity: seeded gate soups (every IR kind, 3-5-qubit unitaries,
swaps and diagonal gates between dense gates) under randomly drawn plan options
(tile size, low qubits, fusion width, kernel variant, precision) against the
complex128 oracle, per amplitude within 1e-5 and fidelity >= 1 - 1e-6."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    import paper_2512_04216_gb300 as P
    return P


def _case(seed):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(6, 15))
    circ = W.random_gate_soup(n, int(rng.integers(40, 220)), 2000 + seed)
    for _ in range(int(rng.integers(0, 3))):
        k = int(rng.integers(3, min(n, 5) + 1))
        qs = tuple(int(q) for q in rng.choice(n, size=k, replace=False))
        a = rng.standard_normal((1 << k, 1 << k)) + 1j * rng.standard_normal((1 << k, 1 << k))
        u, _ = np.linalg.qr(a)
        circ.insert(int(rng.integers(0, len(circ) + 1)), ("unitary", qs, (u,)))
    T = int(rng.integers(min(n, 7), min(n, 13) + 1))
    opts = dict(tile_qubits=T, low_qubits=int(rng.integers(1, min(T, 5) + 1)),
                k_max=int(rng.integers(1, 6)), kernel_variant=int(rng.integers(0, 3)),
                precision=(1 + seed % 2) if rng.random() < 0.3 else 0)
    return n, circ, opts


@pytest.mark.parametrize("seed", range(40))
def test_fuzz(P, seed):
    n, circ, opts = _case(seed)
    rng = np.random.default_rng(seed)
    psi0 = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    psi0 = (psi0 / np.linalg.norm(psi0)).astype(np.complex64)
    s = P.StateVector(n)
    try:
        s.set_amplitudes(psi0)
        try:
            s.apply(circ, **opts)
        except P.capi.SvError as e:
            # only option combinations the planner documents as invalid may be refused
            assert "too small" in str(e), (opts, str(e))
            return
        got = s.amplitudes().astype(np.complex128)
    finally:
        s.close()
    ref = oracle.run(n, circ, psi0.astype(np.complex128))
    err = float(np.max(np.abs(got - ref)))
    assert err <= 1e-5, (seed, n, opts, err)
    assert oracle.fidelity(ref, got) >= 1 - 1e-6, (seed, n, opts)
