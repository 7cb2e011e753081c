"""Pauli-string expectations on the GPU (sv_expect_pauli with X, Y and Z
components) against the oracle's plain definition, <psi|P psi> / <psi|psi>
with P built qubit by qubit, on the GPU's own complex64 state: the one-read
pair reduction (exact float32 products, compensated sums, double across
threads) agrees within 1e-12."""
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


def _masks(n, rng, count):
    full = (1 << n) - 1
    out = [(1, 0), (1, 1), (full, 0), (full, full), (1 << (n - 1), 1 << (n - 1))]
    for _ in range(count):
        out.append((int(rng.integers(1, 1 << n)), int(rng.integers(0, 1 << n))))
    return [(x & full, z & full) for x, z in out]


@pytest.mark.parametrize("n", [1, 2, 5, 9, 13, 17])
def test_pauli_random_states(P, n):
    rng = np.random.default_rng(100 + n)
    psi = (rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)) * 0.3
    s = P.StateVector(n)
    s.set_amplitudes(psi.astype(np.complex64))
    g = s.amplitudes().astype(np.complex128)
    for x, z in _masks(n, rng, 10):
        want = oracle.expect_pauli(g, x, z)
        got = P.capi.sv_expect_pauli(s.h, x, z)
        assert abs(got - want.real) <= 1e-12, (n, x, z, got, want)
    s.close()


@pytest.mark.parametrize("n", [12, 20])
def test_pauli_circuit_states(P, n):
    rng = np.random.default_rng(7 + n)
    s = P.StateVector(n)
    s.apply(W.random_layered(n, 8, 30 + n))
    g = s.amplitudes().astype(np.complex128)
    for x, z in _masks(n, rng, 6):
        want = oracle.expect_pauli(g, x, z)
        got = P.capi.sv_expect_pauli(s.h, x, z)
        assert abs(got - want.real) <= 1e-12, (n, x, z, got, want)
    s.close()


def test_pauli_closed_forms(P):
    # GHZ_n: <X...X> = 1, <Y Y X...X> = -1, <X on one qubit> = 0; Bell <YY> = -1
    n = 16
    s = P.StateVector(n)
    s.apply(W.ghz(n))
    full = (1 << n) - 1
    assert abs(P.capi.sv_expect_pauli(s.h, full, 0) - 1) < 1e-6
    assert abs(P.capi.sv_expect_pauli(s.h, full, 3) + 1) < 1e-6
    assert abs(P.capi.sv_expect_pauli(s.h, 1 << 7, 0)) < 1e-6
    s.close()
    b = P.StateVector(2)
    b.apply([("h", (0,), ()), ("cx", (0, 1), ())])
    assert abs(P.capi.sv_expect_pauli(b.h, 3, 3) + 1) < 1e-6
    assert abs(P.capi.sv_expect_pauli(b.h, 3, 0) - 1) < 1e-6
    b.close()
