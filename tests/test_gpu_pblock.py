"""Partitioned blocks through the C-ABI against the oracle (§II p-block
simulation, §III-E): registers simulated apart, merged on their first
interaction, and communication qubits taken out after measurement, give the
monolithic result (per amplitude within 1e-5, fidelity >= 1 - 1e-6)."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
AMP_TOL, FID_TOL = 1e-5, 1e-6


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    import paper_2512_04216_gb300 as P
    return P


def _check(gpu, ref, what):
    gpu = gpu.astype(np.complex128)
    err = float(np.max(np.abs(gpu - ref)))
    assert err <= AMP_TOL, f"{what}: max abs err {err:.3e}"
    assert oracle.fidelity(ref, gpu) >= 1 - FID_TOL, what


def _shift(circ, k):
    return [(g, tuple(q + k for q in qs), p) for g, qs, p in circ]


@pytest.mark.parametrize("na,nb", [(1, 1), (5, 7), (13, 9)])
def test_merge_matches_oracle_and_monolithic(P, na, nb):
    ca, cb = W.random_layered(na, 4, 60 + na), W.random_layered(nb, 4, 70 + nb)
    a, b = P.StateVector(na), P.StateVector(nb)
    a.apply(ca)
    b.apply(cb)
    m = a.merge(b)
    ref = oracle.kron(oracle.run(na, ca), oracle.run(nb, cb))
    _check(m.amplitudes(), ref, f"merge {na}+{nb}")
    # cross gates after the merge equal the monolithic circuit
    cross = [("cx", (0, na), ()), ("cp", (na - 1, na + nb - 1), (0.7,)), ("u3", (na,), (0.3, 0.2, 0.1))]
    m.apply(cross)
    mono = oracle.run(na + nb, ca + _shift(cb, na) + cross)
    _check(m.amplitudes(), mono, f"merged + cross gates {na}+{nb}")
    for s in (a, b, m):
        s.close()


def test_take_qubit(P):
    n = 12
    s = P.StateVector(n)
    s.apply(W.random_layered(n, 5, 9))
    b, _ = s.measure(4, 0.3)
    psi = s.amplitudes().astype(np.complex128)
    t, v = s.take_qubit(4)
    assert v == b
    _check(t.amplitudes(), oracle.take_qubit(psi, 4, v), "take after measurement")
    with pytest.raises(P.capi.SvError):
        s2 = P.StateVector(3)
        s2.apply([("h", (1,), ())])
        try:
            s2.take_qubit(1)
        finally:
            s2.close()
    t.close()
    s.close()


def test_teleportation_between_registers(P):
    """Two 6-qubit hosts, each with one communication qubit: merge the hosts,
    teleport host A's data qubit 0 onto host B's qubit 5 through the
    communication pair, then drop both communication qubits -- against the
    same gates on one monolithic 12-qubit oracle state."""
    na = nb = 6
    ca, cb = W.random_layered(na - 1, 3, 81), W.random_layered(nb - 1, 3, 82)
    # host A: qubits 0..4 data, 5 communication; host B: 6..10 data, 11 communication
    a, b = P.StateVector(na), P.StateVector(nb)
    a.apply(ca)
    b.apply(cb)
    m = a.merge(b)
    ent = [("h", (5,), ()), ("cx", (5, 11), ())]
    tele = [("cx", (0, 5), ()), ("h", (0,), ())]
    m.apply(ent + tele)
    mono = oracle.run(12, ca + _shift(cb, 6) + ent + tele)
    _check(m.amplitudes(), mono, "before measurement")
    u0, u5 = 0.31, 0.77
    b0, _ = m.measure(0, u0)
    b5, _ = m.measure(5, u5)
    o0, _, mono = oracle.measure(mono, 0, u0)
    o5, _, mono = oracle.measure(mono, 5, u5)
    assert (b0, b5) == (o0, o5)
    fix = ([("x", (11,), ())] if b5 else []) + ([("z", (11,), ())] if b0 else [])
    m.apply(fix)
    mono = oracle.run(12, fix, mono)
    # communication qubits leave: qubit 5 first, then qubit 0
    m2, v5 = m.take_qubit(5)
    m3, v0 = m2.take_qubit(0)
    assert (v0, v5) == (b0, b5)
    ref = oracle.take_qubit(oracle.take_qubit(mono, 5, v5), 0, v0)
    _check(m3.amplitudes(), ref, "after teleportation and removal")
    for s in (a, b, m, m2, m3):
        s.close()


def test_merge_large(P):
    """14 + 14 qubits -> 28 (2 GiB): spot amplitudes against the factors."""
    a, b = P.StateVector(14), P.StateVector(14)
    a.apply(W.random_layered(14, 3, 1))
    b.apply(W.random_layered(14, 3, 2))
    A, B = a.amplitudes().astype(np.complex128), b.amplitudes().astype(np.complex128)
    m = a.merge(b)
    rng = np.random.default_rng(0)
    for i in rng.integers(0, 1 << 28, 64):
        i = int(i)
        got = complex(m.amplitudes(i, 1)[0])
        want = B[i >> 14] * A[i & ((1 << 14) - 1)]
        assert abs(got - want) < 1e-7
    assert abs(m.norm2() - 1.0) < 1e-5
    for s in (a, b, m):
        s.close()
