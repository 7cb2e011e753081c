"""Pins for the oracle: checks against what the mathematics fixes, not against
the oracle itself.  Each ``pin_*`` takes an ``oracle.Oracle`` and raises
AssertionError on a mismatch, so the same pins run on the real oracle
(test_oracle_pins.py) and on deliberately broken copies of it
(test_oracle_mutants.py).

Sources of truth used here:
* textbook gate identities and special cases (OpenQASM 2 definitions; the paper
  ingests OpenQASM 2 / Qiskit circuits, §III-A);
* Kronecker-product brute force: every gate's full 2^n x 2^n unitary is built
  from np.kron with identities and adjacent-qubit SWAP conjugations;
* closed forms: GHZ state, QFT of a basis state (and the explicit DFT matrix /
  numpy's inverse FFT for n <= 10);
* invariants: norm preservation, circuit * inverse = |0...0> (the paper's
  mirror-circuit check, §IV-A);
* sampling (§III-B) and expectation values from the final state (§III-B):
  a hand-worked fixture, basis states, GHZ, np.searchsorted(side="right") as
  the library special case of "first index with C_i > t", exact ⟨Z⟩ closed forms.
"""
from __future__ import annotations

import math
from fractions import Fraction
import os

import numpy as np

import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

I2 = np.eye(2, dtype=np.complex128)
X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
H = np.array([[1, 1], [1, -1]], dtype=np.complex128) / math.sqrt(2.0)
S = np.array([[1, 0], [0, 1j]], dtype=np.complex128)
T = np.array([[1, 0], [0, (1 + 1j) / math.sqrt(2.0)]], dtype=np.complex128)
SWAP2 = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=np.complex128)


def _close(a, b, tol=1e-12, what=""):
    a = np.asarray(a)
    b = np.asarray(b)
    err = float(np.max(np.abs(a - b))) if a.size else 0.0
    assert err <= tol, f"{what}: max abs err {err:.3e} > {tol:.1e}"


# ---------------------------------------------------------------------------
# Kronecker-product brute force (independent of the oracle's gather/scatter)
# ---------------------------------------------------------------------------

def _kron_all(mats):
    out = np.ones((1, 1), dtype=np.complex128)
    for m in mats:
        out = np.kron(out, m)
    return out


def _adjacent_swap(n, q):
    """Full unitary swapping qubits q and q+1 (qubit 0 = least significant)."""
    # kron order lists the most significant qubit first.
    mats = []
    q_hi = n - 1
    while q_hi >= 0:
        if q_hi == q + 1:
            mats.append(SWAP2)
            q_hi -= 2
        else:
            mats.append(I2)
            q_hi -= 1
    return _kron_all(mats)


def _low_embed(n, M):
    """I ⊗ M with M acting on the k lowest qubits (matrix bit m = qubit m)."""
    k = int(M.shape[0]).bit_length() - 1
    return np.kron(np.eye(1 << (n - k), dtype=np.complex128), M)


def kron_full(n, targets, M):
    """Full 2^n unitary of M on `targets` (t_0 = least significant matrix bit).

    Conjugate the low-embedded M by a product of adjacent swaps that carries
    qubit t_m to position m for every m.
    """
    order = list(range(n))  # order[pos] = logical qubit currently at pos
    P = np.eye(1 << n, dtype=np.complex128)
    for m, t in enumerate(targets):
        pos = order.index(t)
        while pos > m:
            P = _adjacent_swap(n, pos - 1) @ P
            order[pos - 1], order[pos] = order[pos], order[pos - 1]
            pos -= 1
    return P.conj().T @ _low_embed(n, M) @ P


def _textbook_matrix(name, params):
    """Gate matrices from identities of the textbook gates, not from the u3 formula."""
    if name == "h":
        return H
    if name == "x":
        return X
    if name == "y":
        return Y
    if name == "z":
        return Z
    if name == "s":
        return S
    if name == "sdg":
        return S.conj().T
    if name == "t":
        return T
    if name == "tdg":
        return T.conj().T
    if name == "rx":
        return _expm_pauli(X, params[0])
    if name == "ry":
        return _expm_pauli(Y, params[0])
    if name == "rz":
        return _expm_pauli(Z, params[0])
    if name == "p":
        return np.diag([1.0, np.exp(1j * params[0])])
    if name == "u3":
        # U3(θ,φ,λ) = e^{i(φ+λ)/2} RZ(φ) RY(θ) RZ(λ)
        th, ph, la = params
        return np.exp(0.5j * (ph + la)) * (_expm_pauli(Z, ph) @ _expm_pauli(Y, th) @ _expm_pauli(Z, la))
    if name == "cx":   # control = matrix bit 0, target = matrix bit 1
        P0 = np.diag([1.0, 0.0]).astype(np.complex128)
        P1 = np.diag([0.0, 1.0]).astype(np.complex128)
        return np.kron(I2, P0) + np.kron(X, P1)
    if name == "cz":
        return np.diag([1, 1, 1, -1]).astype(np.complex128)
    if name == "cp":
        return np.diag([1, 1, 1, np.exp(1j * params[0])])
    if name == "swap":
        return SWAP2
    if name == "unitary":
        return params[0]
    raise KeyError(name)


def _expm_pauli(P, theta):
    """exp(-i θ P / 2) for a Pauli P (P^2 = I)."""
    return math.cos(theta / 2) * I2 - 1j * math.sin(theta / 2) * P


def random_unitary(k, rng):
    a = rng.standard_normal((1 << k, 1 << k)) + 1j * rng.standard_normal((1 << k, 1 << k))
    q, r = np.linalg.qr(a)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def random_state(n, rng):
    v = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    return v / np.linalg.norm(v)


# ---------------------------------------------------------------------------
# pins
# ---------------------------------------------------------------------------

def pin_gate_identities(o):
    """Every gate kind equals its textbook matrix; u3 special cases."""
    rng = np.random.default_rng(11)
    _close(o.gate_matrix("u3", (0,), (math.pi, 0.0, math.pi)), X, what="U3(π,0,π)=X")
    _close(o.gate_matrix("u3", (0,), (math.pi / 2, 0.0, math.pi)), H, what="U3(π/2,0,π)=H")
    for _ in range(5):
        th, ph, la = rng.uniform(-math.pi, math.pi, 3)
        _close(o.gate_matrix("u3", (0,), (th, ph, la)), _textbook_matrix("u3", (th, ph, la)),
               what="U3 vs e^{i(φ+λ)/2} RZ RY RZ")
        _close(o.gate_matrix("rx", (0,), (th,)), _expm_pauli(X, th), what="RX")
        _close(o.gate_matrix("ry", (0,), (th,)), _expm_pauli(Y, th), what="RY")
        _close(o.gate_matrix("rz", (0,), (th,)), _expm_pauli(Z, th), what="RZ")
        _close(o.gate_matrix("p", (0,), (th,)), np.diag([1, np.exp(1j * th)]), what="P")
        _close(o.gate_matrix("cp", (0, 1), (th,)), np.diag([1, 1, 1, np.exp(1j * th)]), what="CP")
    for name, M in [("h", H), ("x", X), ("y", Y), ("z", Z), ("s", S), ("t", T),
                    ("sdg", S.conj().T), ("tdg", T.conj().T), ("swap", SWAP2),
                    ("cz", np.diag([1, 1, 1, -1]))]:
        qs = (0, 1) if M.shape[0] == 4 else (0,)
        _close(o.gate_matrix(name, qs), M, what=name)
    _close(o.gate_matrix("h") @ o.gate_matrix("x") @ o.gate_matrix("h"), Z, what="HXH=Z")
    _close(o.gate_matrix("s") @ o.gate_matrix("s"), Z, what="S^2=Z")
    _close(o.gate_matrix("t") @ o.gate_matrix("t"), S, what="T^2=S")
    cx = o.gate_matrix("cx", (0, 1))
    _close(cx @ cx, np.eye(4), what="CX^2=I")
    _close(cx, _textbook_matrix("cx", ()), what="CX = I⊗|0><0| + X⊗|1><1|")


def pin_kron_bruteforce(o, n_max=7, gates_per=24):
    """Oracle output equals the product of Kronecker-built full unitaries (n<=8)."""
    rng = np.random.default_rng(5)
    for n in range(1, n_max + 1):
        circ = W.random_gate_soup(n, gates_per, seed=100 + n)
        if n >= 3:
            for _ in range(2):
                qs = tuple(int(q) for q in rng.choice(n, size=3, replace=False))
                circ.append(("unitary", qs, (random_unitary(3, rng),)))
        U = np.eye(1 << n, dtype=np.complex128)
        for name, qs, ps in circ:
            U = kron_full(n, qs, _textbook_matrix(name, ps)) @ U
        psi0 = random_state(n, rng)
        _close(o.run(n, circ, psi0), U @ psi0, tol=1e-11, what=f"kron n={n}")
        _close(o.run(n, circ), U[:, 0], tol=1e-11, what=f"kron |0> n={n}")


def pin_apply_matrix_k5(o):
    """A dense 5-qubit matrix on scattered targets matches the Kronecker build."""
    rng = np.random.default_rng(7)
    n = 7
    for targets in [(0, 1, 2, 3, 4), (6, 2, 0, 5, 3), (1, 6, 4, 2, 5)]:
        M = random_unitary(5, rng)
        psi = random_state(n, rng)
        _close(o.apply_matrix(psi, targets, M), kron_full(n, targets, M) @ psi, tol=1e-11,
               what=f"k=5 {targets}")


def pin_ghz(o):
    for n in range(1, 13):
        psi = o.run(n, W.ghz(n))
        want = np.zeros(1 << n, dtype=np.complex128)
        want[0] = want[-1] = 1 / math.sqrt(2.0)
        _close(psi, want, tol=1e-13, what=f"GHZ n={n}")


def pin_qft(o):
    """QFT|x> = 2^{-n/2} Σ_y e^{+2πi x y / 2^n}|y>: explicit DFT matrix (n<=8),
    numpy inverse FFT (n<=10), closed form (n<=14)."""
    for n in range(1, 15):
        N = 1 << n
        x = W.basis_index(n, 40 + n)
        psi = o.run(n, W.qft(n), _basis(n, x))
        y = np.arange(N)
        closed = np.exp(2j * math.pi * ((x * y) % N) / N) / math.sqrt(N)
        _close(psi, closed, tol=1e-11, what=f"QFT closed form n={n}")
        if n <= 10:
            e = np.zeros(N, dtype=np.complex128)
            e[x] = 1.0
            _close(psi, np.fft.ifft(e) * math.sqrt(N), tol=1e-11, what=f"QFT ifft n={n}")
        if n <= 8:
            F = np.exp(2j * math.pi * np.outer(y, y) / N) / math.sqrt(N)
            rng = np.random.default_rng(n)
            v = random_state(n, rng)
            _close(o.run(n, W.qft(n), v), F @ v, tol=1e-11, what=f"QFT DFT matrix n={n}")


def _basis(n, x):
    v = np.zeros(1 << n, dtype=np.complex128)
    v[x] = 1.0
    return v


def pin_norm_and_mirror(o):
    """Unitarity keeps ||psi|| = 1; C·C^-1|0> = |0> (mirror circuit, §IV-A)."""
    for n, d, seed in [(12, 20, 1), (9, 30, 2), (13, 8, 3)]:
        c = W.random_layered(n, d, seed)
        psi = o.run(n, c)
        assert abs(o.norm2(psi) - 1.0) < 1e-12, f"norm n={n}"
        assert abs(np.vdot(psi, psi).real - 1.0) < 1e-12
        back = o.run(n, W.inverse(c), psi)
        assert abs(back[0]) ** 2 > 1 - 1e-12, f"mirror n={n}: {abs(back[0])**2}"
        soup = W.random_gate_soup(n, 60, seed)
        back2 = o.run(n, soup + W.inverse(soup))
        assert abs(back2[0]) ** 2 > 1 - 1e-12, f"mirror soup n={n}"


def pin_norm_sum(o):
    rng = np.random.default_rng(3)
    v = rng.standard_normal(1000) + 1j * rng.standard_normal(1000)
    assert abs(o.norm2(v) - float(np.sum(np.abs(v) ** 2))) < 1e-9
    C = o.cdf(v)
    _close(C, np.cumsum(np.abs(v) ** 2), tol=1e-9, what="cdf")


def load_sampler_golden():
    amps, rows = None, []
    with open(os.path.join(GOLDEN, "sampler_cases.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            if parts[0] == "amplitudes":
                amps = np.array([float(v) for v in parts[1:]], dtype=np.complex128)
            else:
                rows.append((float(parts[0]), int(parts[1]), int(parts[2])))
    return amps, rows


def pin_sampler(o):
    amps, rows = load_sampler_golden()
    u = np.array([r[0] for r in rows])
    x, b, nb = o.sample(amps, u)
    assert [int(v) for v in x] == [r[1] for r in rows], f"golden x {x}"
    assert [int(v) for v in b] == [r[2] for r in rows], f"golden boundary {b}"
    # basis states: every draw returns the basis index
    for n, idx in [(3, 5), (6, 0), (6, 63), (8, 77)]:
        x, _, _ = o.sample(_basis(n, idx), W.shot_uniforms(9, 500))
        assert np.all(x == idx), f"basis {idx}"
    # first index with C_i > t, against numpy's searchsorted(side="right")
    rng = np.random.default_rng(21)
    for n in (1, 3, 6, 10):
        v = random_state(n, rng)
        v[rng.random(1 << n) < 0.3] = 0.0
        if not np.any(v):
            v[0] = 1.0
        u = W.shot_uniforms(31 + n, 3000)
        x, _, _ = o.sample(v, u)
        C = np.cumsum(np.abs(v) ** 2)
        want = np.minimum(np.searchsorted(C, u * C[-1], side="right"), len(C) - 1)
        assert np.array_equal(x.astype(np.int64), want), f"searchsorted n={n}"
        assert np.all(np.abs(v[x.astype(np.int64)]) > 0), "zero-probability index drawn"
    # GHZ: only 0 and 2^n-1, each near 1/2; Hellinger fidelity near 1 - N/(8S) (§IV-C)
    n, Sh = 6, 20000
    x, _, _ = o.sample(o.run(n, W.ghz(n)), W.shot_uniforms(77, Sh))
    assert set(np.unique(x).tolist()) <= {0, (1 << n) - 1}
    frac = float(np.mean(x == 0))
    assert abs(frac - 0.5) < 5 * math.sqrt(0.25 / Sh), f"GHZ freq {frac}"
    # chi-square against exact probabilities on a random 5-qubit state
    v = random_state(5, rng)
    p = np.abs(v) ** 2
    Sh = 40000
    x, _, _ = o.sample(v, W.shot_uniforms(5, Sh))
    cnt = np.bincount(x.astype(np.int64), minlength=32)
    chi2 = float(np.sum((cnt - Sh * p) ** 2 / (Sh * p)))
    assert chi2 < 31 + 6 * math.sqrt(62), f"chi2 {chi2}"
    hell = float(np.sum(np.sqrt(p * cnt / Sh))) ** 2
    assert hell > 1 - 32 / (8 * Sh) * 4, f"hellinger {hell}"


def pin_expectation(o):
    rng = np.random.default_rng(8)
    for _ in range(4):
        th, ph, la = rng.uniform(-math.pi, math.pi, 3)
        psi = o.run(1, [("u3", (0,), (th, ph, la))])
        assert abs(o.expect_z(psi, 1) - math.cos(th)) < 1e-12, "<Z> = cos θ"
    n = 7
    g = o.run(n, W.ghz(n))
    for m in range(1, 1 << n):
        want = 1.0 if bin(m).count("1") % 2 == 0 else 0.0
        assert abs(o.expect_z(g, m) - want) < 1e-12, f"GHZ <Z_{m}>"
    v = random_state(n, rng) * 1.7
    for m in (1, 5, 64, 127, 0):
        diag = _kron_all([np.diag([1.0, -1.0]) if (m >> q) & 1 else np.eye(2)
                          for q in range(n - 1, -1, -1)]).diagonal().real
        want = float(np.sum(np.abs(v) ** 2 * diag) / np.sum(np.abs(v) ** 2))
        assert abs(o.expect_z(v, m) - want) < 1e-12, f"kron <Z_{m}>"


def pin_expect_pauli(o):
    """<X^x Z^z> (Y where both masks hold the qubit) against eigenstates, Bell
    and GHZ closed forms, the Z-only routine, and Kronecker-built Pauli
    matrices with textbook X, Y, Z on random states."""
    s2 = 1 / math.sqrt(2)
    plus = np.array([s2, s2], dtype=np.complex128)
    minus = np.array([s2, -s2], dtype=np.complex128)
    plus_i = np.array([s2, 1j * s2], dtype=np.complex128)
    minus_i = np.array([s2, -1j * s2], dtype=np.complex128)
    for psi, x, z, want in ((plus, 1, 0, 1), (minus, 1, 0, -1), (plus_i, 1, 1, 1), (minus_i, 1, 1, -1),
                            (plus, 1, 1, 0), (plus_i, 1, 0, 0), (np.array([1, 0], np.complex128), 0, 1, 1),
                            (np.array([0, 1], np.complex128), 0, 1, -1), (np.array([1, 0], np.complex128), 1, 0, 0)):
        got = o.expect_pauli(psi, x, z)
        assert abs(got - want) < 1e-12, ("eigenstate", x, z, got)
    bell = o.run(2, [("h", (0,), ()), ("cx", (0, 1), ())])
    for x, z, want in ((3, 0, 1), (3, 3, -1), (0, 3, 1), (1, 0, 0), (3, 1, 0)):
        got = o.expect_pauli(bell, x, z)
        assert abs(got - want) < 1e-12, ("bell XX / YY / ZZ", x, z, got)
    n = 6
    g = o.run(n, W.ghz(n))
    assert abs(o.expect_pauli(g, (1 << n) - 1, 0) - 1) < 1e-12, "GHZ <X...X> = 1"
    # GHZ: <Y^{⊗2} X^{⊗(n-2)}> = -1 (two Y's: i^2 from Y = iXZ on the |1..1> branch)
    assert abs(o.expect_pauli(g, (1 << n) - 1, 3) + 1) < 1e-12, "GHZ <YYXXXX> = -1"
    rng = np.random.default_rng(12)
    X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
    Z = np.diag([1.0, -1.0]).astype(np.complex128)
    for n in (1, 3, 5):
        v = random_state(n, rng) * 0.7
        for _ in range(12):
            x, z = int(rng.integers(0, 1 << n)), int(rng.integers(0, 1 << n))
            mats = []
            for q in range(n - 1, -1, -1):  # qubit 0 is the last Kronecker factor
                xb, zb = (x >> q) & 1, (z >> q) & 1
                mats.append(Y if (xb and zb) else X if xb else Z if zb else np.eye(2))
            Pm = _kron_all(mats)
            want = np.vdot(v, Pm @ v) / np.vdot(v, v)
            got = o.expect_pauli(v, x, z)
            assert abs(got - want) < 1e-12, ("kron", n, x, z, got, want)
            if x == 0:
                assert abs(got.real - o.expect_z(v, z)) < 1e-12, "Z-only routine"
            assert abs(got.imag) < 1e-12, "Hermitian: real expectation"


def pin_validate(o):
    assert o.validate(3, [("cx", (0, 2), ())])
    assert not o.validate(3, [("cx", (0, 3), ())]), "qubit out of range accepted"
    assert not o.validate(3, [("cx", (1, 1), ())]), "repeated qubit accepted"
    assert not o.validate(3, [("u3", (0,), (float("nan"), 0.0, 0.0))]), "NaN accepted"


def pin_measure(o):
    """Mid-circuit measurement and reset against closed forms and a projector
    built by Kronecker products."""
    # basis states: deterministic outcome, state unchanged
    for n, x in ((3, 0b101), (5, 0b10110)):
        psi = _basis(n, x)
        for q in range(n):
            for u in (0.0, 0.37, 0.999):
                b, p, out = o.measure(psi, q, u)
                assert b == (x >> q) & 1 and p == 1.0, "basis measurement"
                _close(out, psi, what="basis collapse")
    # one qubit U3(θ,φ,λ)|0>: P(1) = sin^2(θ/2), post-measurement states are basis states
    for th, ph in ((1.1, 0.4), (2.5, -2.0), (0.3, 3.0)):
        psi = o.run(1, [("u3", (0,), (th, ph, 0.7))])
        p0 = math.cos(th / 2) ** 2
        b, p, out = o.measure(psi, 0, p0 - 1e-6)
        assert b == 0 and abs(p - p0) < 1e-12, "U3 outcome 0"
        _close(out, np.array([1.0, 0.0]), what="U3 collapse to |0>")
        b, p, out = o.measure(psi, 0, p0 + 1e-6)
        assert b == 1 and abs(p - (1 - p0)) < 1e-12, "U3 outcome 1"
        _close(out, np.array([0.0, np.exp(1j * ph)]), what="U3 collapse to |1> keeps the phase")
    # GHZ: one measurement fixes every qubit
    n = 5
    g = o.run(n, W.ghz(n))
    for q in range(n):
        b, p, out = o.measure(g, q, 0.49)
        assert b == 0 and abs(p - 0.5) < 1e-12
        _close(out, _basis(n, 0), what="GHZ -> |0..0>")
        b, p, out = o.measure(g, q, 0.51)
        assert b == 1
        _close(out, _basis(n, (1 << n) - 1), what="GHZ -> |1..1>")
    # projector brute force on random states
    rng = np.random.default_rng(21)
    for n in (1, 3, 4):
        v = random_state(n, rng)
        for q in range(n):
            proj = [np.diag([1.0, 0.0]), np.diag([0.0, 1.0])]
            m = []
            for b in (0, 1):
                P = _kron_all([proj[b] if k == q else np.eye(2) for k in range(n - 1, -1, -1)])
                w = P @ v
                m.append((float(np.vdot(w, w).real), w))
            m0, m1 = m[0][0], m[1][0]
            for u in rng.uniform(0, 1, 6):
                want = 0 if u * (m0 + m1) < m0 else 1
                if abs(u * (m0 + m1) - m0) < 1e-9:
                    continue
                b, p, out = o.measure(v, q, u)
                assert b == want, "outcome rule"
                assert abs(p - m[b][0] / (m0 + m1)) < 1e-12, "outcome probability"
                _close(out, m[b][1] / math.sqrt(m[b][0]), what="projected state")
    # reset: |x> -> |x with bit q cleared>; GHZ reset picks a branch then clears it
    for x, q in ((0b110, 1), (0b110, 0), (0b111, 2)):
        b, out = o.reset_qubit(_basis(3, x), q, 0.5)
        assert b == (x >> q) & 1
        _close(out, _basis(3, x & ~(1 << q)), what="reset of a basis state")
    b, out = o.reset_qubit(g, 2, 0.9)
    assert b == 1
    _close(out, _basis(5, 0b11011), what="reset on GHZ")


def pin_pblock(o):
    """Register merge against numpy's Kronecker product (b on the high qubits is
    np.kron(b, a) in little-endian order) and against running the gates of both
    registers on the merged state; taking a basis-state qubit out undoes a merge
    with |v> and matches a measured register's nonzero half."""
    rng = np.random.default_rng(31)
    for na, nb in ((1, 1), (2, 3), (4, 2)):
        a, b = random_state(na, rng), random_state(nb, rng)
        _close(o.kron(a, b), np.kron(b, a), what="kron vs numpy")
    ca = W.random_layered(3, 3, 1)
    cb = W.random_layered(2, 3, 2)
    merged = o.kron(o.run(3, ca), o.run(2, cb))
    shifted = [(g, tuple(q + 3 for q in qs), p) for g, qs, p in cb]
    _close(merged, o.run(5, ca + shifted), what="merged registers = monolithic run")
    for n, q, v in ((4, 0, 1), (4, 2, 0), (5, 4, 1)):
        rest = random_state(n - 1, rng)
        # insert qubit q in |v>: merge with the one-qubit state, then move it to position q
        full = np.zeros(1 << n, dtype=np.complex128)
        for j in range(1 << (n - 1)):
            low = j & ((1 << q) - 1)
            full[((j >> q) << (q + 1)) | (v << q) | low] = rest[j]
        _close(o.take_qubit(full, q, v), rest, what="take a basis-state qubit")
    g = o.run(4, W.ghz(4))
    b, _, post = o.measure(g, 1, 0.8)
    _close(o.take_qubit(post, 1, b), _basis(3, 0b111), what="take a measured GHZ qubit")


def load_alias_golden():
    rows, draws = {}, []
    with open(os.path.join(GOLDEN, "alias_worked_example.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            if parts[0] == "draw":
                draws.append((float(parts[1]), int(parts[2])))
            else:
                rows[parts[0]] = [int(v) for v in parts[1:]]
    return rows, draws


ALIAS_C = 1 << 31


def alias_masses(own, alias):
    """Units of bucket capacity that reach each outcome: own_i for i itself,
    C - own_k for every bucket k aliasing i."""
    N = own.shape[0]
    own = own.astype(np.int64)
    given = np.bincount(alias.astype(np.int64), weights=(ALIAS_C - own).astype(np.float64), minlength=N)
    return own + given.astype(np.int64)


def pin_alias(o):
    """Alias table: a hand-worked example; on random states, every light item's
    units reach it exactly and the table's only discrepancy from the quantised
    weights is the quantisation residual |N*C - sum Q|; light items alias the
    first heavy item whose excess prefix reaches their deficit prefix (a closed
    form independent of the sweep); the draw rule over a fine grid of uniforms
    reproduces the units; uniform and basis states; chi-square of draws."""
    rows, draws = load_alias_golden()
    psi = np.sqrt(np.array([0.1, 0.2, 0.3, 0.4])).astype(np.complex128)
    Q, own, alias = o.alias_build(psi)
    assert Q.tolist() == rows["Q"], f"golden Q {Q}"
    assert own.tolist() == rows["own"], f"golden own {own}"
    assert alias.tolist() == rows["alias"], f"golden alias {alias}"
    got = o.alias_sample(own, alias, np.array([d[0] for d in draws]))
    assert got.tolist() == [d[1] for d in draws], f"golden draws {got}"
    rng = np.random.default_rng(41)
    for n in (1, 2, 3, 6, 10):
        N = 1 << n
        v = random_state(n, rng)
        v[rng.random(N) < 0.3] = 0.0
        if not np.any(v):
            v[N - 1] = 1.0
        Q, own, alias = o.alias_build(v)
        Q = Q.astype(np.int64)
        p = np.abs(v) ** 2
        assert np.all(np.abs(Q - p * N / math.fsum(p) * ALIAS_C) <= 0.5 + 4e-15 * N * ALIAS_C), "quantised weights"
        assert np.all(own.astype(np.int64) <= ALIAS_C) and np.all(alias < N), "table range"
        M = alias_masses(own, alias)
        assert int(M.sum()) == N * ALIAS_C, "units per bucket"
        light = Q < ALIAS_C
        assert np.array_equal(M[light], Q[light]), "light units"
        resid = abs(N * ALIAS_C - int(Q.sum()))
        assert int(np.abs(M - Q).sum()) == resid, f"discrepancy {np.abs(M - Q).sum()} vs residual {resid}"
        assert resid <= N // 2 + 2, f"residual {resid}"
        heavy_idx = np.nonzero(~light)[0]
        if light.any():
            d = ALIAS_C - Q[light]
            Dex = np.concatenate(([0], np.cumsum(d)[:-1]))
            E = np.cumsum(Q[~light] - ALIAS_C)
            j = np.minimum(np.searchsorted(E, Dex, side="left"), len(E) - 1)
            assert np.array_equal(alias[light].astype(np.int64), heavy_idx[j]), "closed-form alias of light items"
        # the draw rule on a grid of G uniforms per bucket reproduces the units
        G = 256
        u = (np.arange(N * G) + 0.5) / (N * G)
        cnt = np.bincount(o.alias_sample(own, alias, u).astype(np.int64), minlength=N)
        refs = np.bincount(alias.astype(np.int64), minlength=N) + 1
        assert np.all(np.abs(cnt - M * G / ALIAS_C) <= refs), "grid draws vs units"
    # uniform superposition: every bucket full and its own alias
    n = 5
    v = np.full(1 << n, 2.0 ** (-n / 2), dtype=np.complex128)
    Q, own, alias = o.alias_build(v)
    assert np.all(own == ALIAS_C) and np.array_equal(alias, np.arange(1 << n)), "uniform state"
    # a total of many equal small weights and a few large ones (where a plain
    # running sum drifts): the heavy weights still round from the exact total
    v = np.full(1 << 16, 0.01, dtype=np.complex128)
    big = [5, 900, 30000]
    v[big] = 10.0
    Q, own, alias = o.alias_build(v)
    p = np.abs(v) ** 2
    total = math.fsum(p)  # correctly rounded
    exact = [float(Fraction(float(p[i])) * (1 << 16) * ALIAS_C / Fraction(total)) for i in big]
    assert all(abs(int(Q[i]) - e) <= 0.51 for i, e in zip(big, exact)), "heavy weights"
    # basis state: every draw is the basis index
    Q, own, alias = o.alias_build(_basis(6, 45))
    assert np.all(o.alias_sample(own, alias, W.shot_uniforms(3, 2000)) == 45), "basis state"
    # chi-square of draws against |psi|^2 on a random 5-qubit state
    v = random_state(5, rng)
    p = np.abs(v) ** 2
    p = p / p.sum()
    Q, own, alias = o.alias_build(v)
    Sh = 40000
    x = o.alias_sample(own, alias, W.shot_uniforms(6, Sh))
    cnt = np.bincount(x.astype(np.int64), minlength=32)
    chi2 = float(np.sum((cnt - Sh * p) ** 2 / (Sh * p)))
    assert chi2 < 31 + 6 * math.sqrt(62), f"alias chi2 {chi2}"


ALL_PINS = [pin_gate_identities, pin_kron_bruteforce, pin_apply_matrix_k5, pin_ghz, pin_qft,
            pin_norm_and_mirror, pin_norm_sum, pin_sampler, pin_expectation, pin_expect_pauli,
            pin_validate, pin_measure, pin_pblock, pin_alias]
