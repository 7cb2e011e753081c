"""Python access to the complex128 CPU oracle (oracle/sv_oracle.c).

TEST INFRASTRUCTURE ONLY: used by tests/, __graft_entry__.smoke() and the CPU
baseline / reference leg of bench.py.  The CUDA library never imports this
package, and this package never imports the CUDA library.

Functions take circuits in the ``(name, qubits, params)`` form produced by
``workloads``; the gate-name table below is the oracle's own.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))

_KIND = {
    "u3": 1, "h": 2, "x": 3, "y": 4, "z": 5, "s": 6, "sdg": 7, "t": 8, "tdg": 9,
    "rx": 10, "ry": 11, "rz": 12, "p": 13, "cx": 14, "cz": 15, "cp": 16, "swap": 17,
    "unitary": 18,
}


class _Gate(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32),
        ("nq", ctypes.c_int32),
        ("q", ctypes.c_int32 * 5),
        ("_pad", ctypes.c_int32),
        ("p", ctypes.c_double * 3),
        ("mat", ctypes.c_void_p),
    ]


def _gates(circuit):
    arr = (_Gate * max(len(circuit), 1))()
    keep = []
    for a, (name, qs, ps) in enumerate(circuit):
        g = arr[a]
        g.kind = _KIND[name]
        g.nq = len(qs)
        for i, q in enumerate(qs):
            g.q[i] = int(q)
        for i, p in enumerate(ps[:3] if name != "unitary" else ()):
            g.p[i] = float(p)
        if name == "unitary":
            m = np.ascontiguousarray(ps[0], dtype=np.complex128)
            keep.append(m)
            g.mat = m.ctypes.data
    return arr, keep


class Oracle:
    """One loaded copy of the oracle library (the default one, or a test build)."""

    def __init__(self, path: str):
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        u64 = ctypes.c_uint64
        L.orc_run.argtypes = [P, ctypes.c_int, P, u64]
        L.orc_run.restype = ctypes.c_int
        L.orc_validate.argtypes = [ctypes.c_int, P, u64]
        L.orc_validate.restype = ctypes.c_int
        L.orc_gate_matrix.argtypes = [P, P]
        L.orc_gate_matrix.restype = ctypes.c_int
        L.orc_apply_matrix.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P]
        L.orc_apply_matrix.restype = None
        L.orc_norm2.argtypes = [P, u64]
        L.orc_norm2.restype = ctypes.c_double
        L.orc_cdf.argtypes = [P, u64, P]
        L.orc_cdf.restype = None
        L.orc_sample.argtypes = [P, u64, P, u64, ctypes.c_double, P, P]
        L.orc_sample.restype = u64
        L.orc_expect_z.argtypes = [P, u64, u64]
        L.orc_expect_pauli.argtypes = [P, ctypes.c_int, u64, u64, P, P]
        L.orc_expect_pauli.restype = ctypes.c_int
        L.orc_measure.argtypes = [P, u64, ctypes.c_int, ctypes.c_double, P]
        L.orc_measure.restype = ctypes.c_int
        L.orc_reset_qubit.argtypes = [P, u64, ctypes.c_int, ctypes.c_double]
        L.orc_reset_qubit.restype = ctypes.c_int
        L.orc_kron.argtypes = [P, ctypes.c_int, P, ctypes.c_int, P]
        L.orc_kron.restype = None
        L.orc_take_qubit.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, P]
        L.orc_take_qubit.restype = None
        L.orc_expect_z.restype = ctypes.c_double
        L.orc_alias_build.argtypes = [P, u64, P, P, P]
        L.orc_alias_build.restype = ctypes.c_int
        L.orc_alias_sample.argtypes = [P, P, u64, P, u64, P]
        L.orc_alias_sample.restype = None
        L.orc_set_threads.argtypes = [ctypes.c_int]
        L.orc_set_threads.restype = None
        L.orc_max_threads.argtypes = []
        L.orc_max_threads.restype = ctypes.c_int
        self.L = L
        self.path = path

    def set_threads(self, t: int) -> None:
        self.L.orc_set_threads(int(t))

    def max_threads(self) -> int:
        return int(self.L.orc_max_threads())

    def gate_matrix(self, name, qubits=(0,), params=()):
        """The oracle's 2^k x 2^k matrix for one gate (row-major complex128)."""
        arr, keep = _gates([(name, tuple(qubits), tuple(params))])
        m = np.zeros(1024, dtype=np.complex128)
        k = self.L.orc_gate_matrix(ctypes.byref(arr[0]), m.ctypes.data)
        if k < 0:
            raise ValueError(name)
        return m[: (1 << k) * (1 << k)].reshape(1 << k, 1 << k).copy()

    def run(self, n: int, circuit, psi=None) -> np.ndarray:
        """Apply ``circuit`` gate by gate to psi (default |0...0>); returns psi."""
        psi = basis(n) if psi is None else np.array(psi, dtype=np.complex128, copy=True)
        assert psi.shape == (1 << n,)
        arr, keep = _gates(circuit)
        rc = self.L.orc_run(psi.ctypes.data, n, ctypes.cast(arr, ctypes.c_void_p), len(circuit))
        if rc != 0:
            raise ValueError("oracle rejected the circuit")
        return psi

    def validate(self, n: int, circuit) -> bool:
        arr, keep = _gates(circuit)
        return self.L.orc_validate(n, ctypes.cast(arr, ctypes.c_void_p), len(circuit)) == 0

    def apply_matrix(self, psi, targets, M) -> np.ndarray:
        psi = np.array(psi, dtype=np.complex128, copy=True)
        n = int(psi.shape[0]).bit_length() - 1
        t = np.ascontiguousarray(targets, dtype=np.int32)
        M = np.ascontiguousarray(M, dtype=np.complex128)
        self.L.orc_apply_matrix(psi.ctypes.data, n, len(t), t.ctypes.data, M.ctypes.data)
        return psi

    def norm2(self, psi) -> float:
        psi = np.ascontiguousarray(psi, dtype=np.complex128)
        return float(self.L.orc_norm2(psi.ctypes.data, psi.shape[0]))

    def cdf(self, psi) -> np.ndarray:
        psi = np.ascontiguousarray(psi, dtype=np.complex128)
        C = np.empty(psi.shape[0], dtype=np.float64)
        self.L.orc_cdf(psi.ctypes.data, psi.shape[0], C.ctypes.data)
        return C

    def sample(self, psi, uniforms, eps: float = 1e-9):
        """Returns (bitstrings uint64[S], boundary uint8[S], n_boundary)."""
        return self.sample_cdf(self.cdf(psi), uniforms, eps)

    def sample_cdf(self, C, uniforms, eps: float = 1e-9):
        C = np.ascontiguousarray(C, dtype=np.float64)
        u = np.ascontiguousarray(uniforms, dtype=np.float64)
        out = np.empty(u.shape[0], dtype=np.uint64)
        b = np.empty(u.shape[0], dtype=np.uint8)
        nb = self.L.orc_sample(C.ctypes.data, C.shape[0], u.ctypes.data, u.shape[0], eps,
                               out.ctypes.data, b.ctypes.data)
        return out, b, int(nb)

    def expect_z(self, psi, zmask: int) -> float:
        psi = np.ascontiguousarray(psi, dtype=np.complex128)
        return float(self.L.orc_expect_z(psi.ctypes.data, psi.shape[0], int(zmask)))


    def expect_pauli(self, psi, x_mask: int, z_mask: int) -> complex:
        """<psi|P|psi>/<psi|psi> for P = X^x Z^z with Y on qubits in both masks."""
        psi = np.ascontiguousarray(psi, dtype=np.complex128)
        n = int(psi.shape[0]).bit_length() - 1
        re, im = ctypes.c_double(), ctypes.c_double()
        if self.L.orc_expect_pauli(psi.ctypes.data, n, int(x_mask), int(z_mask), ctypes.byref(re),
                                   ctypes.byref(im)) != 0:
            raise MemoryError("oracle: no memory for the Pauli copy")
        return complex(re.value, im.value)

    def measure(self, psi, q: int, u: float):
        """Mid-circuit measurement of qubit q: returns (outcome, prob, collapsed copy)."""
        psi = np.array(psi, dtype=np.complex128, copy=True)
        prob = ctypes.c_double()
        out = self.L.orc_measure(psi.ctypes.data, psi.shape[0], int(q), float(u), ctypes.byref(prob))
        return int(out), float(prob.value), psi

    def reset_qubit(self, psi, q: int, u: float):
        """Reset of qubit q to |0> by measurement: returns (outcome, new copy)."""
        psi = np.array(psi, dtype=np.complex128, copy=True)
        out = self.L.orc_reset_qubit(psi.ctypes.data, psi.shape[0], int(q), float(u))
        return int(out), psi


    def kron(self, a, b):
        """Merged register a (x) b, a on the low qubits."""
        a = np.ascontiguousarray(a, dtype=np.complex128)
        b = np.ascontiguousarray(b, dtype=np.complex128)
        na, nb = a.shape[0].bit_length() - 1, b.shape[0].bit_length() - 1
        out = np.empty(a.shape[0] * b.shape[0], dtype=np.complex128)
        self.L.orc_kron(a.ctypes.data, na, b.ctypes.data, nb, out.ctypes.data)
        return out

    def take_qubit(self, psi, q: int, v: int):
        """Register without qubit q, which must be in the basis state |v>."""
        psi = np.ascontiguousarray(psi, dtype=np.complex128)
        n = psi.shape[0].bit_length() - 1
        out = np.empty(psi.shape[0] // 2, dtype=np.complex128)
        self.L.orc_take_qubit(psi.ctypes.data, n, int(q), int(v), out.ctypes.data)
        return out


    def alias_build(self, psi):
        """Walker alias table of |psi|^2: (Q uint64[N], own uint32[N], alias uint32[N])."""
        psi = np.ascontiguousarray(psi, dtype=np.complex128)
        N = psi.shape[0]
        Q = np.empty(N, dtype=np.uint64)
        own = np.empty(N, dtype=np.uint32)
        alias = np.empty(N, dtype=np.uint32)
        rc = self.L.orc_alias_build(psi.ctypes.data, N, Q.ctypes.data, own.ctypes.data, alias.ctypes.data)
        if rc != 0:
            raise ValueError("state has no weight")
        return Q, own, alias

    def alias_sample(self, own, alias, uniforms):
        """Draws from an alias table for the given uniforms (uint64[S])."""
        own = np.ascontiguousarray(own, dtype=np.uint32)
        alias = np.ascontiguousarray(alias, dtype=np.uint32)
        u = np.ascontiguousarray(uniforms, dtype=np.float64)
        out = np.empty(u.shape[0], dtype=np.uint64)
        self.L.orc_alias_sample(own.ctypes.data, alias.ctypes.data, own.shape[0], u.ctypes.data,
                                u.shape[0], out.ctypes.data)
        return out


def basis(n: int, index: int = 0) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[index] = 1.0
    return psi


_default = None


def default() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle(_build.build())
    return _default


def set_threads(t): default().set_threads(t)
def max_threads(): return default().max_threads()
def gate_matrix(name, qubits=(0,), params=()): return default().gate_matrix(name, qubits, params)
def run(n, circuit, psi=None): return default().run(n, circuit, psi)
def validate(n, circuit): return default().validate(n, circuit)
def apply_matrix(psi, targets, M): return default().apply_matrix(psi, targets, M)
def norm2(psi): return default().norm2(psi)
def cdf(psi): return default().cdf(psi)
def sample(psi, uniforms, eps=1e-9): return default().sample(psi, uniforms, eps)
def sample_cdf(C, uniforms, eps=1e-9): return default().sample_cdf(C, uniforms, eps)
def expect_z(psi, zmask): return default().expect_z(psi, zmask)
def expect_pauli(psi, x_mask, z_mask): return default().expect_pauli(psi, x_mask, z_mask)
def measure(psi, q, u): return default().measure(psi, q, u)
def reset_qubit(psi, q, u): return default().reset_qubit(psi, q, u)
def kron(a, b): return default().kron(a, b)
def take_qubit(psi, q, v): return default().take_qubit(psi, q, v)
def alias_build(psi): return default().alias_build(psi)
def alias_sample(own, alias, uniforms): return default().alias_sample(own, alias, uniforms)


def fidelity(a, b) -> float:
    """|<a|b>|^2 / (||a||^2 ||b||^2) in double precision."""
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    ov = np.vdot(a, b)
    return float(abs(ov) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real))
