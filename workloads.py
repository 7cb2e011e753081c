"""Seeded synthetic inputs for the state-vector hot path.

This module is the one piece shared by the oracle, the tests, the benchmark and
the CUDA path's callers.  It only *draws* inputs: gate lists (names, qubit
indices, angles), basis-state indices, measurement uniforms, batch and serving
request mixes.  It holds none of the simulation arithmetic (no gate matrices,
no amplitudes, no probabilities).

Circuits are lists of ``(name, qubits, params)`` tuples using OpenQASM 2 gate
names (the paper's front end ingests Qiskit circuits and OpenQASM 2, §III-A):
``u3 h x y z s sdg t tdg rx ry rz p cx cz cp swap``.  ``qubits`` is a tuple of
ints, ``params`` a tuple of floats.  Qubit q is bit q of an amplitude index
(little-endian, Qiskit's convention); for ``cx`` the first qubit is the control.

Random numbers
--------------
* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): state += 0x9E3779B97F4A7C15,
  output = mix(state).  Used to seed xoshiro256** and, counter-style, for
  measurement uniforms: the i-th uniform of seed s is
  ``mix(s + (i + 1) * 0x9E3779B97F4A7C15) >> 11`` times 2^-53.
* xoshiro256** (Blackman & Vigna, 2018) for circuit structure and angles.
* A uniform double is ``(x >> 11) * 2**-53`` in [0, 1).
* Stream ids separate independent draws made from one user seed.
"""
from __future__ import annotations

import math

import numpy as np

MASK64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15

STREAM_CIRCUIT = 1
STREAM_BASIS = 2
STREAM_SHOTS = 3
STREAM_ARRIVALS = 4
STREAM_MIX = 5


def splitmix64_mix(z: int) -> int:
    """The SplitMix64 output function applied to a 64-bit state value."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


class SplitMix64:
    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next(self) -> int:
        self.state = (self.state + GOLDEN) & MASK64
        return splitmix64_mix(self.state)


def _rotl(x: int, k: int) -> int:
    return ((x << k) | (x >> (64 - k))) & MASK64


class Xoshiro256ss:
    """xoshiro256** seeded from SplitMix64(seed ^ stream * 0xD1B54A32D192ED03)."""

    def __init__(self, seed: int, stream: int = STREAM_CIRCUIT):
        sm = SplitMix64((seed ^ ((stream * 0xD1B54A32D192ED03) & MASK64)) & MASK64)
        self.s = [sm.next() for _ in range(4)]

    def next(self) -> int:
        s = self.s
        result = (_rotl((s[1] * 5) & MASK64, 7) * 9) & MASK64
        t = (s[1] << 17) & MASK64
        s[2] ^= s[0]
        s[3] ^= s[1]
        s[1] ^= s[2]
        s[0] ^= s[3]
        s[2] ^= t
        s[3] = _rotl(s[3], 45)
        return result

    def uniform(self) -> float:
        return (self.next() >> 11) * (1.0 / 9007199254740992.0)

    def below(self, m: int) -> int:
        """Integer in [0, m) as floor(u * m) (u a 53-bit uniform; m < 2^53)."""
        return min(int(self.uniform() * m), m - 1)


def shot_uniforms(seed: int, shots: int) -> np.ndarray:
    """Counter-based SplitMix64 uniforms u_0..u_{S-1} in [0,1) for measurement.

    u_i = (mix(seed + (i+1)*GOLDEN) >> 11) * 2^-53, i.e. the i-th output of a
    SplitMix64 stream seeded with ``seed``.  Vectorised with wrapping uint64.
    """
    with np.errstate(over="ignore"):
        i = np.arange(1, shots + 1, dtype=np.uint64)
        z = np.uint64(seed & MASK64) + i * np.uint64(GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


# ---------------------------------------------------------------------------
# circuits
# ---------------------------------------------------------------------------

def random_layered(n: int, depth: int, seed: int):
    """Random layered circuit: per layer U3(θ,φ,λ) on every qubit (angles iid
    U[0, 2π)), then CX on a seeded random perfect matching.

    The matching is a Fisher-Yates permutation π of 0..n-1 (for i = n-1 down to
    1, swap π[i] with π[below(i+1)]); pairs are (π0,π1), (π2,π3), ...; the
    first of each pair is the control; with odd n the last qubit idles.
    Draw order per layer: θ, φ, λ for qubit 0, 1, ..., n-1, then the matching.
    """
    rng = Xoshiro256ss(seed, STREAM_CIRCUIT)
    two_pi = 2.0 * math.pi
    gates = []
    for _ in range(depth):
        for q in range(n):
            th, ph, la = (two_pi * rng.uniform() for _ in range(3))
            gates.append(("u3", (q,), (th, ph, la)))
        perm = list(range(n))
        for i in range(n - 1, 0, -1):
            j = rng.below(i + 1)
            perm[i], perm[j] = perm[j], perm[i]
        for p in range(0, n - 1, 2):
            gates.append(("cx", (perm[p], perm[p + 1]), ()))
    return gates


def qft(n: int):
    """Quantum Fourier transform as H / controlled-phase / SWAP gates.

    For j = n-1 down to 0: H(j), then CP(π / 2^(j-k)) on (k, j) for k = j-1
    down to 0; finally SWAP(i, n-1-i) for i < n/2.  With little-endian qubits
    this maps |x> to 2^(-n/2) Σ_y exp(+2πi x y / 2^n) |y>.
    """
    gates = []
    for j in range(n - 1, -1, -1):
        gates.append(("h", (j,), ()))
        for k in range(j - 1, -1, -1):
            gates.append(("cp", (k, j), (math.pi / float(1 << (j - k)),)))
    for i in range(n // 2):
        gates.append(("swap", (i, n - 1 - i), ()))
    return gates


def ghz(n: int):
    """H on qubit 0 then a CX chain 0→1→…→n-1."""
    gates = [("h", (0,), ())]
    for q in range(n - 1):
        gates.append(("cx", (q, q + 1), ()))
    return gates


_SELF_INVERSE = {"h", "x", "y", "z", "cx", "cz", "swap"}
_SWAP_PAIR = {"s": "sdg", "sdg": "s", "t": "tdg", "tdg": "t"}
_NEGATE = {"rx", "ry", "rz", "p", "cp"}


def inverse(gates):
    """Inverse circuit: reverse order, invert each gate.

    U3(θ,φ,λ)^-1 = U3(-θ,-λ,-φ); rotations/phases negate their angle; S/T map
    to their daggers; the rest listed in _SELF_INVERSE are involutions.
    """
    out = []
    for name, qs, ps in reversed(gates):
        if name == "u3":
            th, ph, la = ps
            out.append(("u3", qs, (-th, -la, -ph)))
        elif name in _SELF_INVERSE:
            out.append((name, qs, ps))
        elif name in _SWAP_PAIR:
            out.append((_SWAP_PAIR[name], qs, ps))
        elif name in _NEGATE:
            out.append((name, qs, tuple(-p for p in ps)))
        else:
            raise ValueError(f"no inverse rule for gate {name!r}")
    return out


def basis_index(n: int, seed: int) -> int:
    """Seeded uniform basis-state index in [0, 2^n)."""
    rng = Xoshiro256ss(seed, STREAM_BASIS)
    return rng.next() >> (64 - n) if n > 0 else 0


def random_gate_soup(n: int, count: int, seed: int, kinds=None):
    """Mixed gates of every IR kind on random qubits (for oracle/kernel tests)."""
    rng = Xoshiro256ss(seed, STREAM_MIX)
    one = ["u3", "h", "x", "y", "z", "s", "sdg", "t", "tdg", "rx", "ry", "rz", "p"]
    two = ["cx", "cz", "cp", "swap"]
    pool = kinds if kinds is not None else (one + two if n >= 2 else one)
    nparams = {"u3": 3, "rx": 1, "ry": 1, "rz": 1, "p": 1, "cp": 1}
    gates = []
    for _ in range(count):
        name = pool[rng.below(len(pool))]
        if name in two:
            a = rng.below(n)
            b = rng.below(n - 1)
            b = b + 1 if b >= a else b
            qs = (a, b)
        else:
            qs = (rng.below(n),)
        ps = tuple(2.0 * math.pi * rng.uniform() - math.pi for _ in range(nparams.get(name, 0)))
        gates.append((name, qs, ps))
    return gates


# ---------------------------------------------------------------------------
# batched and serving mixes
# ---------------------------------------------------------------------------

def batch_mix(count: int, seed: int, n_lo: int = 10, n_hi: int = 20, d_lo: int = 10, d_hi: int = 60):
    """(n, depth, circuit_seed) for a batch of independent random layered
    circuits: n ~ U{n_lo..n_hi}, depth ~ U{d_lo..d_hi}, circuit seed = seed + i."""
    rng = Xoshiro256ss(seed, STREAM_MIX)
    out = []
    for i in range(count):
        n = n_lo + rng.below(n_hi - n_lo + 1)
        d = d_lo + rng.below(d_hi - d_lo + 1)
        out.append((n, d, seed + i))
    return out


def geometric_skew_p(n_lo: int = 8, n_hi: int = 30, mean: float = 16.0) -> float:
    """p with E[n] = mean for P(n) ∝ (1-p)^(n-n_lo) on n_lo..n_hi (bisection)."""
    lo, hi = 1e-9, 1.0 - 1e-9
    ns = np.arange(n_lo, n_hi + 1, dtype=np.float64)
    for _ in range(200):
        p = 0.5 * (lo + hi)
        w = (1.0 - p) ** (ns - n_lo)
        m = float((w * ns).sum() / w.sum())
        if m > mean:
            lo = p
        else:
            hi = p
    return 0.5 * (lo + hi)


def serving_requests(count: int, seed: int, rate_hz: float, n_lo: int = 8, n_hi: int = 30,
                     mean_n: float = 16.0, d_lo: int = 10, d_hi: int = 100, shots: int = 1000):
    """Poisson request stream.  Each request is a dict with arrival time (s),
    n (geometric-skewed on n_lo..n_hi with mean ≈ mean_n), depth ~ U{d_lo..d_hi},
    circuit seed, and either ``shots`` or a non-empty random Z ``zmask`` (50/50)."""
    p = geometric_skew_p(n_lo, n_hi, mean_n)
    ns = np.arange(n_lo, n_hi + 1)
    w = (1.0 - p) ** (ns - n_lo)
    cdf = np.cumsum(w / w.sum())
    rng = Xoshiro256ss(seed, STREAM_ARRIVALS)
    t = 0.0
    reqs = []
    for i in range(count):
        t += -math.log(1.0 - rng.uniform()) / rate_hz
        n = int(ns[min(int(np.searchsorted(cdf, rng.uniform(), side="right")), len(ns) - 1)])
        d = d_lo + rng.below(d_hi - d_lo + 1)
        req = {"id": i, "t": t, "n": n, "depth": d, "seed": seed * 1000003 + i}
        if rng.uniform() < 0.5:
            req["shots"] = shots
            req["shot_seed"] = (seed * 7919 + i) & MASK64
        else:
            m = 0
            while m == 0:
                m = rng.next() & ((1 << n) - 1)
            req["zmask"] = m
        reqs.append(req)
    return reqs


def calibration_circuits(n: int, seed: int = 7):
    """Circuits the runtime model is calibrated on at n qubits: random layered
    circuits of depth 2, 8, 24 and 60, the QFT, GHZ and a single gate."""
    return [random_layered(n, 8, seed + n), random_layered(n, 2, seed + 2 * n),
            random_layered(n, 24, seed + 3 * n), random_layered(n, 60, seed + 4 * n),
            qft(n), ghz(n), ghz(n)[:1]]
