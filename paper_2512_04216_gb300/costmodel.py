"""GPU-calibrated runtime model (Eq. 1: T_total ~ sum over operations of a
hardware-calibrated coefficient times the operation's complexity term).

For this state-vector backend the operations are the plan's HBM passes and
its dense-block arithmetic, and the end-of-circuit sampling:

    T_apply(n, circuit) ~ c_fix + c_gate * dense_gates + C_pass(n) * passes
                          + c_flop * flops + c_phase * phase_ops * 2^n
    T_shots(n, S)       ~ c1(n) + c2 * S

`dense_gates` counts the non-diagonal gates, each of which the host planner
multiplies into a fused block (this host work dominates small states;
diagonal gates only add phase terms).  `passes`, dense-block flops and phase
ops come from the host planner (sv_plan_stats, no GPU work); a phase op
(per-thread phase sums, exponentials and a complex product per amplitude) has
its own coefficient per amplitude, fitted like the others.
The coefficients are measured once on the device by `calibrate` (synthetic
circuits of different densities over a grid of qubit counts, one joint least
squares fit) and C_pass is interpolated in n with a monotone piecewise cubic
Hermite interpolant (Fritsch-Carlson slopes) on log coefficients, as the paper
does for its C_op(n) curves; T_shots is a linear regression in S.  The serving loop uses the
predictions to order waiting requests (shortest predicted first).
"""
from __future__ import annotations

import json
import math
from dataclasses import asdict, dataclass, field

import numpy as np


# ---------------------------------------------------------------------------
# monotone piecewise cubic Hermite interpolation (Fritsch & Carlson, 1980)
# ---------------------------------------------------------------------------

def _pchip_slopes(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    h = np.diff(x)
    delta = np.diff(y) / h
    m = np.zeros_like(y)
    if len(x) == 2:
        m[:] = delta[0]
        return m
    for k in range(1, len(x) - 1):
        if delta[k - 1] * delta[k] <= 0.0:
            m[k] = 0.0
        else:
            w1 = 2.0 * h[k] + h[k - 1]
            w2 = h[k] + 2.0 * h[k - 1]
            m[k] = (w1 + w2) / (w1 / delta[k - 1] + w2 / delta[k])
    # one-sided three-point end slopes, kept shape-preserving
    for end, (h0, h1, d0, d1) in ((0, (h[0], h[1], delta[0], delta[1])),
                                  (len(x) - 1, (h[-1], h[-2], delta[-1], delta[-2]))):
        s = ((2.0 * h0 + h1) * d0 - h0 * d1) / (h0 + h1)
        if s * d0 <= 0.0:
            s = 0.0
        elif d0 * d1 <= 0.0 and abs(s) > abs(3.0 * d0):
            s = 3.0 * d0
        m[end] = s
    return m


def pchip(x, y):
    """Returns f(t): the monotone cubic Hermite interpolant through (x, y)
    (x strictly increasing), constant-slope extrapolation outside."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    if x.ndim != 1 or x.shape != y.shape or x.shape[0] < 2 or np.any(np.diff(x) <= 0):
        raise ValueError("pchip needs >= 2 strictly increasing knots")
    m = _pchip_slopes(x, y)

    def f(t):
        t = np.asarray(t, dtype=np.float64)
        k = np.clip(np.searchsorted(x, t, side="right") - 1, 0, len(x) - 2)
        h = x[k + 1] - x[k]
        s = (t - x[k]) / h
        h00 = (1 + 2 * s) * (1 - s) ** 2
        h10 = s * (1 - s) ** 2
        h01 = s * s * (3 - 2 * s)
        h11 = s * s * (s - 1)
        inner = h00 * y[k] + h10 * h * m[k] + h01 * y[k + 1] + h11 * h * m[k + 1]
        lo = y[0] + m[0] * (t - x[0])
        hi = y[-1] + m[-1] * (t - x[-1])
        return np.where(t < x[0], lo, np.where(t > x[-1], hi, inner))

    return f


def linear_fit(x, y):
    """Least-squares (c1, c2) of y ~ c1 + c2 x."""
    A = np.stack([np.ones(len(x)), np.asarray(x, dtype=np.float64)], axis=1)
    (c1, c2), *_ = np.linalg.lstsq(A, np.asarray(y, dtype=np.float64), rcond=None)
    return float(c1), float(c2)


# ---------------------------------------------------------------------------
# the model
# ---------------------------------------------------------------------------

@dataclass
class CostModel:
    ns: list = field(default_factory=list)        # calibrated qubit counts
    c_pass: list = field(default_factory=list)    # ms per HBM pass at each n
    c_flop: float = 0.0                           # ms per dense-block flop
    c_phase: float = 0.0                          # ms per amplitude per phase op
    c_fix: float = 0.0                            # ms per apply call (upload, launches)
    c_gate: float = 0.0                           # ms of host fusion per non-diagonal gate
    c_shot1: list = field(default_factory=list)   # ms of CDF build + fixed sampling cost at each n
    c_shot2: float = 0.0                          # ms per shot

    @staticmethod
    def eff_flops(n: int, stats: dict) -> float:
        """Dense-block flops of a plan."""
        return float(stats["flops"])

    @staticmethod
    def phase_amps(n: int, stats: dict) -> float:
        """Phase ops times amplitudes."""
        return float(stats["n_phase"]) * float(1 << n)

    def _curve(self, vals, n):
        v = np.maximum(np.asarray(vals, dtype=np.float64), 1e-30)
        return float(np.exp(pchip(self.ns, np.log(v))(float(n))))

    # IR kinds of diagonal gates (z, s, sdg, t, tdg, rz, p, cz, cp)
    DIAGONAL_KINDS = (5, 6, 7, 8, 9, 12, 13, 15, 16)

    @staticmethod
    def dense_gates(ir, n_gates: int) -> int:
        kinds = np.asarray(ir["kind"][:n_gates])
        return int(n_gates - np.isin(kinds, CostModel.DIAGONAL_KINDS).sum())

    def apply_ms(self, n: int, passes: int, eff_flops: float, dense_gates: int = 0,
                 phase_amps: float = 0.0) -> float:
        return (self.c_fix + self.c_gate * dense_gates + self._curve(self.c_pass, n) * passes
                + self.c_flop * eff_flops + self.c_phase * phase_amps)

    def shots_ms(self, n: int, shots: int) -> float:
        return self._curve(self.c_shot1, n) + self.c_shot2 * shots

    def predict_ms(self, n: int, circuit, shots: int = 0, opts=None) -> float:
        from . import capi
        st = capi.sv_plan_stats(n, circuit, opts)
        ir, _keep = capi.to_ir(circuit)
        return (self.apply_ms(n, st["n_passes"], self.eff_flops(n, st), self.dense_gates(ir, len(circuit)),
                              self.phase_amps(n, st))
                + (self.shots_ms(n, shots) if shots else 0.0))

    def to_json(self) -> str:
        return json.dumps(asdict(self))

    @staticmethod
    def from_json(s: str) -> "CostModel":
        return CostModel(**json.loads(s))


def calibrate(circuits_for, ns=(10, 12, 14, 16, 18, 20, 22, 24, 26, 28), reps: int = 2, opts=None) -> CostModel:
    """Measures the coefficients on the current device (a one-time routine):
    one joint least-squares fit of T = c_fix + c_gate * dense gates + C_pass(n)
    * passes + c_flop * effective flops over the caller's calibration circuits at
    every n in `ns` (each timed warm: best of reps + 1 runs on one state).
    `circuits_for(n)` returns the gate lists to time at n qubits; a mix of
    shallow and deep circuits, with and without diagonal gates, makes the fit
    well conditioned."""
    import torch

    from . import capi
    from .statevector import StateVector

    model = CostModel(ns=[int(n) for n in ns])
    rows, times, shot_samples = [], [], []
    for i, n in enumerate(ns):
        circuits = list(circuits_for(n))
        s = StateVector(n)
        for c in circuits:
            st = capi.sv_plan_stats(n, c, opts)
            ir, keep = capi.to_ir(c)
            best = math.inf
            for _ in range(reps + 1):
                s.reset(0)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s.stream)
                capi.sv_apply_circuit(s.h, ir, len(c), opts)
                e1.record(s.stream)
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1))
            row = [0.0] * (len(ns) + 4)
            row[i] = float(st["n_passes"])
            row[len(ns)] = CostModel.eff_flops(n, st)
            row[len(ns) + 1] = 1.0
            row[len(ns) + 2] = float(CostModel.dense_gates(ir, len(c)))
            row[len(ns) + 3] = CostModel.phase_amps(n, st)
            rows.append(row)
            times.append(best)
        for S in (1, 1000, 100000):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s.stream)
            s.sample(S, 3)
            e1.record(s.stream)
            torch.cuda.synchronize()
            shot_samples.append((n, S, e0.elapsed_time(e1)))
        s.close()
    A = np.asarray(rows, dtype=np.float64)
    scale = np.maximum(np.abs(A).max(axis=0), 1e-30)
    sol, *_ = np.linalg.lstsq(A / scale, np.asarray(times), rcond=None)
    sol = sol / scale
    model.c_pass = [max(float(v), 1e-6) for v in sol[:len(ns)]]
    model.c_flop = max(float(sol[len(ns)]), 0.0)
    model.c_fix = max(float(sol[len(ns) + 1]), 0.0)
    model.c_gate = max(float(sol[len(ns) + 2]), 0.0)
    model.c_phase = max(float(sol[len(ns) + 3]), 0.0)
    _, c2 = linear_fit([S for _, S, _ in shot_samples], [t for _, _, t in shot_samples])
    model.c_shot2 = max(c2, 0.0)
    for n in ns:
        pts = [(S, t) for m, S, t in shot_samples if m == n]
        c1 = float(np.mean([t - model.c_shot2 * S for S, t in pts]))
        model.c_shot1.append(max(c1, 1e-4))
    return model
