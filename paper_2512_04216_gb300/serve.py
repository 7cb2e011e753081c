"""Continuous-batching request loop over the C-ABI.

The paper routes heterogeneous streams of circuits through one service and
schedules them with runtime estimates (§III-C, §IV-B, §VI); this module is the
GPU state-vector version of that service loop.  Requests (a circuit IR plus
either a shot count or a Z-string mask) arrive over time; the server

  * keeps a waiting queue and admits work whenever capacity frees up -- it
    never waits for the current work to drain (continuous batching);
  * sends small requests (<= ``small_max_qubits``) to one graph-captured
    persistent batch launch (sv_batch_*) per scheduling round, so hundreds of
    circuits share one launch;
  * gives each larger request its own resident state on one of a pool of CUDA
    streams, admitted only while the sum of admitted footprints
    (2^n * 8 bytes plus measurement scratch) stays within an HBM budget, so
    their passes interleave on the device;
  * records arrival, start and finish times of every request;
  * with a calibrated cost model (costmodel.py, Eq. 1), admits waiting large
    requests shortest predicted runtime first instead of fewest qubits first;
  * with ``tc_from_qubits``, applies requests of at least that many qubits with
    the tensor-core passes (``tc_opts``, precision 1) and smaller ones with
    ``opts`` (on a GB300 the tensor-core path is faster from ~24 qubits; below,
    planning and launches dominate a circuit and it is slightly slower).

The plain path (``run_plain``) serves the same requests one at a time: create
a state, apply, measure, destroy, on one stream, with the same per-size options.  Control is Python; every
simulation step is a library call, and ctypes releases the GIL during each
call so worker threads overlap.
"""
from __future__ import annotations

import concurrent.futures as cf
import queue
import threading
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import capi
from .batch import Batch
from .statevector import StateVector


@dataclass
class Request:
    id: int
    t: float            # arrival time (s from the start of the run)
    n: int
    ir: np.ndarray      # sv_gate array
    n_gates: int
    shots: int = 0
    shot_seed: int = 0
    zmask: int = 0


@dataclass
class Result:
    id: int
    t_arrival: float
    t_start: float
    t_done: float
    path: str
    samples: np.ndarray | None = None
    expect: float | None = None

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


def footprint_bytes(n: int) -> int:
    """Device bytes a resident request holds: the complex64 state plus the
    sampler's double chunk sums, block prefix and partials."""
    amps = 1 << n
    return amps * 8 + (amps >> 6) * 8 + (amps >> 12) * 24 + (1 << 20)


def make_requests(specs, circuit_fn):
    """specs: dicts from workloads.serving_requests; circuit_fn(n, depth, seed)
    -> gate list.  IR marshalling happens here, outside any timed region."""
    reqs = []
    for sp in specs:
        circ = circuit_fn(sp["n"], sp["depth"], sp["seed"])
        ir, _ = capi.to_ir(circ)
        reqs.append(Request(id=sp["id"], t=sp["t"], n=sp["n"], ir=ir, n_gates=len(circ),
                            shots=sp.get("shots", 0), shot_seed=sp.get("shot_seed", 0),
                            zmask=sp.get("zmask", 0)))
    return reqs


def default_tc_opts():
    """Options of the tensor-core path: 3xTF32 stage products, blocks up to 4 qubits."""
    return capi.make_opts(k_max=5, precision=1)


def _opts_for(req: Request, opts, tc_opts, tc_from):
    return tc_opts if (tc_from is not None and req.n >= tc_from) else opts


def _run_single(req: Request, stream, opts, t0: float) -> Result:
    t_start = time.perf_counter() - t0
    with torch.cuda.stream(stream):
        s = StateVector(req.n, stream=stream)
        capi.sv_apply_circuit(s.h, req.ir, req.n_gates, opts)
        samples = expect = None
        if req.shots:
            samples = np.empty(req.shots, dtype=np.uint64)
            capi.sv_sample(s.h, req.shots, req.shot_seed, samples, False)
        else:
            expect = capi.sv_expect_pauli(s.h, 0, req.zmask)
        s.close()
    return Result(req.id, req.t, t_start, time.perf_counter() - t0, "stream", samples, expect)


class Server:
    def __init__(self, small_max_qubits: int = 14, streams: int = 8, hbm_budget: int | None = None,
                 batch_max: int = 1024, opts=None, batch_opts=None, cost_model=None,
                 tc_from_qubits: int | None = None, tc_opts=None):
        self.small_max = small_max_qubits
        self.n_streams = streams
        if hbm_budget is None:
            free, _total = torch.cuda.mem_get_info()
            hbm_budget = int(free * 0.6)
        self.budget = hbm_budget
        self.batch_max = batch_max
        self.opts = opts if opts is not None else capi.make_opts()
        self.tc_from = tc_from_qubits
        self.tc_opts = tc_opts if tc_opts is not None else default_tc_opts()
        self.batch_opts = batch_opts or {}
        self.streams = queue.SimpleQueue()
        for _ in range(streams):
            self.streams.put(torch.cuda.Stream())
        self.batch_stream = torch.cuda.Stream()
        self.cost_model = cost_model
        self._pred = {}

    def predicted_ms(self, r: Request) -> float:
        """Cost-model runtime of a request (cached; planning on the host only)."""
        if r.id not in self._pred:
            st = capi.sv_plan_stats_ir(r.n, r.ir, r.n_gates, self._opts(r))
            ms = self.cost_model.apply_ms(r.n, st["n_passes"], self.cost_model.eff_flops(r.n, st),
                                          self.cost_model.dense_gates(r.ir, r.n_gates),
                                          self.cost_model.phase_amps(r.n, st))
            ms += self.cost_model.shots_ms(r.n, r.shots) if r.shots else self.cost_model.shots_ms(r.n, 0)
            self._pred[r.id] = ms
        return self._pred[r.id]

    def _opts(self, r: Request):
        return _opts_for(r, self.opts, self.tc_opts, self.tc_from)

    def _order_key(self, r: Request):
        if self.cost_model is None:
            return (r.n, r.t)
        return (self.predicted_ms(r), r.t)

    def _run_batch(self, reqs, t0):
        t_start = time.perf_counter() - t0
        b = Batch(None, [r.n for r in reqs], [r.shots for r in reqs], [r.shot_seed for r in reqs],
                  zmasks=[r.zmask for r in reqs], irs=[(r.ir, r.n_gates) for r in reqs],
                  stream=self.batch_stream, **self.batch_opts)
        b.launch()
        b.synchronize()
        out = []
        for i, r in enumerate(reqs):
            samples = b.samples(i) if r.shots else None
            expect = b.expectation(i)[0] if (r.zmask and not r.shots) else None
            out.append(Result(r.id, r.t, t_start, time.perf_counter() - t0, "batch", samples, expect))
        b.close()
        return out

    def run(self, requests, max_wall_s: float = 600.0):
        """Serve `requests` (arrival times relative to the start) to completion."""
        reqs = sorted(requests, key=lambda r: r.t)
        results: list[Result] = []
        waiting_small: list[Request] = []
        waiting_large: list[Request] = []
        used = 0
        inflight = {}          # future -> (kind, bytes, stream)
        batch_busy = False
        nxt = 0
        pool = cf.ThreadPoolExecutor(max_workers=self.n_streams + 1)
        t0 = time.perf_counter()
        try:
            while len(results) < len(reqs):
                now = time.perf_counter() - t0
                if now > max_wall_s:
                    raise TimeoutError(f"serving did not finish in {max_wall_s} s")
                while nxt < len(reqs) and reqs[nxt].t <= now:
                    r = reqs[nxt]
                    (waiting_small if r.n <= self.small_max else waiting_large).append(r)
                    nxt += 1
                # admit large requests while slots and memory allow (smallest first
                # among those that arrived, so small-footprint work is not starved)
                waiting_large.sort(key=self._order_key)
                i = 0
                while i < len(waiting_large):
                    r = waiting_large[i]
                    need = footprint_bytes(r.n)
                    if need > self.budget:
                        raise ValueError(f"request {r.id} ({r.n} qubits) exceeds the HBM budget")
                    if used + need <= self.budget and not self.streams.empty():
                        st = self.streams.get()
                        fut = pool.submit(_run_single, r, st, self._opts(r), t0)
                        inflight[fut] = ("single", need, st)
                        used += need
                        waiting_large.pop(i)
                    else:
                        i += 1
                # one batch launch in flight at a time; it takes everything waiting
                if waiting_small and not batch_busy:
                    take, waiting_small = waiting_small[:self.batch_max], waiting_small[self.batch_max:]
                    fut = pool.submit(self._run_batch, take, t0)
                    inflight[fut] = ("batch", 0, None)
                    batch_busy = True
                # wait for a completion or the next arrival
                timeout = None
                if nxt < len(reqs):
                    timeout = max(0.0, reqs[nxt].t - (time.perf_counter() - t0))
                if inflight:
                    done, _ = cf.wait(list(inflight), timeout=timeout if timeout is not None else 0.05,
                                      return_when=cf.FIRST_COMPLETED)
                    for fut in done:
                        kind, nbytes, st = inflight.pop(fut)
                        res = fut.result()
                        if kind == "batch":
                            results.extend(res)
                            batch_busy = False
                        else:
                            results.append(res)
                            used -= nbytes
                            self.streams.put(st)
                elif timeout:
                    time.sleep(min(timeout, 0.05))
        finally:
            pool.shutdown(wait=True)
        return sorted(results, key=lambda r: r.id)


def run_plain(requests, opts=None, max_wall_s: float = 600.0, tc_from_qubits: int | None = None, tc_opts=None):
    """One circuit at a time, in arrival order, on one stream."""
    reqs = sorted(requests, key=lambda r: r.t)
    opts = opts if opts is not None else capi.make_opts()
    tc_opts = tc_opts if tc_opts is not None else default_tc_opts()
    stream = torch.cuda.current_stream()
    results = []
    t0 = time.perf_counter()
    for r in reqs:
        now = time.perf_counter() - t0
        if now > max_wall_s:
            raise TimeoutError(f"plain path did not finish in {max_wall_s} s")
        if r.t > now:
            time.sleep(r.t - now)
        res = _run_single(r, stream, _opts_for(r, opts, tc_opts, tc_from_qubits), t0)
        res.path = "plain"
        results.append(res)
    return sorted(results, key=lambda r: r.id)


def summarize(results) -> dict:
    lat = np.array([r.latency for r in results]) * 1e3
    t_first = min(r.t_arrival for r in results)
    t_last = max(r.t_done for r in results)
    return {
        "requests": len(results),
        "circuits_per_s": len(results) / (t_last - t_first) if t_last > t_first else float("nan"),
        "p50_ms": float(np.percentile(lat, 50)),
        "p99_ms": float(np.percentile(lat, 99)),
        "makespan_s": t_last - t_first,
    }
