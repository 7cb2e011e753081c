#!/usr/bin/env python3
"""Benchmark of the state-vector hot path on GB300.

One step = the whole path on the 28-qubit workload: reset to |0..0>, apply a
random layered circuit (n=28, depth 40, 1680 gates: fusion, pass planning and
the pass kernels), FP64 CDF + 1e5 shots from pre-drawn uniforms with the FP64
norm and a Z-string expectation taken from the same read of the state, then
reset to a seeded basis state and apply the 28-qubit QFT.  The complex64 state is 2 GiB, larger than the 129 MB L2, so every pass
streams from HBM.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  ``value`` is algorithmic HBM GB/s over the step (bytes
the path must move: 16 B per amplitude per pass, 8 B per amplitude per reset
and for the one readout read that builds the CDF and the norm and expectation
sums) divided by device time.  ``roofline`` refers
to the pass kernel, timed per launch with CUDA events on the state's stream.
``--impl reference`` times the complex128 CPU oracle on a bounded sample of the
same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

N_QUBITS = 28
DEPTH = 40
SEED = 2
SHOTS = 100_000
ZMASK = 0b1011  # <Z_0 Z_1 Z_3>
# precision 1: dense blocks as 3xTF32 tensor-core stage products, except on the
# light passes the planner puts on the CUDA-core register kernel (its per-pass
# estimate of both kernels' times); precision 2 puts every pass on the tensor cores
OPTS = dict(k_max=5, tile_qubits=12, low_qubits=5, precision=1, kernel_variant=0)
METRIC = "state-vector apply HBM GB/s vs peak"
SERVE_SMALL_MAX = 14  # requests up to this many qubits go to the batched kernel
# FP32 FMA peak: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def workload_name():
    return (f"random layered n={N_QUBITS} depth={DEPTH} + QFT-{N_QUBITS} on a seeded basis state; "
            f"FP64 norm, CDF and {SHOTS} shots; <Z> expectation")
# DRAM bytes (read + write) of one pass-kernel launch from an ncu capture of the
# current kernel, keyed by (n, tile qubits, low qubits, precision, kernel variant); see profiles/.
PASS_TRAFFIC_BYTES = {(28, 12, 5, 0, 0): 4238000000, (28, 12, 5, 1, 0): 4235000000, (28, 12, 5, 2, 0): 4235000000}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.remove(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def max_over_ranks(x: float, device) -> float:
    """The slowest rank's figure (every rank calls this; a no-op without a process group)."""
    import torch
    import torch.distributed as td
    if not (td.is_available() and td.is_initialized()) or td.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    td.all_reduce(t, op=td.ReduceOp.MAX)
    return float(t.item())


def job_value(bytes_per_step: float, steps: int, world: int, seconds: float) -> float:
    """Whole-job GB/s: every replica moves bytes_per_step per step; the job takes
    the slowest replica's time."""
    return world * bytes_per_step * steps / seconds / 1e9


def step_bytes(plan_rand, plan_qft, n):
    amps = float(1 << n)
    return plan_rand["bytes"] + plan_qft["bytes"] + 3 * 8.0 * amps  # 2 resets + one readout read


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2512_04216_gb300 import capi

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    n = N_QUBITS
    circ = W.random_layered(n, DEPTH, SEED)
    qft = W.qft(n)
    x = W.basis_index(n, SEED)
    opts = capi.make_opts(**OPTS)
    ir_r, keep_r = capi.to_ir(circ)
    ir_q, keep_q = capi.to_ir(qft)
    plan_r = capi.sv_plan_stats(n, circ, opts)
    plan_q = capi.sv_plan_stats(n, qft, opts)
    bytes_step = step_bytes(plan_r, plan_q, n)
    flops_pass_step = float(plan_r["flops"] + plan_q["flops"])

    stream = torch.cuda.Stream(dev)
    amps = torch.empty(1 << n, dtype=torch.complex64, device=dev)
    h = capi.sv_wrap(amps, n, capi.SV_C64, stream)
    u_host = W.shot_uniforms(SEED, SHOTS)
    u_dev = torch.as_tensor(u_host, device=dev)
    out_dev = torch.empty(SHOTS, dtype=torch.int64, device=dev)
    L = capi._L
    import ctypes

    ex, n2 = ctypes.c_double(), ctypes.c_double()

    def step_device():
        capi.sv_reset(h, 0)
        capi.sv_apply_circuit(h, ir_r, len(circ), opts)
        # draws, <Z_mask> and the norm from one read of the state
        capi._check(L.sv_sample_expect_z(h, u_dev.data_ptr(), SHOTS, out_dev.data_ptr(), None, 1, ZMASK,
                                         ctypes.byref(ex), ctypes.byref(n2)))
        capi.sv_reset(h, x)
        capi.sv_apply_circuit(h, ir_q, len(qft), opts)

    u_pin = torch.from_numpy(u_host).pin_memory()
    out_host = np.empty(SHOTS, dtype=np.uint64)
    nb = ctypes.c_uint64()

    def step_e2e():
        capi.sv_reset(h, 0)
        capi.sv_apply_circuit(h, ir_r, len(circ), opts)
        capi._check(L.sv_sample_expect_z(h, u_pin.data_ptr(), SHOTS, out_host.ctypes.data, ctypes.byref(nb), 0,
                                         ZMASK, ctypes.byref(ex), ctypes.byref(n2)))
        capi.sv_reset(h, x)
        capi.sv_apply_circuit(h, ir_q, len(qft), opts)
        capi.sv_synchronize(h)

    dist = world > 1
    if dist:
        import torch.distributed as td

    def barrier():
        if dist:
            td.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        step_device()
    barrier()

    # ---- device-timed steps (inputs resident in HBM) ----
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    capi.sv_profile_enable(h, True)
    capi.sv_profile_read(h)  # reset records
    launches0 = capi.sv_launch_count()
    with ClockSampler(local_rank) as clk:
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            step_device()
        ev1.record(stream)
        barrier()
    launches = capi.sv_launch_count() - launches0
    prof = capi.sv_profile_read(h)
    capi.sv_profile_enable(h, False)
    dev_ms = max_over_ranks(ev0.elapsed_time(ev1), dev)
    clocks = clk.summary()

    # ---- end-to-end steps through the public API, host buffers ----
    for _ in range(max(1, args.warmup // 2)):
        step_e2e()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step_e2e()
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dev)

    # parity spot check on the final state (QFT of |x>), outside the timed regions
    idx = np.array([0, 1, 12345, (1 << n) - 1], dtype=np.int64)
    got = np.array([capi_get(capi, h, int(i)) for i in idx])
    want = np.exp(2j * np.pi * ((x * idx) % (1 << n)) / (1 << n)) / math.sqrt(1 << n)
    spot_err = float(np.max(np.abs(got - want)))
    capi.sv_destroy(h)

    peak, peak_kind = peaks()
    # the pass kernels together: tensor-core and CUDA-core register passes (with
    # precision 1 the planner picks one per pass), one HBM pass over the state each
    recs = [prof[k] for k in ("pass_tc", "pass") if k in prof]
    pk = ({"launches": sum(r["launches"] for r in recs), "ms": sum(r["ms"] for r in recs),
           "bytes": sum(r["bytes"] for r in recs)} if recs else {"launches": 0, "ms": float("nan"), "bytes": 0.0})
    pass_s = pk["ms"] * 1e-3
    achieved = pk["bytes"] / pass_s / 1e9 if pk["launches"] else float("nan")
    achieved_tf = flops_pass_step * args.steps / pass_s / 1e12 if pk["launches"] else float("nan")
    # the pass kernels' lower bound is the larger of HBM time and FP32 FMA time
    alu_bound = flops_pass_step / (FP32_PEAK_TFLOPS * 1e12) > (pk["bytes"] / max(args.steps, 1)) / (peak * 1e9)
    if OPTS["precision"]:
        alu_bound = False  # tensor-core stage products: reported against HBM
    if alu_bound:
        roof = {"bound": "alu", "achieved": round(achieved_tf, 2), "peak": round(FP32_PEAK_TFLOPS, 1),
                "unit": "TFLOP/s", "frac": round(achieved_tf / FP32_PEAK_TFLOPS, 4),
                "peak_source": "derived (152 SMs x 128 FP32 FMA/clk x 2 x 2.07 GHz)"}
    else:
        roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "peak_source": peak_kind}
    roof.update({"kernel": "pass kernels (k_pass_tc and k_pass_reg launches together; one HBM pass over the state each)",
                 "traffic": PASS_TRAFFIC_BYTES.get((n, OPTS["tile_qubits"], OPTS["low_qubits"], OPTS["precision"],
                                                    OPTS.get("kernel_variant", 0))),
                 "algorithmic_bytes_per_launch": 16 * (1 << n),
                 "algorithmic_flops_per_step": flops_pass_step,
                 "hbm_GBps": round(achieved, 1), "hbm_frac": round(achieved / peak, 4),
                 "fp32_TFLOPs": round(achieved_tf, 2), "fp32_frac": round(achieved_tf / FP32_PEAK_TFLOPS, 4),
                 "avg_launch_ms": round(pk["ms"] / max(pk["launches"], 1), 4)})
    config = config_dict(world)
    # the default step's statistics are also stored for the reference arm; a
    # non-default run (other size or options) reports its own plan
    config["passes_per_step"] = plan_r["n_passes"] + plan_q["n_passes"]
    value = job_value(bytes_step, args.steps, world, dev_ms * 1e-3)
    e2e_val = job_value(bytes_step, args.steps, world, e2e_s)
    h2d = plan_r["upload_bytes"] + plan_q["upload_bytes"] + SHOTS * 8
    d2h = SHOTS * 8 + 8 + 2 * 8
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dev_ms / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64",
        "data": "synthetic (seeded random layered circuit, QFT, SplitMix64 uniforms)",
        "config": config,
        "roofline": roof,
        "kernels": {k: {"launches": v["launches"], "ms": round(v["ms"], 3),
                        "GB/s": round(v["bytes"] / (v["ms"] * 1e-3) / 1e9, 1) if v["ms"] > 0 and v["bytes"] else None,
                        "hbm_frac": round(v["bytes"] / (v["ms"] * 1e-3) / 1e9 / peak, 4)
                        if v["ms"] > 0 and v["bytes"] else None}
                    for k, v in prof.items()},
        "e2e": {"value": round(e2e_val, 1), "unit": "GB/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "ms_per_step": round(e2e_s * 1e3 / args.steps, 3)},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "spot_check_max_abs_err": spot_err,
    }
    return line


def capi_get(capi, h, i):
    out = np.empty(1, dtype=np.complex64)
    capi.sv_get_amplitudes(h, out, i, 1, False)
    return complex(out[0])


# Plan statistics of the default step (n=28 depth-40 random circuit + QFT-28 with
# OPTS): the reference arm reports them without loading the library;
# tests/test_bench_host.py checks them against the planner.
DEFAULT_PLAN = {"passes_per_step": 68, "bytes_step": 298500227072.0}


def oracle_gate_time(threads: int, reps: int = 3):
    """Seconds per gate of each kind in the step (U3 and CX of the random circuit;
    H, CP and SWAP of the QFT): the oracle applies a gate of each kind in turn to a
    2^28 complex128 state with `threads` threads, `reps` rounds, and each kind
    keeps its fastest time.  Returns ({kind: seconds}, threads used)."""
    import oracle
    o = oracle.default()
    o.set_threads(threads)
    used = o.max_threads()
    n = N_QUBITS
    circ = W.random_layered(n, DEPTH, SEED)
    qft = W.qft(n)
    pick = {}
    for g in circ + qft:
        pick.setdefault(g[0], g)
    psi = oracle.basis(n)
    psi = o.run(n, [pick["u3"]], psi)  # untimed: touches every page of the new state
    times = {}
    for _ in range(reps):
        for kind, g in pick.items():
            t0 = time.perf_counter()
            psi = o.run(n, [g], psi)
            times[kind] = min(times.get(kind, math.inf), time.perf_counter() - t0)
    del psi
    return times, used


def oracle_step_time(threads: int, measure_psi=None):
    """The oracle's time for one step, by gate kind: sum over kinds of (gates of
    that kind in the step) x (its measured per-gate time), plus the measured
    CDF + 1e5 draws, norm and <Z> on a 2^28 state (psi, or a fresh basis state).
    Returns (seconds, threads used, description)."""
    import oracle
    from collections import Counter
    n = N_QUBITS
    counts = Counter(g[0] for g in W.random_layered(n, DEPTH, SEED) + W.qft(n))
    per_gate, used = oracle_gate_time(threads, reps=3 if threads > 1 else 1)
    t_gates = sum(counts[k] * per_gate[k] for k in counts)
    o = oracle.default()
    o.set_threads(threads)
    psi = oracle.basis(n, W.basis_index(n, SEED)) if measure_psi is None else measure_psi
    t0 = time.perf_counter()
    o.sample(psi, W.shot_uniforms(SEED, SHOTS))
    o.norm2(psi)
    o.expect_z(psi, ZMASK)
    t_m = time.perf_counter() - t0
    del psi
    desc = (f"oracle (complex128, {used} thread{'s' if used > 1 else ''}) at n={n}: a gate of each kind "
            f"(fastest of {3 if threads > 1 else 1}) "
            f"({', '.join(f'{k} {per_gate[k]:.3f} s' for k in sorted(per_gate))}) times the step's "
            f"{sum(counts.values())} gates by kind, + measured CDF/{SHOTS} draws/norm/<Z> ({t_m:.2f} s)")
    return t_gates + t_m, used, desc


def oracle_config1_s() -> float:
    """The oracle on the small configuration in full (n=12 random layered depth 20,
    CDF and 1024 draws), one thread."""
    import oracle
    o = oracle.default()
    o.set_threads(1)
    t0 = time.perf_counter()
    psi = o.run(12, W.random_layered(12, 20, 1))
    o.sample(psi, W.shot_uniforms(1, 1024))
    return time.perf_counter() - t0


def cpu_baseline() -> dict:
    """The oracle as it stands on the host cores: all cores (the line's value)
    and one thread, each extrapolated from a by-kind gate sample of the step, and
    the small configuration timed in full."""
    bstep = DEFAULT_PLAN["bytes_step"]
    t_all, cores, desc = oracle_step_time(os.cpu_count() or 1)
    t_one, _, desc1 = oracle_step_time(1)
    return {"value": bstep / t_all / 1e9, "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": desc,
            "ms_per_step": t_all * 1e3,
            "single_thread": {"value": bstep / t_one / 1e9, "ms_per_step": t_one * 1e3, "sample": desc1},
            "config1_full_one_thread_ms": oracle_config1_s() * 1e3}


def config_dict(world: int) -> dict:
    """The workload description both arms print (plan statistics from DEFAULT_PLAN)."""
    n = N_QUBITS
    return {"workload": workload_name(), "n_qubits": n, "depth": DEPTH,
            "gates": len(W.random_layered(n, DEPTH, SEED)) + len(W.qft(n)),
            "shots": SHOTS, "fusion_k_max": OPTS["k_max"], "tile_qubits": OPTS["tile_qubits"], "low_qubits": OPTS["low_qubits"],
            "kernel_variant": OPTS.get("kernel_variant", 0), "precision": OPTS["precision"],
            "passes_per_step": DEFAULT_PLAN["passes_per_step"],
            "l2": f"inputs larger than L2 ({(8 << n) / 2**30:.3g} GiB state vs 129 MB L2)",
            "parallelism": f"replicas{world}"}


def run_reference(args):
    """The oracle arm: every step is a by-kind gate sample of the step at n=28 on
    all host cores plus the measured readout, extrapolated to the whole step."""
    bstep = DEFAULT_PLAN["bytes_step"]
    vals = []
    desc = threads = None
    for i in range(args.warmup + args.steps):
        t_step, threads, desc = oracle_step_time(os.cpu_count() or 1)
        if i >= args.warmup:
            vals.append(t_step)
    t = statistics.median(vals)
    v = bstep / t / 1e9
    world = int(os.environ.get("WORLD_SIZE", "1"))
    return {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
        "config": config_dict(world),
        "cpu_baseline": {"value": v, "unit": "GB/s", "cores": threads, "kind": "oracle", "sample": desc},
        "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_batch_mode(args):
    """Config: many independent random layered circuits (n ~ U{10..20},
    depth ~ U{10..60}, 4096 shots each) in one persistent graph-captured launch,
    autotuned on the batch itself, against the plain one-circuit-at-a-time
    path timed on a sample and scaled to the batch."""
    import torch
    from paper_2512_04216_gb300 import Batch, StateVector, capi
    count = args.batch_circuits
    mix = W.batch_mix(count, 3)
    circs = [W.random_layered(n, d, s) for n, d, s in mix]
    ns = [m[0] for m in mix]
    shots = [4096] * count
    seeds = [m[2] for m in mix]
    # tuned on the batch itself: a sample too small to fill the GPU times one large
    # circuit's latency, not the batch's throughput
    best, best_ms = capi.sv_batch_autotune(capi.BatchArgs(circs, ns, shots, seeds), reps=1)
    b = Batch(circs, ns, shots, seeds, k_max=best.k_max, tile_qubits=best.tile_qubits)
    for _ in range(args.warmup):
        b.launch()
    b.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = capi.sv_launch_count()
    ev0.record()
    for _ in range(args.steps):
        b.launch()
    b.synchronize()
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    stats = b.stats()
    b.close()
    # plain path: each circuit alone (create, apply, sample, destroy), on a sample
    psample = list(range(0, count, max(1, count // 64)))
    t0 = time.perf_counter()
    for i in psample:
        s = StateVector(ns[i])
        s.apply(circs[i])
        s.sample(shots[i], seeds[i])
        s.close()
    plain_s = (time.perf_counter() - t0) * count / len(psample)
    return {
        "metric": "batched circuits/s", "value": count / (ms * 1e-3), "unit": "circuits/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
        "config": {"workload": f"{count} random layered circuits, n~U{{10..20}}, depth~U{{10..60}}, 4096 shots each, "
                               "one persistent launch under a CUDA graph",
                   "autotuned": {"k_max": best.k_max, "tile_qubits": best.tile_qubits, "sample_ms": best_ms},
                   "arena_passes": stats["passes"]},
        "plain_path": {"circuits_per_s": count / plain_s, "sample": f"{len(psample)} circuits, scaled"},
        "speedup_vs_plain": (count / (ms * 1e-3)) / (count / plain_s),
        "gpu_launches": int(capi.sv_launch_count() - launches0),
    }


def run_dynamic_mode(args):
    """Per-shot trajectories with mid-circuit measurement (§III-B): a 28-qubit
    random prefix (depth 20) runs once; each trajectory clones the state,
    measures qubits 3 and 17, resets qubit 25, applies a depth-2 suffix and
    draws one bitstring.  Reports trajectories/s and the collapse kernel's HBM
    rate (16 B per amplitude: read and write once)."""
    import torch
    from paper_2512_04216_gb300 import StateVector, capi
    n = 28
    traj = 8
    prefix, suffix = W.random_layered(n, 20, 31), W.random_layered(n, 2, 32)
    s = StateVector(n)
    s.apply(prefix)
    torch.cuda.synchronize()
    u = W.shot_uniforms(33, 4 * traj * (args.steps + args.warmup))
    peak, peak_kind = peaks()
    prof_tot = {}

    def trajectory(k, prof):
        c = s.clone()
        if prof:
            capi.sv_profile_enable(c.h, True)
        c.measure(3, float(u[4 * k]))
        c.measure(17, float(u[4 * k + 1]))
        c.reset_qubit(25, float(u[4 * k + 2]))
        c.apply(suffix)
        c.sample_uniforms(np.array([u[4 * k + 3]]))
        if prof:
            for name, v in capi.sv_profile_read(c.h).items():
                t = prof_tot.setdefault(name, {"launches": 0, "ms": 0.0, "bytes": 0.0})
                for key in t:
                    t[key] += v[key]
        c.close()

    k = 0
    for _ in range(args.warmup):
        for _ in range(traj):
            trajectory(k, False)
            k += 1
    torch.cuda.synchronize()
    launches0 = capi.sv_launch_count()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for _ in range(traj):
            trajectory(k, True)
            k += 1
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    s.close()
    col = prof_tot.get("collapse", {"launches": 0, "ms": float("nan"), "bytes": 0.0})
    col_gbs = col["bytes"] / (col["ms"] * 1e-3) / 1e9 if col["launches"] else float("nan")
    return {
        "metric": "mid-circuit trajectories/s", "value": args.steps * traj / dt, "unit": "trajectories/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
        "config": {"workload": f"n={n} random prefix depth 20 once; per trajectory: clone (2 GiB), measure 2 qubits, "
                               f"reset 1, suffix depth 2, 1 shot; {traj} trajectories per step"},
        "roofline": {"bound": "hbm", "kernel": "k_collapse", "achieved": round(col_gbs, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(col_gbs / peak, 4), "peak_source": peak_kind,
                     "algorithmic_bytes_per_launch": 16 * (1 << n), "traffic": None},
        "kernels": {k2: {"launches": v["launches"], "ms": round(v["ms"], 3)} for k2, v in prof_tot.items()},
        "gpu_launches": int(capi.sv_launch_count() - launches0),
    }


def run_pblock_mode(args):
    """Distributed-register pattern (§III-E): two 14-qubit hosts, each with one
    communication qubit, are simulated apart, merged into one 28-qubit register
    (2 GiB), entangled through the communication pair, the communication qubits
    measured and taken out (27 then 26 qubits).  Reports steps/s and the merge
    and take kernels' HBM rates (CUDA events on the states' stream; the take
    interval includes its mass reduction, 8 B per amplitude read)."""
    import torch
    from paper_2512_04216_gb300 import StateVector, capi
    na = nb = 14
    ca, cb = W.random_layered(na, 10, 41), W.random_layered(nb, 10, 42)
    peak, peak_kind = peaks()
    prof_tot = {}

    def step(k, prof):
        a, b = StateVector(na), StateVector(nb)
        a.apply(ca)
        b.apply(cb)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record()
        m = a.merge(b)
        ev[1].record()
        m.apply([("h", (na - 1,), ()), ("cx", (na - 1, na + nb - 1), ()), ("cx", (0, na - 1), ())])
        m.measure(na - 1, 0.25 + 0.5 * (k % 2))
        m.measure(na + nb - 1, 0.6)
        ev[2].record()
        m2, _ = m.take_qubit(na + nb - 1)
        ev[3].record()
        m3, _ = m2.take_qubit(na - 1)
        torch.cuda.synchronize()
        if prof:
            for name, (e0, e1, nbytes) in {"merge": (ev[0], ev[1], 8.0 * (1 << (na + nb))),
                                           "take": (ev[2], ev[3], 8.0 * (1 << (na + nb)))}.items():
                t = prof_tot.setdefault(name, {"launches": 0, "ms": 0.0, "bytes": 0.0})
                t["launches"] += 1
                t["ms"] += e0.elapsed_time(e1)
                t["bytes"] += nbytes
        for st in (a, b, m, m2, m3):
            st.close()

    for k in range(args.warmup):
        step(k, False)
    torch.cuda.synchronize()
    launches0 = capi.sv_launch_count()
    t0 = time.perf_counter()
    for k in range(args.steps):
        step(k, True)
    dt = time.perf_counter() - t0
    rates = {k: (v["bytes"] / (v["ms"] * 1e-3) / 1e9 if v["ms"] > 0 and v["bytes"] else None)
             for k, v in prof_tot.items()}
    mg = rates.get("merge") or float("nan")
    return {
        "metric": "p-block steps/s", "value": args.steps / dt, "unit": "steps/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
        "config": {"workload": "two 14-qubit hosts (depth 10) merged to 28 qubits, communication pair "
                               "entangled, measured and taken out; state allocation inside the step"},
        "roofline": {"bound": "hbm", "kernel": "k_kron", "achieved": round(mg, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(mg / peak, 4), "peak_source": peak_kind,
                     "algorithmic_bytes_per_launch": 8 * (1 << (na + nb)), "traffic": None},
        "kernels": {k: {"launches": v["launches"], "ms": round(v["ms"], 3),
                        "GB/s": round(rates[k], 1) if rates[k] else None} for k, v in prof_tot.items()},
        "gpu_launches": int(capi.sv_launch_count() - launches0),
    }


def run_alias_mode(args):
    """Alias sampling (§III-C) against the CDF sampler on the 28-qubit bench
    state (random layered depth 40): per step, one alias-table build and S
    draws, and one CDF build and S draws, for S in 1e4, 1e6, 1e8 (device output
    buffers).  Kernel times from CUDA events on the state's stream; the
    crossover is the shot count above which build + draws is cheaper with the
    alias table."""
    import torch
    from paper_2512_04216_gb300 import StateVector, capi
    n = N_QUBITS
    N = 1 << n
    s = StateVector(n)
    s.apply(W.random_layered(n, DEPTH, 2))
    shots_list = [10_000, 1_000_000, 100_000_000]
    out = torch.empty(max(shots_list), dtype=torch.int64, device=s.device)
    peak, peak_kind = peaks()

    def one(prof_on, k):
        s.profile(prof_on)
        for S in shots_list:
            s.alias_build()
            capi.sv_alias_sample(s.h, S, 1000 + k, out, True)
            capi.sv_sample(s.h, S, 2000 + k, out, True)
        torch.cuda.synchronize()
        s.profile(False)

    for k in range(args.warmup):
        one(False, k)
    s.profile_read()
    launches0 = capi.sv_launch_count()
    t0 = time.perf_counter()
    for k in range(args.steps):
        one(True, k)
    dt = time.perf_counter() - t0
    st = s.profile_read()
    steps = args.steps
    per = {k: v["ms"] / v["launches"] for k, v in st.items() if v["launches"]}
    build_ms = per["alias_build"] + per["reduce"]
    cdf_ms = per["cdf"]
    # draws: three shot counts per step, separate launches; per-shot cost from the 1e8 launches
    S_tot = sum(shots_list)
    alias_ns = st["alias_sample"]["ms"] / steps / S_tot * 1e6
    cdf_ns = st["sample"]["ms"] / steps / S_tot * 1e6
    cross = (build_ms - cdf_ms) / ((cdf_ns - alias_ns) * 1e-6) if cdf_ns > alias_ns else None
    build_bytes = st["alias_build"]["bytes"] / st["alias_build"]["launches"]
    build_gbs = build_bytes / (per["alias_build"] * 1e-3) / 1e9
    s.close()
    return {
        "metric": "alias vs CDF sampler, 28-qubit state", "value": alias_ns, "unit": "ns per shot (alias draws)",
        "n_gpus": 1, "steps": steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / steps,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "c64/f64/u64",
        "data": "synthetic",
        "config": {"workload": f"random layered n={n} depth={DEPTH}; per step an alias build and a CDF build, "
                               f"each with 1e4, 1e6 and 1e8 draws (device output)"},
        "alias": {"build_ms": round(build_ms, 3), "table_ms": round(per["alias_build"], 3),
                  "norm_ms": round(per["reduce"], 3), "ns_per_shot": round(alias_ns, 4)},
        "cdf": {"build_ms": round(cdf_ms, 3), "ns_per_shot": round(cdf_ns, 4)},
        "crossover_shots": round(cross) if cross else None,
        "roofline": {"bound": "hbm", "kernel": "alias table build (6 kernels)", "achieved": round(build_gbs, 1),
                     "peak": peak, "unit": "GB/s", "frac": round(build_gbs / peak, 4), "peak_source": peak_kind,
                     "algorithmic_bytes_per_launch": build_bytes, "traffic": None},
        "gpu_launches": int(capi.sv_launch_count() - launches0),
    }


LARGE_QUBITS = 25  # requests from here on bound both serving paths by their device time
SERVE_TC_FROM = 24  # both serving paths apply requests from here on with tensor-core passes


def serving_sweep(count: int, factors, small_max: int) -> dict:
    """Poisson stream of random layered circuits (n geometric-skewed on 8..30,
    mean ~16; depth ~ U{10..100}; 1000 shots or a Z-string mask), served by the
    continuous-batching loop and by the plain one-circuit-at-a-time path at
    rates `factors` x the plain path's capacity.  Also the Amdahl ceiling of the
    served/plain circuits/s ratio: the plain makespan of the whole stream over
    the plain time of its >= 25-qubit requests, whose device work (the same pass
    kernels on both paths, each saturating the GPU) no scheduling removes."""
    from paper_2512_04216_gb300 import serve
    specs0 = W.serving_requests(count, 4, 1.0)
    reqs0 = serve.make_requests(specs0, W.random_layered)
    for r in reqs0:
        r.t = 0.0
    res0 = serve.run_plain(reqs0, tc_from_qubits=SERVE_TC_FROM)
    cap = serve.summarize(res0)
    n_of = {r.id: r.n for r in reqs0}
    large_s = sum(r.t_done - r.t_start for r in res0 if n_of[r.id] >= LARGE_QUBITS)
    n_large = sum(1 for r in reqs0 if r.n >= LARGE_QUBITS)
    out = {"requests_per_point": count, "small_max_qubits": small_max, "tensor_core_from_qubits": SERVE_TC_FROM,
           "plain_capacity_circuits_per_s": cap["circuits_per_s"],
           "amdahl_ceiling": {"ratio": cap["makespan_s"] / large_s if large_s > 0 else None,
                              "plain_makespan_s": cap["makespan_s"], "large_requests": n_large,
                              "large_qubits_from": LARGE_QUBITS, "large_plain_s": large_s},
           "points": []}
    for f in factors:
        rate = f * cap["circuits_per_s"]
        specs = W.serving_requests(count, 4, rate)
        reqs = serve.make_requests(specs, W.random_layered)
        res = serve.Server(small_max_qubits=small_max, tc_from_qubits=SERVE_TC_FROM).run(reqs)
        srv = serve.summarize(res)
        srv["batched_requests"] = sum(1 for r in res if r.path == "batch")
        pl = serve.summarize(serve.run_plain(reqs, tc_from_qubits=SERVE_TC_FROM))
        out["points"].append({"rate_factor": f, "rate_hz": rate, "served": srv, "plain": pl,
                              "circuits_per_s_ratio": srv["circuits_per_s"] / pl["circuits_per_s"]})
    return out


def run_serve_mode(args):
    """Config: the serving stream (serving_sweep) at every --rate-factors point,
    then the runtime model's held-out accuracy and shortest-predicted-first admission."""
    from paper_2512_04216_gb300 import serve
    count = args.requests
    out = serving_sweep(count, [float(x) for x in args.rate_factors.split(",")], args.serve_small_max)
    plain_cap = out["plain_capacity_circuits_per_s"]
    # runtime model (Eq. 1) calibrated on this GPU: held-out accuracy, and the
    # highest-rate point again with shortest-predicted-first admission
    from paper_2512_04216_gb300 import costmodel
    t0 = time.perf_counter()
    model = costmodel.calibrate(W.calibration_circuits, ns=tuple(range(8, 31, 2)), reps=1)
    cal_s = time.perf_counter() - t0
    import torch
    from paper_2512_04216_gb300 import StateVector, capi
    errs = []
    for n, d, sd in ((11, 40, 1), (15, 70, 2), (19, 30, 3), (23, 50, 4), (27, 20, 5)):
        c = W.random_layered(n, d, 900 + sd)
        s = StateVector(n)
        ir, keep = capi.to_ir(c)
        capi.sv_apply_circuit(s.h, ir, len(c))  # warm, as in the calibration
        best = math.inf
        for _ in range(2):
            s.reset(0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s.stream)
            capi.sv_apply_circuit(s.h, ir, len(c))
            e1.record(s.stream)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        s.close()
        errs.append(abs(model.predict_ms(n, c) - best) / best)
    f = float(args.rate_factors.split(",")[-1])
    specs = W.serving_requests(count, 4, f * plain_cap)
    reqs = serve.make_requests(specs, W.random_layered)
    spt = serve.summarize(serve.Server(small_max_qubits=args.serve_small_max, cost_model=model,
                                       tc_from_qubits=SERVE_TC_FROM).run(reqs))
    out["cost_model"] = {"calibration_s": cal_s, "held_out_abs_rel_err": [round(e, 3) for e in errs],
                         "rate_factor": f, "served_shortest_predicted_first": spt}
    best = max(p["circuits_per_s_ratio"] for p in out["points"])
    return {"metric": "mixed-stream circuits/s & p99 vs plain path", "value": best,
            "unit": "x plain circuits/s", "n_gpus": 1, "higher_is_better": True, "vs_baseline": None,
            "dtype": "c64", "data": "synthetic",
            "config": {"workload": f"{count} Poisson requests per point, n geometric on 8..30 (mean ~16), "
                                   "depth U{10..100}, 1000 shots or <Z>"}, "serving": out}


def main():
    global N_QUBITS, DEPTH, SHOTS
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n-qubits", type=int, default=N_QUBITS,
                    help="smaller states for profiling captures (the bench line uses 28)")
    ap.add_argument("--depth", type=int, default=DEPTH)
    ap.add_argument("--tile-qubits", type=int, default=OPTS["tile_qubits"])
    ap.add_argument("--low-qubits", type=int, default=OPTS["low_qubits"],
                    help="qubits every tile holds (HBM runs of 2^c amplitudes)")
    ap.add_argument("--k-max", type=int, default=OPTS["k_max"])
    ap.add_argument("--kernel-variant", type=int, default=0)
    ap.add_argument("--precision", type=int, default=OPTS["precision"],
                    help="0: FP32 CUDA cores; 1: 3xTF32 tensor-core stage products")
    ap.add_argument("--workload", choices=["statevector", "large", "batch", "serve", "dynamic", "pblock", "alias"],
                    default="statevector",
                    help="statevector: the bench line; large: the 34-qubit (128 GiB) single state, "
                         "depth 30, 1e6 shots; batch / serve: the batched and serving patterns; "
                         "dynamic: per-shot trajectories with mid-circuit measurement; "
                         "pblock: merged registers with communication qubits; "
                         "alias: alias-table sampling against the CDF sampler")
    ap.add_argument("--batch-circuits", type=int, default=4096)
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--rate-factors", default="0.5,1,2,4")
    ap.add_argument("--serve-small-max", type=int, default=SERVE_SMALL_MAX,
                    help="largest request (qubits) the server sends to the batched kernel")
    ap.add_argument("--no-serving", action="store_true",
                    help="leave the serving sweep out of the bench line (profiling runs)")
    args = ap.parse_args()
    N_QUBITS, DEPTH = args.n_qubits, args.depth
    if args.workload == "large":
        N_QUBITS, DEPTH, SHOTS = 34, 30, 1_000_000
        args.no_cpu_baseline = True  # the complex128 oracle would need 256 GiB of host memory
    OPTS.update(tile_qubits=args.tile_qubits, low_qubits=args.low_qubits, k_max=args.k_max,
                kernel_variant=args.kernel_variant,
                precision=args.precision)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    if args.workload in ("batch", "serve", "dynamic", "pblock", "alias"):
        if rank == 0:
            fn = {"batch": run_batch_mode, "serve": run_serve_mode, "dynamic": run_dynamic_mode,
                  "pblock": run_pblock_mode, "alias": run_alias_mode}[args.workload]
            print(json.dumps(fn(args)), flush=True)
        return

    if world > 1:
        import torch
        import torch.distributed as td
        torch.cuda.set_device(local_rank)
        td.init_process_group("nccl")
    line = run_ours(args, rank, world, local_rank)
    if rank == 0 and world == 1 and not args.no_serving:
        # the metric's second half: mixed-stream circuits/s and p50/p99 against the
        # plain path, bounded to 200 requests at 1x and 4x the plain capacity
        line["serving"] = serving_sweep(200, (1.0, 4.0), args.serve_small_max)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as td
        td.destroy_process_group()


if __name__ == "__main__":
    main()
