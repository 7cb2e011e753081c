"""bench.py host logic (CPU): the plan statistics the reference arm reports
without loading the library match the planner, and the reference arm (the
oracle timed on the host) runs without importing the product package."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_default_plan_constants_match_the_planner():
    sys.path.insert(0, ROOT)
    import bench
    import workloads as W
    from paper_2512_04216_gb300 import capi
    n = bench.N_QUBITS
    opts = capi.make_opts(**bench.OPTS)
    pr = capi.sv_plan_stats(n, W.random_layered(n, bench.DEPTH, bench.SEED), opts)
    pq = capi.sv_plan_stats(n, W.qft(n), opts)
    assert pr["n_passes"] + pq["n_passes"] == bench.DEFAULT_PLAN["passes_per_step"]
    assert bench.step_bytes(pr, pq, n) == bench.DEFAULT_PLAN["bytes_step"]


def test_reference_arm_runs_without_the_product_library():
    code = ("import runpy, sys; sys.argv = ['bench.py', '--impl', 'reference', '--n-qubits', '10', "
            "'--steps', '1', '--warmup', '0']; runpy.run_path('bench.py', run_name='__main__'); "
            "print('LOADED', any(m.startswith('paper_2512_04216_gb300') for m in sys.modules))")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = r.stdout.strip().splitlines()
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["config"]["parallelism"] == "replicas1"
    assert lines[-1] == "LOADED False"
