"""The host planner against gate-by-gate application (CPU only).

tests/plan_semantics/plan_check.cpp compiles the planner source with the host
compiler, fuses a whole circuit into one pass (all qubits in the tile), applies
the resulting dense blocks and phase terms -- and the SWAP relabeling of
register passes -- to a random complex128 state, and compares with applying the
circuit's gates one at a time.  Covers register-pass fusion (two-qubit phase
terms, relabeling, blocks kept open past queued diagonal gates) and the
shared-memory pass's fusion, at fusion widths 2 and 5.

tests/plan_semantics/plan_exec.cpp goes further: it plans with build_plan and
executes the packed register-stage and tensor-core passes the way the kernels
read their records (load rows, stage thread bits and swizzled exchange offsets,
register-position matrices or stage products, phase classes, the store's qubit
map), so the packing is checked on the host too."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2512_04216_gb300", "csrc")


def _cuda_include():
    for base in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if base and os.path.exists(os.path.join(base, "include", "cuda_runtime.h")):
            return os.path.join(base, "include")
    nvcc = shutil.which("nvcc")
    if nvcc:
        inc = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "include")
        if os.path.exists(os.path.join(inc, "cuda_runtime.h")):
            return inc
    return None


def _compile(tmp_path_factory, name):
    inc = _cuda_include()
    if inc is None or shutil.which("g++") is None:
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("plan") / name)
    subprocess.run(["g++", "-O2", "-std=c++17", "-w", f"-I{inc}", f"-I{CSRC}", "-o", exe,
                    os.path.join(HERE, "plan_semantics", name + ".cpp")], check=True)
    return exe


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    return _compile(tmp_path_factory, "plan_check")


@pytest.fixture(scope="module")
def executor(tmp_path_factory):
    return _compile(tmp_path_factory, "plan_exec")


def _encode(n, circuit):
    """kind nq qubits p0 p1 p2 per gate; a UNITARY gate's parameter is its
    matrix, written after three zeros as row-major (re, im) pairs."""
    from paper_2512_04216_gb300 import capi  # gate kind numbers only (no library call)
    lines = [f"{n} {len(circuit)}"]
    for name, qs, ps in circuit:
        if name == "unitary":
            m = np.asarray(ps[0], dtype=np.complex128).reshape(-1)
            flat = np.stack([m.real, m.imag], axis=1).reshape(-1)
            lines.append(" ".join(map(str, [capi.GATE_KIND[name], len(qs), *qs, 0.0, 0.0, 0.0]))
                         + " " + " ".join(repr(float(x)) for x in flat))
            continue
        ps = list(ps) + [0.0] * (3 - len(ps))
        lines.append(" ".join(map(str, [capi.GATE_KIND[name], len(qs), *qs, *ps[:3]])))
    return "\n".join(lines) + "\n"


def _interleaved(n, seed):
    import numpy as np
    rng = np.random.default_rng(seed)
    c = []
    for _ in range(60):
        a, b = (int(x) for x in rng.choice(n, 2, replace=False))
        kind = rng.integers(0, 5)
        if kind == 0:
            c.append(("h", (a,), ()))
        elif kind == 1:
            c.append(("cp", (a, b), (float(rng.uniform(0, 6.3)),)))
        elif kind == 2:
            c.append(("cx", (a, b), ()))
        elif kind == 3:
            c.append(("rz", (a,), (float(rng.uniform(0, 6.3)),)))
        else:
            c.append(("u3", (a,), tuple(float(x) for x in rng.uniform(0, 6.3, 3))))
    return c


CASES = ([("qft", 8, W.qft(8)), ("qft", 10, W.qft(10)), ("ghz", 9, W.ghz(9)),
          ("random_layered", 8, W.random_layered(8, 6, 1)), ("random_layered", 10, W.random_layered(10, 5, 2))]
         + [("gate_soup", 8, W.random_gate_soup(8, 120, s)) for s in range(8)]
         + [("interleaved", 7, _interleaved(7, s)) for s in range(6)])


@pytest.mark.parametrize("pairs,kmax", [(1, 2), (1, 5), (0, 2), (0, 5)])
def test_fused_pass_equals_gates(checker, pairs, kmax):
    bad = []
    for name, n, c in CASES:
        r = subprocess.run([checker, str(pairs), str(kmax)], input=_encode(n, c), capture_output=True, text=True)
        if r.returncode != 0:
            bad.append(f"{name} n={n}: {r.stdout.strip()} {r.stderr.strip()[:200]}")
    assert not bad, bad


def _wide_unitary_circuit(n, seed):
    """Random layers with 5-qubit UNITARY gates among them (a pass holding such
    a block takes 5-qubit tensor-core stages)."""
    rng = np.random.default_rng(seed)
    circ = W.random_layered(n, 4, seed)
    for _ in range(3):
        qs = tuple(int(x) for x in rng.choice(n, 5, replace=False))
        z = rng.standard_normal((32, 32)) + 1j * rng.standard_normal((32, 32))
        u, _ = np.linalg.qr(z)
        circ.insert(int(rng.integers(0, len(circ) + 1)), ("unitary", qs, (u,)))
    return circ


EXEC_CASES = ([("qft", 13, W.qft(13)), ("qft", 14, W.qft(14)), ("ghz", 14, W.ghz(14)),
               ("random_layered", 14, W.random_layered(14, 12, 3)), ("random_layered", 12, W.random_layered(12, 8, 4))]
              + [("gate_soup", 13, W.random_gate_soup(13, 160, s)) for s in range(4)]
              + [("interleaved", 12, _interleaved(12, s)) for s in range(3)])
WIDE_CASES = [("wide_unitary", 13, _wide_unitary_circuit(13, s)) for s in range(2)]


@pytest.mark.parametrize("k_max,T,c,variant", [(2, 12, 5, 0), (5, 12, 5, 0), (4, 11, 5, 2), (2, 10, 5, 0),
                                               (2, 12, 4, 0), (3, 12, 5, 1), (5, 10, 3, 1)])
def test_packed_passes_equal_gates(executor, k_max, T, c, variant):
    """Register passes (variants 0 and 2; k_max 5 mixes in shared-memory passes
    for 5-qubit blocks) and shared-memory passes (variant 1)."""
    bad = []
    for name, n, circ in EXEC_CASES:
        r = subprocess.run([executor, str(k_max), str(T), str(c), str(variant)], input=_encode(n, circ),
                           capture_output=True, text=True)
        if r.returncode != 0:
            bad.append(f"{name} n={n}: rc={r.returncode} {r.stdout.strip()}")
    assert not bad, bad


@pytest.mark.parametrize("k_max,T,c,variant", [(4, 12, 5, 0), (4, 11, 5, 0), (2, 13, 5, 0), (5, 12, 4, 0),
                                               (4, 11, 3, 0), (5, 12, 5, 2), (5, 13, 5, 2), (3, 12, 4, 2)])
def test_packed_tensor_core_passes_equal_gates(executor, k_max, T, c, variant):
    """Tensor-core passes: each stage's dense blocks folded into one 16x16
    product (32x32 with 5-qubit stages: variant 2, or a pass holding a
    5-qubit block), the real embedding B, phase ops after it, no store-only
    stage (the last stage stores whatever bits it holds), executed from the
    packed records against gate-by-gate application."""
    bad, n_tc = [], 0
    for name, n, circ in EXEC_CASES + WIDE_CASES:
        r = subprocess.run([executor, str(k_max), str(T), str(c), str(variant), "0", "2"], input=_encode(n, circ),
                           capture_output=True, text=True)
        if r.returncode != 0:
            bad.append(f"{name} n={n}: rc={r.returncode} {r.stdout.strip()}")
        elif " tensor-core " in r.stdout:
            n_tc += int(r.stdout.split(" tensor-core ")[1].split()[0])
    assert not bad, bad
    assert n_tc > 0


def test_mixed_precision_passes_equal_gates(executor):
    """Precision 1: the planner's per-pass choice puts light passes on the
    CUDA-core register kernel (SWAPs folded into the store) and the rest on
    the tensor cores; the mixed plans, streamed in chunks or whole, still equal
    gate-by-gate application, and both kinds occur."""
    bad, kinds = [], set()
    circs = [("qft", 16, W.qft(16)), ("random_layered", 18, W.random_layered(18, 12, 5)),
             ("qft_after_layers", 16, W.random_layered(16, 6, 6) + W.qft(16))]
    for name, n, circ in circs:
        for chunk in ("0", "2"):
            r = subprocess.run([executor, "5", "12", "5", "0", chunk, "1"], input=_encode(n, circ),
                               capture_output=True, text=True)
            if r.returncode != 0:
                bad.append(f"{name} n={n} chunk={chunk}: rc={r.returncode} {r.stdout.strip()}")
            if "kinds:" in r.stdout:
                kinds.update(r.stdout.split("kinds:")[1].split())
    assert not bad, bad
    assert {"1", "2"} <= kinds, kinds


@pytest.mark.parametrize("chunk", [1, 2, 3])
def test_streamed_plan_chunks_compose(executor, chunk):
    """Planning a few passes at a time (as sv_apply_circuit streams its plan)
    gives chunks whose passes, run in order, still equal the circuit."""
    bad = []
    for name, n, circ in EXEC_CASES[:6]:
        r = subprocess.run([executor, "2", "12", "5", "0", str(chunk)], input=_encode(n, circ),
                           capture_output=True, text=True)
        if r.returncode != 0:
            bad.append(f"{name} n={n}: rc={r.returncode} {r.stdout.strip()}")
    assert not bad, bad
