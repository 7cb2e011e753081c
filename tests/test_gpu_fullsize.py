"""Parity at the benchmark's sizes (GPU required), through the C-ABI.

* n = 28, the benchmark's random layered circuit (depth 40) with the
  benchmark's plan options and its 1e5 pre-drawn uniforms: the GPU's draws
  against the oracle's sampler run on the GPU's own final state (promoted to
  complex128).  At this size the device CDF scan runs over 2^16 blocks of 4096
  amplitudes in 32 segments; the draws must be identical except those the
  oracle flags within 1e-9 of a CDF boundary.
* n = 24, the same circuit family at depth 40 with k_max = 5, T = 12, c = 5, on
  the CUDA-core path and on the tensor-core path: every amplitude against the
  oracle's complex128 state (|a_gpu - a_oracle| <= 1e-5, fidelity >= 1 - 1e-6),
  and 1e5 draws against the oracle's own state, mismatches allowed only within
  delta = max_i |C_gpu_i - C_oracle_i| + 1e-9 of a boundary.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

AMP_TOL = 1e-5
FID_TOL = 1e-6


@pytest.fixture(scope="module")
def sv():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2512_04216_gb300 as P
    return P


def test_sampler_parity_28_bench(sv):
    import bench
    n = bench.N_QUBITS
    s = sv.StateVector(n)
    s.apply(W.random_layered(n, bench.DEPTH, bench.SEED), **bench.OPTS)
    u = W.shot_uniforms(bench.SEED, bench.SHOTS)
    x_gpu, nb_gpu = s.sample_uniforms(u)
    g = s.amplitudes()
    s.close()
    x_or, bnd, nb_or = oracle.sample(g, u)
    diff = x_gpu.astype(np.int64) != x_or.astype(np.int64)
    assert np.all(bnd[diff] == 1), f"{int(diff.sum())} mismatches, {nb_or} boundary draws"
    # the draws cover the state: more than half of the shots are distinct outcomes
    assert np.unique(x_gpu).size > bench.SHOTS // 2


@pytest.fixture(scope="module")
def ref24():
    n = 24
    circ = W.random_layered(n, 40, 24)
    return n, circ, oracle.run(n, circ)


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_full_state_parity_24(sv, ref24, precision):
    n, circ, ref = ref24
    s = sv.StateVector(n)
    s.apply(circ, k_max=5, tile_qubits=12, low_qubits=5, precision=precision)
    info = sv.capi.sv_plan_stats(n, circ, sv.capi.make_opts(5, 12, 5, precision))
    if precision == 2:
        assert info["passes_by_kind"][2] == info["n_passes"]  # every pass on the tensor cores
    elif precision == 1:
        assert info["passes_by_kind"][2] > 0  # the planner's per-pass choice
    u = W.shot_uniforms(24, 100_000)
    x_gpu, _ = s.sample_uniforms(u)
    g = s.amplitudes().astype(np.complex128)
    s.close()
    err = float(np.max(np.abs(g - ref)))
    fid = oracle.fidelity(ref, g)
    assert err <= AMP_TOL, f"precision {precision}: max abs err {err:.3e}"
    assert fid >= 1 - FID_TOL, f"precision {precision}: fidelity {fid!r}"
    C_gpu, C_ref = oracle.cdf(g), oracle.cdf(ref)
    delta = float(np.max(np.abs(C_gpu - C_ref))) + 1e-9
    x_ref, bnd_ref, _ = oracle.sample_cdf(C_ref, u, eps=delta)
    diff = x_gpu.astype(np.int64) != x_ref.astype(np.int64)
    assert np.all(bnd_ref[diff] == 1), f"{int(diff.sum())} mismatches beyond delta={delta:.2e}"
