"""Batched mode: every circuit of a mixed batch against the complex128 oracle;
samples against the oracle's draws on the same final state (identical except
draws within 1e-9 of a CDF boundary); the graph replays deterministically."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

AMP_TOL = 1e-5
FID_TOL = 1e-6


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    import paper_2512_04216_gb300 as P
    return P


def _mix(count, seed, n_lo=10, n_hi=20, d_lo=4, d_hi=12):
    mix = W.batch_mix(count, seed, n_lo, n_hi, d_lo, d_hi)
    circs = [W.random_layered(n, d, s) for n, d, s in mix]
    return mix, circs


@pytest.mark.parametrize("k_max,T", [(2, 13), (1, 11), (3, 12)])
def test_batch_matches_oracle(P, k_max, T):
    mix, circs = _mix(24, 3, d_hi=10)
    ns = [m[0] for m in mix]
    shots = [512] * len(mix)
    seeds = [1000 + i for i in range(len(mix))]
    b = P.Batch(circs, ns, shots, seeds, k_max=k_max, tile_qubits=T, keep_states=True)
    b.launch()
    b.synchronize()
    for i, (n, d, s) in enumerate(mix):
        g = b.amplitudes(i).astype(np.complex128)
        ref = oracle.run(n, circs[i])
        err = float(np.max(np.abs(g - ref)))
        assert err <= AMP_TOL, (i, n, err)
        assert oracle.fidelity(ref, g) >= 1 - FID_TOL
        x = b.samples(i)
        xo, bnd, _ = oracle.sample(g, W.shot_uniforms(seeds[i], shots[i]))
        bad = (x.astype(np.int64) != xo.astype(np.int64)) & (bnd == 0)
        assert not bad.any(), (i, int(bad.sum()))
    b.close()


def test_batch_small_and_edge_sizes(P):
    ns = [1, 2, 5, 6, 7, 13, 14]
    circs = [W.random_layered(n, 5, 40 + n) for n in ns]
    b = P.Batch(circs, ns, [100] * len(ns), list(range(len(ns))), keep_states=True)
    b.launch()
    b.synchronize()
    for i, n in enumerate(ns):
        g = b.amplitudes(i).astype(np.complex128)
        assert np.max(np.abs(g - oracle.run(n, circs[i]))) <= AMP_TOL
    b.close()


def test_batch_replay_is_deterministic_and_matches_single_state(P):
    mix, circs = _mix(12, 9, 10, 16)
    ns = [m[0] for m in mix]
    b = P.Batch(circs, ns, [1000] * len(ns), [7 + i for i in range(len(ns))])
    b.launch()
    first = [b.samples(i) for i in range(len(ns))]
    b.launch()
    second = [b.samples(i) for i in range(len(ns))]
    for a, c in zip(first, second):
        assert np.array_equal(a, c)
    # same circuit alone through the single-state path: same draws except boundary ones
    for i in (0, 5, 11):
        s = P.StateVector(ns[i])
        s.apply(circs[i])
        g = s.amplitudes().astype(np.complex128)
        x = s.sample(1000, seed=7 + i)
        _, bnd, _ = oracle.sample(g, W.shot_uniforms(7 + i, 1000))
        bad = (x.astype(np.int64) != first[i].astype(np.int64)) & (bnd == 0)
        assert not bad.any()
        s.close()
    b.close()


def test_batch_rejects_bad_input(P):
    with pytest.raises(P.capi.SvError):
        P.Batch([W.ghz(3)], [3], [10], [1], k_max=4)
    u = np.eye(16, dtype=np.complex128)
    with pytest.raises(P.capi.SvError):  # a 4-qubit block is wider than the batched kernel's limit
        P.Batch([[("unitary", (0, 1, 2, 3), (u,))]], [5], [10], [1])
    with pytest.raises(P.capi.SvError):
        P.Batch([[("cx", (0, 5), ())]], [3], [10], [1])


def test_batch_autotune_returns_a_candidate(P):
    mix, circs = _mix(16, 11, 12, 18)
    args = P.capi.BatchArgs(circs, [m[0] for m in mix], [256] * 16, list(range(16)))
    best, ms = P.capi.sv_batch_autotune(args, reps=1)
    assert best.k_max in (1, 2, 3) and best.tile_qubits in (10, 11, 12, 13)
    assert ms > 0


def test_batch_records_reach_the_device_before_the_launch_under_copy_traffic(P):
    # A batch's plan records and circuit table must be on the device before its
    # graph runs, whatever else the copy engines are doing: here a 2 GiB
    # host-to-device copy on another stream is queued right before each batch is
    # created and launched on a fresh (non-blocking) stream.  A launch that read
    # stale records would fail the kernel's record validation (synchronize
    # raises) or give wrong states.
    import torch
    mix, circs = _mix(48, 9, n_lo=8, n_hi=14, d_hi=8)
    ns = [m[0] for m in mix]
    shots = [64] * len(mix)
    seeds = [2000 + i for i in range(len(mix))]
    host = torch.empty(1 << 29, dtype=torch.float32).pin_memory()
    dev = torch.empty(1 << 29, dtype=torch.float32, device="cuda")
    side = torch.cuda.Stream()
    for rep in range(4):
        with torch.cuda.stream(side):
            dev.copy_(host, non_blocking=True)
        b = P.Batch(circs, ns, shots, seeds, keep_states=True, stream=torch.cuda.Stream())
        b.launch()
        b.synchronize()
        for i in (0, len(mix) // 2, len(mix) - 1):
            g = b.amplitudes(i).astype(np.complex128)
            assert oracle.fidelity(oracle.run(ns[i], circs[i]), g) >= 1 - FID_TOL, (rep, i)
        b.close()
    torch.cuda.synchronize()


@pytest.mark.parametrize("k_max", [1, 2, 3])
def test_batch_arena_register_passes_match_oracle(P, k_max):
    # States above 13 qubits live in the arena; with 12-qubit tiles their passes
    # run as register stages (phase ops, SWAPs folded into the store, dense blocks
    # up to k_max qubits).  Every circuit against the oracle.
    circs, ns = [], []
    for n in (14, 15, 16, 18):
        circs += [W.qft(n), W.ghz(n), W.random_gate_soup(n, 120, seed=900 + n), W.random_layered(n, 6, 950 + n)]
        ns += [n] * 4
    seeds = [3000 + i for i in range(len(ns))]
    b = P.Batch(circs, ns, [256] * len(ns), seeds, k_max=k_max, tile_qubits=12, keep_states=True)
    b.launch()
    b.synchronize()
    for i, n in enumerate(ns):
        g = b.amplitudes(i).astype(np.complex128)
        ref = oracle.run(n, circs[i])
        assert float(np.max(np.abs(g - ref))) <= AMP_TOL, (i, n)
        assert oracle.fidelity(ref, g) >= 1 - FID_TOL, (i, n)
        x = b.samples(i)
        xo, bnd, _ = oracle.sample(g, W.shot_uniforms(seeds[i], 256))
        assert not ((x.astype(np.int64) != xo.astype(np.int64)) & (bnd == 0)).any(), i
    b.close()
