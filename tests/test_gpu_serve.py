"""Serving loop: every request's result is the same served alone and served in
a mixed stream (bit-identical samples, equal expectations), and agrees with
the complex128 oracle (samples identical except draws within delta of a CDF
boundary, delta = 1e-6 covering complex64 vs complex128 CDFs at n <= 18;
expectations within 1e-5).  Admission respects the HBM budget."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    from paper_2512_04216_gb300 import serve
    return serve


def _requests(S, count, seed, rate, n_hi=18, d_hi=16):
    specs = W.serving_requests(count, seed, rate, n_lo=8, n_hi=n_hi, mean_n=12.0, d_lo=4, d_hi=d_hi, shots=300)
    return S.make_requests(specs, W.random_layered), specs


def _check_against_oracle(res, spec):
    circ = W.random_layered(spec["n"], spec["depth"], spec["seed"])
    ref = oracle.run(spec["n"], circ)
    if "shots" in spec:
        u = W.shot_uniforms(spec["shot_seed"], spec["shots"])
        xo, bnd, _ = oracle.sample_cdf(oracle.cdf(ref), u, eps=1e-6)
        bad = (res.samples.astype(np.int64) != xo.astype(np.int64)) & (bnd == 0)
        assert not bad.any(), (spec["id"], int(bad.sum()))
    else:
        assert abs(res.expect - oracle.expect_z(ref, spec["zmask"])) <= 1e-5


@pytest.mark.parametrize("tc_from", [None, 14])
def test_mix_equals_alone_and_oracle(S, tc_from):
    # tc_from: requests of >= 14 qubits on the tensor-core passes, the rest of the
    # stream path on CUDA cores
    reqs, specs = _requests(S, 40, 5, rate=400.0)
    server = S.Server(small_max_qubits=12, streams=4, tc_from_qubits=tc_from)
    mixed = server.run(reqs)
    assert {r.path for r in mixed} == {"batch", "stream"}
    for res, req, spec in zip(mixed, sorted(reqs, key=lambda r: r.id), sorted(specs, key=lambda s: s["id"])):
        req.t = 0.0
        (alone,) = server.run([req])
        assert alone.path == res.path
        if req.shots:
            assert np.array_equal(alone.samples, res.samples), req.id
        else:
            assert alone.expect == res.expect, req.id
        _check_against_oracle(res, spec)


@pytest.mark.parametrize("tc_from", [None, 13])
def test_plain_path_agrees(S, tc_from):
    reqs, specs = _requests(S, 16, 8, rate=1000.0, n_hi=16)
    plain = S.run_plain(reqs, tc_from_qubits=tc_from)
    for res, spec in zip(plain, sorted(specs, key=lambda s: s["id"])):
        _check_against_oracle(res, spec)
    s = S.summarize(plain)
    assert s["requests"] == 16 and s["circuits_per_s"] > 0 and s["p99_ms"] >= s["p50_ms"]


def test_admission_under_memory_pressure(S):
    reqs, specs = _requests(S, 12, 11, rate=10000.0, n_hi=18)
    biggest = max(r.n for r in reqs)
    # room for one resident large state at a time
    server = S.Server(small_max_qubits=9, streams=4, hbm_budget=S.footprint_bytes(biggest) + 1)
    out = server.run(reqs)
    ref = S.Server(small_max_qubits=9, streams=4).run(reqs)
    for a, b in zip(out, ref):
        if a.samples is not None:
            assert np.array_equal(a.samples, b.samples)
        else:
            assert a.expect == b.expect
    big = [r for r in reqs if r.n > 9]
    # with the budget above, large requests never overlapped
    spans = sorted((r.t_start, r.t_done) for r in out if r.path == "stream")
    for (s0, e0), (s1, e1) in zip(spans, spans[1:]):
        assert s1 >= e0 - 1e-3 or len(big) <= 1
    with pytest.raises(ValueError):
        S.Server(small_max_qubits=9, hbm_budget=1024).run(reqs)
