"""Cross-stream ordering of state operations (GPU required), through the C-ABI.

A clone or merge reads its sources on the new state's stream; work queued on
a source's own stream afterwards -- an apply that overwrites it -- must wait
for that read.  Changing a state's stream must keep the order of the work
queued on it.  Each case queues the conflicting work immediately, with no host
synchronisation in between, and checks the results against the oracle.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sv():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    import paper_2512_04216_gb300 as P
    return P


def test_clone_is_not_overwritten_by_later_source_work(sv):
    import torch
    n = 22
    c1, c2 = W.random_layered(n, 10, 61), W.random_layered(n, 30, 62)
    s = sv.StateVector(n, stream=torch.cuda.Stream())
    s.apply(c1)
    cl = s.clone(stream=torch.cuda.Stream())
    s.apply(c2)  # queued on the source's stream right after the clone was queued
    got = cl.amplitudes().astype(np.complex128)
    ref = oracle.run(n, c1)
    assert oracle.fidelity(ref, got) >= 1 - 1e-6
    assert np.max(np.abs(got - ref)) <= 1e-5
    cl.close()
    s.close()


def test_merge_sources_are_not_overwritten_before_the_merge(sv):
    import torch
    na, nb = 11, 10
    ca, cb = W.random_layered(na, 8, 63), W.random_layered(nb, 8, 64)
    a = sv.StateVector(na, stream=torch.cuda.Stream())
    b = sv.StateVector(nb, stream=torch.cuda.Stream())
    a.apply(ca)
    b.apply(cb)
    m = a.merge(b, stream=torch.cuda.Stream())
    a.apply(W.random_layered(na, 40, 65))
    b.apply(W.random_layered(nb, 40, 66))
    got = m.amplitudes().astype(np.complex128)
    ref = np.kron(oracle.run(nb, cb), oracle.run(na, ca))
    assert oracle.fidelity(ref, got) >= 1 - 1e-6
    m.close()
    a.close()
    b.close()


def test_set_stream_keeps_the_order_of_queued_work(sv):
    import torch
    n = 21
    c1, c2 = W.random_layered(n, 20, 67), W.random_layered(n, 4, 68)
    s = sv.StateVector(n, stream=torch.cuda.Stream())
    s.apply(c1)
    st2 = torch.cuda.Stream()
    sv.capi.sv_set_stream(s.h, st2)
    s.stream = st2
    s.apply(c2)  # must follow c1, which may still be running on the first stream
    got = s.amplitudes().astype(np.complex128)
    ref = oracle.run(n, c1 + c2)
    assert oracle.fidelity(ref, got) >= 1 - 1e-6
    s.close()
