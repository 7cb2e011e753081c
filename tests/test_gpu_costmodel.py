"""The calibrated runtime model (Eq. 1) predicts held-out circuits' apply time
on this GPU within 35%, and the serving loop runs with it."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    import paper_2512_04216_gb300 as P
    return P


def test_prediction_on_held_out_circuits(P):
    import torch
    from paper_2512_04216_gb300 import capi, costmodel
    model = costmodel.calibrate(W.calibration_circuits, ns=(12, 15, 18, 21, 24), reps=1)
    errs = []
    for n, c in ((13, W.random_layered(13, 30, 1)), (17, W.random_layered(17, 25, 2)),
                 (20, W.qft(20)), (23, W.random_layered(23, 12, 3)), (22, W.random_gate_soup(22, 300, 4))):
        s = P.StateVector(n)
        ir, keep = capi.to_ir(c)
        best = float("inf")
        for _ in range(3):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s.stream)
            capi.sv_apply_circuit(s.h, ir, len(c))
            e1.record(s.stream)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        s.close()
        pred = model.predict_ms(n, c)
        errs.append(abs(pred - best) / best)
    assert max(errs) <= 0.35, errs


def test_server_with_cost_model(P):
    from paper_2512_04216_gb300 import costmodel, serve
    model = costmodel.calibrate(W.calibration_circuits, ns=(8, 12, 16, 20), reps=1)
    specs = W.serving_requests(20, 3, 500.0, n_lo=8, n_hi=18, mean_n=12.0, d_lo=4, d_hi=12, shots=200)
    reqs = serve.make_requests(specs, W.random_layered)
    a = serve.Server(small_max_qubits=10, streams=4, cost_model=model).run(reqs)
    b = serve.Server(small_max_qubits=10, streams=4).run(reqs)
    for x, y in zip(a, b):
        if x.samples is not None:
            assert np.array_equal(x.samples, y.samples)
        else:
            assert x.expect == y.expect
