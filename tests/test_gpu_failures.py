"""Failure handling without faulting, trapping or hanging the GPU: a device
wait that nothing satisfies gives up and reports SV_ERR_TIMEOUT; allocation
failures and invalid requests return status codes and leave the library (and
other states) usable."""
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


def test_bounded_wait_times_out(P):
    capi = P.capi
    assert capi.sv_diag_bounded_wait(50) == capi.SV_ERR_TIMEOUT
    assert "gave up" in capi.sv_last_error()
    # the context is still usable afterwards
    s = P.StateVector(10)
    s.apply(W.ghz(10))
    assert abs(s.norm2() - 1.0) < 1e-6
    s.close()


def test_state_allocation_failure_is_reported(P):
    capi = P.capi
    keep = P.StateVector(12)
    keep.apply(W.ghz(12))
    with pytest.raises(capi.SvError) as e:
        capi.sv_create(36)  # 512 GiB of complex64: more than the device holds
    assert e.value.code == capi.SV_ERR_OOM
    # an existing state is unaffected
    g = keep.amplitudes()
    assert abs(abs(g[0]) ** 2 - 0.5) < 1e-6 and abs(abs(g[-1]) ** 2 - 0.5) < 1e-6
    keep.close()


def test_bad_arguments_are_rejected(P):
    capi = P.capi
    s = P.StateVector(6)
    for fn in (lambda: capi.sv_reset(s.h, 1 << 6),
               lambda: capi.sv_expect_pauli(s.h, 1 << 6, 0),
               lambda: capi.sv_probabilities(s.h, np.empty(4), 62, 4, False),
               lambda: capi.sv_create(0),
               lambda: capi.sv_create(8, capi.SV_C128)):
        with pytest.raises(capi.SvError):
            fn()
    s.apply(W.ghz(6))
    assert abs(s.norm2() - 1) < 1e-6
    s.close()
