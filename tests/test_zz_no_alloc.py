"""sv_expect_z_static: the allocation-free expectation entry point.

It exists for callers that cannot allocate device memory when they need an
expectation value (all free GPU memory reserved up front for resident states,
or a latency-critical loop that cannot take cudaMalloc's device-wide
synchronisation).  Its result must equal the existing entry points'
(sv_expect_pauli, sv_norm) on the same state, call after call, although every
call reuses one fixed scratch array, and equal the oracle's double sums on the
GPU's own state, up to the array's 28-qubit limit (where it is exactly full).
This file is collected last so that a stop-at-first-failure run has already run
every other test.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-12  # the tolerance the other GPU tests use for norms and expectations


@pytest.fixture(scope="module")
def sv():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    import paper_2512_04216_gb300 as P
    return P


def test_static_expectation_matches_existing_entry_points(sv):
    import torch
    capi = sv.capi
    for n, seed in ((5, 1), (13, 2), (20, 3), (28, 4)):
        s = sv.StateVector(n)
        s.apply(W.random_layered(n, 8, seed))
        psi = s.amplitudes()
        out = torch.zeros(2, dtype=torch.float64, device=s.device)
        masks = [1, (1 << n) - 1, 0b101 & ((1 << n) - 1), 0]
        for _ in range(2):  # two calls in a row on the shared scratch array
            for m in masks:
                out.fill_(-7.0)
                capi.sv_expect_z_static(s.amps, n, m, out, s.stream)
                s.stream.synchronize()
                got = out.cpu().numpy()
                assert abs(got[0] - s.expect_z(m)) <= TOL, (n, m, got[0])
                assert abs(got[1] - s.norm2()) <= TOL, (n, m, got[1])
                assert abs(got[0] - oracle.expect_z(psi, m)) <= TOL, (n, m, got[0])
        s.close()


def test_static_expectation_of_a_zero_state_is_nan(sv):
    import torch
    capi = sv.capi
    buf = torch.zeros(1 << 6, dtype=torch.complex64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    capi.sv_expect_z_static(buf, 6, 1, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert math.isnan(got[0]) and got[1] == 0.0


def test_static_expectation_rejects_states_beyond_its_limit(sv):
    import torch
    capi = sv.capi
    buf = torch.zeros(16, dtype=torch.complex64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(capi.SvError) as e:
        capi.sv_expect_z_static(buf, 29, 1, out)
    assert e.value.code == capi.SV_ERR_ARG
    assert "28" in str(e.value)
    with pytest.raises(capi.SvError):
        capi.sv_expect_z_static(buf, 4, 1 << 4, out)
