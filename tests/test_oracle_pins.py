"""The oracle against the mathematics (CPU only)."""
import pytest

import oracle
from tests import oracle_pins as P


@pytest.mark.parametrize("pin", P.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(pin):
    pin(oracle.default())


def test_inverse_rules_are_inverses():
    # Each inverse rule of the input generator undoes its gate exactly.
    import numpy as np
    import workloads as W
    o = oracle.default()
    soup = W.random_gate_soup(3, 200, seed=4)
    for g in soup:
        (gi,) = W.inverse([g])
        n = 3
        M = P.kron_full(n, g[1], o.gate_matrix(g[0], g[1], g[2]))
        Mi = P.kron_full(n, gi[1], o.gate_matrix(gi[0], gi[1], gi[2]))
        assert np.allclose(Mi @ M, np.eye(8), atol=1e-12), g
