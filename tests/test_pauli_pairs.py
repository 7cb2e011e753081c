"""The pair decomposition the GPU Pauli-string reduction uses, emulated on the
CPU (CPU only): for x != 0, b = x's lowest set bit, every pair (i, j = i ^ x)
with bit b of i clear contributes 2 s_i Re(w) (-1)^(k/2) (k even) or
-2 s_i Im(w) (-1)^((k-1)/2) (k odd), w = conj(psi_i) psi_j,
s_i = (-1)^popcount(j & z), k = popcount(x & z); <P> is the sum over the
pairs divided by the norm.  It must equal the oracle's plain definition."""
import numpy as np
import pytest

import oracle


def _pairs_expectation(psi, x, z):
    n = int(psi.shape[0]).bit_length() - 1
    b = (x & -x).bit_length() - 1
    k = bin(x & z).count("1")
    m = np.arange(psi.shape[0] // 2, dtype=np.int64)
    low = (1 << b) - 1
    i = ((m & ~low) << 1) | (m & low)
    j = i ^ x
    assert np.all((i >> b) & 1 == 0) and len(np.unique(np.concatenate([i, j]))) == 1 << n
    w = np.conj(psi[i]) * psi[j]
    s = 1 - 2 * (np.array([bin(int(v) & z).count("1") for v in j]) & 1)
    if k % 2 == 0:
        c = s * w.real * (-1) ** (k // 2)
    else:
        c = -s * w.imag * (-1) ** ((k - 1) // 2)
    return 2 * float(np.sum(c)) / float(np.sum(np.abs(psi) ** 2))


@pytest.mark.parametrize("n", [1, 2, 4, 7])
def test_pair_decomposition_equals_the_definition(n):
    rng = np.random.default_rng(n)
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    for _ in range(20):
        x = int(rng.integers(1, 1 << n))
        z = int(rng.integers(0, 1 << n))
        want = oracle.expect_pauli(psi, x, z)
        assert abs(_pairs_expectation(psi, x, z) - want.real) < 1e-12, (n, x, z)
