"""Walker alias sampling on the GPU (§III-C: shots by alias sampling, O(1) per
shot) against the oracle's alias table.

Both sides quantise the weights to units of 2^-31 of a bucket; the GPU does it
with float32 pairs (~46 bits) and its own total W (compensated float32 sums,
relative error below 2^-44), so an item's Q may differ from the oracle's by one
unit where the exact value lies next to a half-unit boundary, plus Q * 2^-44
from W; prefixes drift by the sum of these, at most DRIFT(N) = N * 2^-13 units
from W (the weights total N * 2^31) plus the count of flipped roundings.  Hence:
  * own_i within OWN_TOL + DRIFT(N) units of the oracle's for every bucket;
  * aliases identical, except where the oracle's deficit and excess prefixes
    are within OWN_TOL units of each other (a tie the drift can flip);
  * draws identical for the same uniforms, except in such buckets or where the
    coin f * 2^31 is within OWN_TOL units of own_i;
  * the table's implied units (own_i plus every C - own_k aliasing i) equal the
    oracle's quantised weights within one unit for light outcomes, and their
    total discrepancy is the quantisation residual plus the drift.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from tests.oracle_pins import ALIAS_C, alias_masses

pytestmark = pytest.mark.gpu
OWN_TOL = 256


def DRIFT(N):
    return N >> 13


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    import paper_2512_04216_gb300 as P
    return P


def _state(n, seed, zero_frac=0.0, kind="random"):
    """Seeded complex64 amplitudes (the oracle reads the same values in complex128)."""
    rng = np.random.default_rng(seed)
    N = 1 << n
    if kind == "uniform":
        v = np.full(N, 2.0 ** (-n / 2))
    elif kind == "spiky":
        v = np.full(N, 0.01 + 0j)
        v[rng.integers(0, N, 3)] = 10.0
    else:
        v = rng.normal(size=N) + 1j * rng.normal(size=N)
        v[rng.random(N) < zero_frac] = 0
        if not np.any(v):
            v[N - 1] = 1
    v = v / np.linalg.norm(v)
    return v.astype(np.complex64)


def _oracle_prefixes(Q):
    light = Q < ALIAS_C
    Dex = np.concatenate(([0], np.cumsum(ALIAS_C - Q[light])[:-1])) if light.any() else np.zeros(0, np.int64)
    E = np.cumsum(Q[~light] - ALIAS_C)
    return light, Dex, E


def _compare_tables(n, amps, own, alias):
    Q, own_o, alias_o = oracle.alias_build(amps.astype(np.complex128))
    Q = Q.astype(np.int64)
    own = own.astype(np.int64)
    own_o = own_o.astype(np.int64)
    N = 1 << n
    assert own.shape == (N,) and alias.shape == (N,)
    assert np.all(own <= ALIAS_C) and np.all(alias.astype(np.int64) < N), "table range"
    d_own = np.abs(own - own_o)
    tol = OWN_TOL + DRIFT(N)
    assert int(d_own.max()) <= tol, f"own differs by {int(d_own.max())} units"
    bad = np.nonzero(alias != alias_o)[0]
    if bad.size:
        light, Dex, E = _oracle_prefixes(Q)
        rank = np.cumsum(light) - 1
        for i in bad:
            assert light[i], f"heavy bucket {i} aliases {alias[i]} (oracle {alias_o[i]})"
            margin = np.min(np.abs(E - Dex[rank[i]]))
            assert margin <= tol, f"alias of {i} differs with margin {margin}"
        assert bad.size <= 2, f"{bad.size} alias differences"
    _check_units(N, own, alias, Q)
    return own_o, alias_o, bad


def _check_units(N, own, alias, Q):
    """Implied units against reference weights Q: within one unit everywhere
    except the few heavy outcomes that absorb the quantisation residual (the
    last heavy item, and heavy items the light deficits never reach)."""
    M = alias_masses(own.astype(np.uint32), alias)
    assert int(M.sum()) == N * ALIAS_C, "units per bucket"
    light = Q < ALIAS_C
    assert int(np.abs(M[light] - Q[light]).max(initial=0)) <= 1, "light units"
    # heavy outcomes: one unit of rounding plus the share of W's error
    slack = 1 + (Q.astype(np.float64) * 2.0 ** -44).astype(np.int64)
    off = np.abs(M - Q) > slack
    assert int(off.sum()) <= 3, f"{int(off.sum())} outcomes off by more than their rounding"
    assert not np.any(off & light), "a light outcome absorbs units"
    resid = abs(N * ALIAS_C - int(Q.sum()))
    assert int(np.abs(M - Q)[off].sum()) <= resid + N // 2000 + DRIFT(N) + 8, "unit discrepancy"


def _compare_draws(n, own, own_o, alias_o, bad, u, got):
    want = oracle.alias_sample(own_o.astype(np.uint32), alias_o, u)
    N = 1 << n
    x = u * N
    i = np.minimum(np.floor(x), N - 1).astype(np.int64)
    f = x - i
    near = np.abs(f * ALIAS_C - own_o[i].astype(np.float64)) <= OWN_TOL + DRIFT(N)
    excused = near | np.isin(i, bad) | (own[i].astype(np.int64) != own_o[i].astype(np.int64))
    diff = got.astype(np.int64) != want.astype(np.int64)
    assert not np.any(diff & ~excused), f"{int(np.sum(diff & ~excused))} draws differ"
    assert int(diff.sum()) <= max(2, len(u) // 10000), f"{int(diff.sum())} draws differ"


@pytest.mark.parametrize("n,kind,zero", [(1, "random", 0.0), (2, "random", 0.0), (3, "random", 0.3),
                                         (8, "random", 0.5), (11, "random", 0.0), (12, "random", 0.2),
                                         (13, "random", 0.0), (16, "spiky", 0.0), (16, "uniform", 0.0),
                                         (20, "random", 0.1)])
def test_alias_table_and_draws_match_oracle(P, n, kind, zero):
    amps = _state(n, 100 + n, zero, kind)
    s = P.StateVector(n)
    s.set_amplitudes(amps)
    s.alias_build()
    own, alias = s.alias_table()
    own_o, alias_o, bad = _compare_tables(n, amps, own, alias)
    u = W.shot_uniforms(7 + n, 20000)
    got = s.sample_alias_uniforms(u)
    _compare_draws(n, own, own_o, alias_o, bad, u, got)
    # device-drawn uniforms follow the same SplitMix64 rule as sample()
    got_seeded = s.sample_alias(20000, 7 + n)
    assert np.array_equal(got_seeded, got)
    s.close()


def test_alias_distribution_of_a_circuit_state(P):
    """20-qubit random layered circuit: the table's implied distribution against
    the oracle's |psi|^2 (total variation), and a chi-square of 2e6 draws over
    the 64 most likely outcomes plus the rest pooled."""
    n = 20
    circ = W.random_layered(n, 12, 9)
    s = P.StateVector(n)
    s.apply(circ)
    s.alias_build()
    own, alias = s.alias_table()
    M = alias_masses(own, alias).astype(np.float64) / ((1 << n) * ALIAS_C)
    p = np.abs(oracle.run(n, circ)) ** 2
    p = p / p.sum()
    tv = 0.5 * float(np.abs(M - p).sum())
    assert tv < 1e-4, f"total variation {tv}"
    S = 2_000_000
    x = s.sample_alias(S, 12345).astype(np.int64)
    top = np.argsort(p)[-64:]
    cnt = np.bincount(x, minlength=1 << n)
    obs = np.concatenate([cnt[top], [S - cnt[top].sum()]])
    exp = np.concatenate([S * p[top], [S * (1 - p[top].sum())]])
    chi2 = float(np.sum((obs - exp) ** 2 / exp))
    assert chi2 < 64 + 6 * np.sqrt(128), f"chi2 {chi2}"
    s.close()


def test_alias_full_size_units(P):
    """The 28-qubit bench state (random layered depth 40): every light bucket
    keeps exactly its own units (own_i = Q_i, recomputed here from the read-back
    amplitudes in float64 within one unit) and the table's implied units match
    the quantised weights up to the residual and the drift; sampled draws for
    2^20 uniforms follow the draw rule applied to the read-back table."""
    n = 28
    N = 1 << n
    s = P.StateVector(n)
    s.apply(W.random_layered(n, 40, 2))
    s.alias_build()
    own, alias = s.alias_table()
    a = s.amplitudes()
    p = a.real.astype(np.float64) ** 2 + a.imag.astype(np.float64) ** 2
    del a
    Q = np.rint(p * (N / math.fsum(p)) * ALIAS_C).astype(np.int64)
    del p
    light = Q < ALIAS_C
    o = own.astype(np.int64)
    assert int(np.abs(o[light] - Q[light]).max()) <= 1, "light own units"
    assert np.all(o <= ALIAS_C) and int(alias.max()) < N
    _check_units(N, own, alias, Q)
    u = W.shot_uniforms(99, 1 << 20)
    got = s.sample_alias_uniforms(u).astype(np.int64)
    x = u * N
    i = np.minimum(np.floor(x), N - 1).astype(np.int64)
    f = x - i
    want = np.where(f * ALIAS_C < own[i].astype(np.float64), i, alias[i].astype(np.int64))
    assert np.array_equal(got, want)
    s.close()


def test_alias_errors(P):
    s = P.StateVector(4)
    with pytest.raises(P.capi.SvError):
        s.sample_alias(10, 1)            # no table yet
    s.set_amplitudes(np.zeros(16, dtype=np.complex64))
    with pytest.raises(P.capi.SvError):
        s.alias_build()                  # no weight
    s.reset(3)
    s.alias_build()
    assert np.all(s.sample_alias(1000, 5) == 3)
    s.alias_release()
    with pytest.raises(P.capi.SvError):
        s.sample_alias(10, 1)
    s.close()


def test_alias_maximum_size_ghz32(P):
    """n = 32, the largest table (32-bit outcomes): GHZ has two heavy outcomes,
    0 and N-1, of N/2 buckets each, and N-2 empty light ones.  Light outcomes
    1..N/2 fill from outcome 0, which is then used up exactly (its excess is
    N/2 - 1 buckets) and keeps (almost) nothing, aliasing N-1; lights N/2+1..N-2
    fill from N-1, the last heavy outcome, which keeps a full bucket.  The
    weights come from float32 pairs, so the switch may move by one bucket and
    outcome 0 keeps either a sliver of units or all but a sliver."""
    n = 32
    N = 1 << n
    s = P.StateVector(n)
    s.apply(W.ghz(n))
    s.alias_build()
    own, alias = s.alias_table(0, 1000)
    # Q_0 = N/2 buckets +- a float32-pair rounding: 0 is used up by light N/2 (keeping the
    # excess over N/2 buckets) or one light earlier (keeping almost a full bucket)
    assert (own[0] < 1 << 17 or own[0] > ALIAS_C - (1 << 17)) and alias[0] == N - 1, (own[0], alias[0])
    assert np.all(own[1:] == 0) and np.all(alias[1:] == 0)
    own, alias = s.alias_table(N - 1000, 1000)
    assert np.all(own[:-1] == 0) and np.all(alias[:-1] == N - 1)
    assert own[-1] == ALIAS_C and alias[-1] == N - 1
    own, alias = s.alias_table((N >> 1) - 4, 9)
    assert np.all(own == 0)
    switch = int(np.argmax(alias == N - 1))
    assert np.all(alias[:switch] == 0) and np.all(alias[switch:] == N - 1) and 3 <= switch <= 6, alias
    x = s.sample_alias(1_000_000, 5).astype(np.int64)
    assert set(np.unique(x).tolist()) <= {0, N - 1}
    frac = float(np.mean(x == 0))
    assert abs(frac - 0.5) < 5 * 0.0005, frac
    s.close()
    big = P.StateVector(33)
    with pytest.raises(P.capi.SvError) as e:
        big.alias_build()
    assert e.value.code == P.capi.SV_ERR_UNSUPPORTED
    big.close()
