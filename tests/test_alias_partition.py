"""Index arithmetic of the GPU alias-table build, emulated on the CPU (CPU only).

The GPU build evaluates the sweep's table from two exact prefix sums and a
merge-path partition (4096-outcome blocks for the counts and the placement of
the light/heavy records; 1024 merged items per merge CTA, 8 per thread; one
record past each segment for the clamps).  This emulation follows the same
partition, block by block and thread by thread, from the oracle's quantised
weights Q -- so it checks the closed form, the partition boundaries, the
clamps and the one-past-the-end reads -- and must reproduce the oracle's
sequential sweep exactly, while asserting every index stays in its buffer."""
import numpy as np
import pytest

import oracle
from tests.oracle_pins import ALIAS_C, random_state

BLOCK, MERGE, PER = 4096, 1024, 8
THREADS = MERGE // PER


def _merge_split(A, B, d):
    a, b = len(A), len(B)
    lo, hi = max(0, d - b), min(d, a)
    while lo < hi:
        mid = (lo + hi) >> 1
        assert 0 <= mid < a and 0 <= d - 1 - mid < b
        if A[mid] <= B[d - 1 - mid]:
            lo = mid + 1
        else:
            hi = mid
    return lo


def _emulate(Q):
    Q = [int(x) for x in Q]
    N = len(Q)
    nblk = (N + BLOCK - 1) // BLOCK
    pre, acc = [], [0, 0, 0]
    for bk in range(nblk):
        items = Q[bk * BLOCK:(bk + 1) * BLOCK]
        pre.append(tuple(acc))
        acc = [acc[0] + sum(q < ALIAS_C for q in items), acc[1] + sum(ALIAS_C - q for q in items if q < ALIAS_C),
               acc[2] + sum(q - ALIAS_C for q in items if q >= ALIAS_C)]
    a, dtot = acc[0], acc[1]
    keys, qv, idx = [None] * N, [None] * N, [None] * N
    for bk in range(nblk):
        start = bk * BLOCK
        kl, dp, ep = pre[bk][0], pre[bk][1], pre[bk][2]
        jh = start - pre[bk][0]
        for i in range(start, min(start + BLOCK, N)):
            if Q[i] < ALIAS_C:
                assert kl < a
                keys[kl], qv[kl], idx[kl] = dp, Q[i], i
                dp += ALIAS_C - Q[i]
                kl += 1
            else:
                ep += Q[i] - ALIAS_C
                assert a + jh < N
                keys[a + jh], idx[a + jh] = ep, i
                jh += 1
    b = N - a
    assert b > 0
    A, B, Ai, Bi = keys[:a], keys[a:], idx[:a], idx[a:]
    own, alias = [None] * N, [None] * N
    nm = (N + MERGE - 1) // MERGE
    splits = [_merge_split(A, B, min(x * MERGE, N)) for x in range(nm + 1)]
    for cta in range(nm):
        d0, d1 = cta * MERGE, min(cta * MERGE + MERGE, N)
        ka0, ka1 = splits[cta], splits[cta + 1]
        jb0, jb1 = d0 - ka0, d1 - ka1
        nA, nB = ka1 - ka0, jb1 - jb0
        assert nA >= 0 and nB >= 0 and nA + nB == d1 - d0
        sA = A[ka0:ka1] + [A[ka1] if ka1 < a else dtot]
        sAq, sAi, sB = qv[ka0:ka1], Ai[ka0:ka1], B[jb0:jb1]
        sBi = Bi[jb0:jb1] + [Bi[jb1] if jb1 < b else Bi[b - 1]]
        for t in range(THREADS):
            dd0 = min(t * PER, nA + nB)
            dd1 = min(dd0 + PER, nA + nB)
            lo, hi = max(0, dd0 - nB), min(dd0, nA)
            while lo < hi:
                mid = (lo + hi) >> 1
                if sA[mid] <= sB[dd0 - 1 - mid]:
                    lo = mid + 1
                else:
                    hi = mid
            ka, jb = lo, dd0 - lo
            for _ in range(dd0, dd1):
                if ka < nA and (jb >= nB or sA[ka] <= sB[jb]):
                    assert own[sAi[ka]] is None and jb <= nB
                    own[sAi[ka]], alias[sAi[ka]] = sAq[ka], sBi[jb]
                    ka += 1
                else:
                    assert jb < nB
                    o, al = ALIAS_C, sBi[jb]
                    if jb0 + jb + 1 < b and sA[ka] > sB[jb]:
                        o, al = ALIAS_C - (sA[ka] - sB[jb]), sBi[jb + 1]
                        assert 0 <= o < ALIAS_C
                    assert own[sBi[jb]] is None
                    own[sBi[jb]], alias[sBi[jb]] = o, al
                    jb += 1
    assert all(x is not None for x in own)
    return np.array(own, dtype=np.int64), np.array(alias, dtype=np.int64)


def _states():
    rng = np.random.default_rng(5)
    for n in (1, 2, 5, 11, 12, 13):
        v = random_state(n, rng)
        yield f"random n={n}", v
        w = v.copy()
        w[rng.random(1 << n) < 0.6] = 0
        if not np.any(w):
            w[0] = 1
        yield f"sparse n={n}", w
    n = 13
    yield "basis", oracle.basis(n, (1 << n) - 1)
    yield "uniform", np.full(1 << n, 2.0 ** (-n / 2), dtype=np.complex128)
    z = np.full(1 << n, 0.01, dtype=np.complex128)
    z[[3, 4000, 8000]] = 10
    yield "spiky", z
    y = np.full(1 << n, 1.0, dtype=np.complex128)
    y[rng.integers(0, 1 << n, 150)] = 0.05
    yield "flat", y
    # weights 3, 1, 1, 3 repeated: Q = 1.5 C, 0.5 C, 0.5 C, 1.5 C exactly, so deficit
    # and excess prefixes tie (lights before heavies on ties decides the aliases)
    for n in (2, 12):
        t = np.tile(np.array([np.sqrt(3.0), 1.0, 1.0, np.sqrt(3.0)], dtype=np.complex128), 1 << (n - 2))
        yield f"ties n={n}", t


@pytest.mark.parametrize("name,psi", list(_states()), ids=lambda x: x if isinstance(x, str) else "")
def test_partition_reproduces_the_sweep(name, psi):
    Q, own, alias = oracle.alias_build(psi)
    o2, a2 = _emulate(Q)
    assert np.array_equal(o2, own.astype(np.int64)), name
    assert np.array_equal(a2, alias.astype(np.int64)), name
