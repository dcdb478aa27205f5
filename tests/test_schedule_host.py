"""Host logic of the balanced schedule (pcs_schedule_plan; no GPU needed).

Invariants that make the split solve equal to whole-slice solves: every
slice-iteration is covered exactly once and in order; a slice is split at most
once, between consecutive clusters; the first part ends its cluster's range and
runs first in that cluster's time, the continuation starts the next cluster's
range and runs last, flagged to wait; and in a timeline where every cluster
runs one iteration per time unit no continuation would wait at all.
"""

import pytest

import paper_2006_09808_gb300 as pcs


@pytest.fixture(scope="module")
def lib():
    from paper_2006_09808_gb300 import build

    build.build()
    return pcs.load_library()


@pytest.mark.parametrize("S,N,K", [(64, 500, 36), (64, 500, 37), (38, 500, 36), (100, 7, 36), (64, 1, 36),
                                   (37, 500, 36), (200, 13, 7), (5, 3, 4), (2, 1, 1)])
def test_schedule_invariants(lib, S, N, K):
    segs, off = pcs.pcs_schedule_plan(S, N, K)
    assert off[0] == 0 and off[-1] == len(segs) and all(a <= b for a, b in zip(off, off[1:]))
    T = -(-S * N // K)
    pieces = {s: [] for s in range(S)}
    for c in range(K):
        t = 0
        work = 0
        for k in range(off[c], off[c + 1]):
            s, b, e, f = segs[k]
            assert 0 <= s < S and 0 <= b < e <= N
            assert f == (1 if b > 0 else 0) | (2 if e < N else 0)
            pieces[s].append((b, e, c, t, t + e - b, k - off[c], off[c + 1] - off[c]))
            t += e - b
            work += e - b
        assert work <= T
    for s, p in pieces.items():
        p.sort()
        assert p[0][0] == 0 and p[-1][1] == N
        assert all(p[i][1] == p[i + 1][0] for i in range(len(p) - 1))
        assert len(p) <= 2
        if len(p) == 2:
            (b0, e0, c0, s0, t0, i0, n0), (b1, e1, c1, s1, t1, i1, n1) = p
            assert c1 == c0 + 1
            assert i0 == 0 and i1 == n1 - 1  # first part runs first, continuation last
            assert t0 <= s1  # ideal timeline: no wait


def test_schedule_plan_rejects_what_needs_no_schedule(lib):
    with pytest.raises(pcs.PcsError) as ei:
        pcs.pcs_schedule_plan(36, 500, 36)  # as many clusters as slices: whole slices
    assert ei.value.status == pcs.PCS_EINVAL
