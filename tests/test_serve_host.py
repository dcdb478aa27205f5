"""Host logic of the serving loop's device arena (pcs_serve_arena_plan; no GPU needed).

The server allocates its HBM budget once and places admitted requests in it first fit, in
256-byte aligned ranges, merging a released range with free neighbours.  Checked here: ranges
are aligned, inside the arena and never overlap; a released range is reused; neighbours merge
so that a request needing the whole arena fits again once everything is released; the bytes in
use are the sum of the held ranges; a request that does not fit is refused, not placed.
"""

import random

import pytest

import paper_2006_09808_gb300 as pcs


@pytest.fixture(scope="module")
def lib():
    from paper_2006_09808_gb300 import build

    build.build()
    return pcs.load_library()


def _check_no_overlap(held, cap):
    spans = sorted(held.values())
    for (a, la), (b, _) in zip(spans, spans[1:]):
        assert a + la <= b
    for a, la in spans:
        assert a % 256 == 0 and 0 <= a and a + la <= cap


def test_first_fit_reuse_and_merge(lib):
    cap = 10 * 4096
    ops = [4096, 4096, 4096, -2, 100, -1, -3, 3 * 4096, -5, -8, 10 * 4096]
    off, used = pcs.pcs_serve_arena_plan(cap, ops)
    assert off[:3] == [0, 4096, 8192]
    assert off[4] == 4096          # first fit: the released middle range
    assert used[4] == 2 * 4096 + 256
    # [0, 4096) is too small; releasing the third range merged it with the free ranges on both
    # sides into [4352, cap), which takes the 3-block request
    assert off[7] == 4352
    # everything released: the neighbours merged back into one range holding the whole arena
    assert used[9] == 0 and off[10] == 0 and used[10] == cap


def test_refused_when_it_does_not_fit(lib):
    off, used = pcs.pcs_serve_arena_plan(8192, [6000, 6000, -1, 6000])
    assert off[0] == 0 and off[1] == -1 and used[1] == 6144
    assert off[3] == 0


def test_random_sequences_stay_disjoint(lib):
    rng = random.Random(7)
    cap = 1 << 20
    for trial in range(20):
        ops, live = [], []
        for k in range(200):
            if live and rng.random() < 0.45:
                j = live.pop(rng.randrange(len(live)))
                ops.append(-(j + 1))
            else:
                ops.append(rng.randrange(1, 200_000))
                live.append(k)
        off, used = pcs.pcs_serve_arena_plan(cap, ops)
        held = {}
        for k, o in enumerate(ops):
            if o > 0 and off[k] >= 0:
                held[k] = (off[k], -(-o // 256) * 256)
            elif o < 0:
                held.pop(-o - 1, None)
            _check_no_overlap(held, cap)
            assert used[k] == sum(la for _, la in held.values())
            if o > 0 and off[k] < 0:  # refused: no free gap could hold it
                spans = sorted(held.values())
                edges = [0] + [a + la for a, la in spans]
                starts = [a for a, _ in spans] + [cap]
                assert max(b - e for e, b in zip(edges, starts)) < -(-o // 256) * 256


def test_bad_release_is_refused(lib):
    for ops in ([256, -2], [256, -1, -2]):  # a later op; a release of a release
        with pytest.raises(pcs.PcsError) as ei:
            pcs.pcs_serve_arena_plan(4096, ops)
        assert ei.value.status == pcs.PCS_EINVAL
