"""Balanced schedule: more slices than resident clusters (the default 256 x 256
variant keeps 36 clusters resident) -> some slices run in two parts on two
clusters.  The split is a continuation from the stored state, so every slice
must come out bit-identical to a solve of that slice alone."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2006_09808_gb300 as pcs  # noqa: E402
import phantoms  # noqa: E402

pytestmark = pytest.mark.gpu
STEP = 1.0 / 2.833285229534487  # full-mask ||K|| of 256 x 256 (tests/golden/opnorm_full_mask.txt)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_09808_gb300 import build

    build.build()
    pcs.load_library()


def solve(field, mask, lam, n_iter, **opts):
    S, H, W = field.shape
    f = torch.from_numpy(field).cuda()
    m = torch.from_numpy(mask).cuda()
    chi = torch.full_like(f, float("nan"))
    ctx = pcs.pcs_create(H, W, S, **opts)
    try:
        pcs.pcs_solve_slices(ctx, f, m, lam, STEP, STEP, n_iter, chi)
        pcs.pcs_check(ctx)
    finally:
        pcs.pcs_destroy(ctx)
    return chi.cpu().numpy()


def alone(field, mask, lam, n_iter):
    out = np.empty_like(field)
    for s in range(field.shape[0]):
        out[s] = solve(field[s:s + 1].copy(), mask[s:s + 1].copy(), lam, n_iter)[0]
    return out


@pytest.mark.parametrize("S,n_iter", [(64, 40), (37, 23)])
def test_balanced_schedule_is_bit_identical_to_slices_alone(S, n_iter):
    pb = phantoms.volume(256, 256, S, seed=71, lam=5e-4, n_iter=n_iter)
    got = solve(pb.field, pb.mask, pb.lam, n_iter)
    assert np.all(np.isfinite(got))
    assert np.array_equal(got, alone(pb.field, pb.mask, pb.lam, n_iter))


def test_balanced_schedule_under_graph_replay():
    pb = phantoms.volume(256, 256, 48, seed=72, lam=5e-4, n_iter=30)
    f = torch.from_numpy(pb.field).cuda()
    m = torch.from_numpy(pb.mask).cuda()
    st = torch.cuda.Stream()
    outs = []
    ctx = pcs.pcs_create(256, 256, 48, use_graph=True, stream=st)
    try:
        for _ in range(3):  # capture, then two replays (the flags are cleared inside the graph)
            chi = torch.full_like(f, float("nan"))
            with torch.cuda.stream(st):
                pcs.pcs_solve_slices(ctx, f, m, pb.lam, STEP, STEP, 30, chi)
            pcs.pcs_check(ctx)
            outs.append(chi.cpu().numpy())
    finally:
        pcs.pcs_destroy(ctx)
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    assert np.array_equal(outs[0], solve(pb.field, pb.mask, pb.lam, 30))


def test_bounded_wait_gives_up_and_reports():
    # one warp waits on a flag nothing sets; about 1 ms of SM clock cycles
    assert pcs.pcs_selftest_wait(2_000_000) is True
