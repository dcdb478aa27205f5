"""Monitored solves: FP64 diagnostics every k iterations, exact resume, per-slice early stop."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2006_09808_gb300 as pcs  # noqa: E402
import phantoms  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_09808_gb300 import build

    build.build()
    pcs.load_library()


def _plain(pb, n_iter, tau, **opts):
    S, H, W = pb.field.shape
    f = torch.from_numpy(pb.field).cuda()
    m = torch.from_numpy(pb.mask).cuda()
    chi = torch.empty_like(f)
    ctx = pcs.pcs_create(H, W, S, **opts)
    try:
        pcs.pcs_solve_slices(ctx, f, m, pb.lam, tau, tau, n_iter, chi)
        torch.cuda.synchronize()
    finally:
        pcs.pcs_destroy(ctx)
    return chi.cpu().numpy()


def _monitored(pb, n_iter, tau, every, tol, **opts):
    S, H, W = pb.field.shape
    f = torch.from_numpy(pb.field).cuda()
    m = torch.from_numpy(pb.mask).cuda()
    chi = torch.full_like(f, float("nan"))
    ctx = pcs.pcs_create(H, W, S, **opts)
    try:
        rep = pcs.pcs_solve_slices_monitored(ctx, f, m, pb.lam, tau, tau, n_iter, every, tol, chi)
    finally:
        pcs.pcs_destroy(ctx)
    return chi.cpu().numpy(), rep


@pytest.mark.parametrize("H,S", [(256, 4), (64, 3)])
def test_chunked_resume_is_exact(H, S):
    pb = phantoms.volume(H, H, S, seed=H + S, lam=5e-4, n_iter=200)
    tau = 1.0 / 2.8333
    got, rep = _monitored(pb, 200, tau, 37, 0.0)
    ref = _plain(pb, 200, tau, kernel=pcs.KERNEL_STREAMING)
    assert np.array_equal(got, ref)
    assert all(r["iters"] == 200 for r in rep)
    assert all(r["gap"] >= 0 for r in rep)


def test_early_stop_per_slice():
    pb = phantoms.volume(64, 64, 6, seed=3, lam=10.0, n_iter=600)
    tau = 1.0 / 2.8326
    tol = 2e-3
    got, rep = _monitored(pb, 600, tau, 50, tol)
    iters = [r["iters"] for r in rep]
    assert min(iters) < 600  # something stopped early
    for s, r in enumerate(rep):
        if r["iters"] < 600:
            assert r["gap"] <= tol * r["objective"]
        ref = _plain(pb, r["iters"], tau, kernel=pcs.KERNEL_STREAMING)
        assert np.array_equal(got[s], ref[s]), s


def test_monitored_with_more_slices_than_resident_clusters():
    """40 slices of 256 x 256 (the default variant keeps 36 clusters resident, so clusters take
    several slices per chunk on the plain persistent loop, and the report kernel several slices
    per launch): chunked == one straight solve bit for bit, and two sampled slices' FP64 reports
    against the oracle's diagnostics."""
    from oracle import pd_oracle as O

    pb = phantoms.volume(256, 256, 40, seed=44, lam=10.0, n_iter=120)
    tau = 1.0 / 2.8333
    got, rep = _monitored(pb, 120, tau, 50, 0.0)
    ref = _plain(pb, 120, tau, kernel=pcs.KERNEL_STREAMING)
    assert np.array_equal(got, ref)
    assert all(r["iters"] == 120 for r in rep)
    for s in (0, 39):
        st = O.pd_solve(pb.field[s].astype(np.float64), pb.mask[s], pb.lam, tau, tau, 120, return_state=True)
        d = O.diagnostics(st, pb.field[s].astype(np.float64), pb.mask[s], pb.lam)
        assert np.linalg.norm(got[s] - st.chi) / np.linalg.norm(st.chi) <= 1e-4, s
        assert rep[s]["objective"] == pytest.approx(d.primal, rel=1e-4), s
        assert rep[s]["data_residual"] == pytest.approx(d.data_residual, rel=1e-4), s
        assert rep[s]["gap"] == pytest.approx(d.gap, rel=2e-2, abs=1e-4 * d.primal), s
