"""Non-binary data weighting W (Eq. (1): W weights the data residual, M masks
the TV term) through pcs_solve_slices_weighted, against the FP64 oracle run
with the same W and M = mask.
"""

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2006_09808_gb300 as pcs  # noqa: E402
import phantoms  # noqa: E402
from oracle import pd_oracle as O  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_09808_gb300 import build

    build.build()
    pcs.load_library()


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def steps(H):
    import os

    path = os.path.join(os.path.dirname(__file__), "golden", "opnorm_full_mask.txt")
    for line in open(path):
        t = line.split()
        if t and not t[0].startswith("#") and int(t[0]) == H and int(t[1]) == H and int(t[2]) == 0:
            L = float(t[3])
            return L, 1.0 / L, 1.0 / L
    raise KeyError(H)


def solve(pb, weight, n_iter, report=False, **opts):
    S, H, W = pb.field.shape
    f = torch.from_numpy(pb.field).cuda()
    m = torch.from_numpy(pb.mask).cuda()
    w = torch.from_numpy(weight).cuda()
    chi = torch.full_like(f, float("nan"))
    L, tau, sigma = steps(H)
    ctx = pcs.pcs_create(H, W, S, kernel=pcs.KERNEL_STREAMING, **opts)
    try:
        rep = pcs.pcs_solve_slices_weighted(ctx, f, m, w, pb.lam, tau, sigma, n_iter, chi, report=report)
        torch.cuda.synchronize()
    finally:
        pcs.pcs_destroy(ctx)
    return chi.cpu().numpy(), rep


@pytest.mark.parametrize("H,S,n_iter,lam", [(64, 3, 300, 1.0), (128, 2, 150, 1.0), (256, 2, 100, 5e-4)])
def test_weighted_parity(H, S, n_iter, lam):
    pb = phantoms.volume(H, H, S, seed=41, lam=lam, n_iter=n_iter)
    w = phantoms.magnitude_weight(pb.mask, seed=42)
    L, tau, sigma = steps(H)
    ref = O.pd_solve(pb.field.astype(np.float64), pb.mask, lam, tau, sigma, n_iter, weight=w.astype(np.float64))
    got, _ = solve(pb, w, n_iter)
    unweighted = O.pd_solve(pb.field.astype(np.float64), pb.mask, lam, tau, sigma, n_iter)
    for s in range(S):
        assert rel_l2(got[s], ref[s]) <= TOL, s
        # the weighting changes the solution well beyond the tolerance
        assert rel_l2(ref[s], unweighted[s]) > 100 * TOL, s


def test_binary_weight_is_bit_identical_to_the_unweighted_solve():
    pb = phantoms.volume(256, 256, 3, seed=43, lam=5e-4, n_iter=60)
    got, _ = solve(pb, pb.mask.astype(np.float32), 60)
    f = torch.from_numpy(pb.field).cuda()
    m = torch.from_numpy(pb.mask).cuda()
    chi = torch.empty_like(f)
    L, tau, sigma = steps(256)
    ctx = pcs.pcs_create(256, 256, 3, kernel=pcs.KERNEL_STREAMING)
    try:
        pcs.pcs_solve_slices(ctx, f, m, pb.lam, tau, sigma, 60, chi)
        torch.cuda.synchronize()
    finally:
        pcs.pcs_destroy(ctx)
    assert np.array_equal(got, chi.cpu().numpy())


def test_weighted_report_matches_oracle_diagnostics():
    pb = phantoms.volume(64, 64, 2, seed=44, lam=10.0, n_iter=200)
    w = phantoms.magnitude_weight(pb.mask, seed=45)
    L, tau, sigma = steps(64)
    got, rep = solve(pb, w, 200, report=True)
    for s in range(2):
        st = O.pd_solve(pb.field[s].astype(np.float64), pb.mask[s], pb.lam, tau, sigma, 200, weight=w[s].astype(np.float64),
                        return_state=True)
        d = O.diagnostics(st, pb.field[s].astype(np.float64), pb.mask[s], pb.lam, weight=w[s].astype(np.float64))
        r = rep[s]
        assert r["objective"] == pytest.approx(d.primal, rel=1e-4)
        assert r["data_residual"] == pytest.approx(d.data_residual, rel=1e-4)
        assert r["gap"] == pytest.approx(d.gap, rel=2e-2, abs=1e-4 * d.primal)
        assert r["stationarity"] == pytest.approx(d.stationarity, rel=2e-2, abs=1e-4)


def test_weighted_errors():
    lib = pcs.load_library()
    f = torch.zeros((1, 64, 64), device="cuda")
    m = torch.ones((1, 64, 64), dtype=torch.uint8, device="cuda")
    ctx = pcs.pcs_create(64, 64, 1, kernel=pcs.KERNEL_RESIDENT)
    try:
        with pytest.raises(pcs.PcsError) as ei:
            pcs.pcs_solve_slices_weighted(ctx, f, m, torch.ones_like(f), 1.0, 0.3, 0.3, 5, torch.empty_like(f))
        assert ei.value.status == pcs.PCS_EUNSUPPORTED
    finally:
        pcs.pcs_destroy(ctx)
    chi = torch.empty_like(f)
    ctx = pcs.pcs_create(64, 64, 1, kernel=pcs.KERNEL_STREAMING)
    try:
        st = lib.pcs_solve_slices_weighted(ctx, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(m.data_ptr()), None, 1,
                                           1.0, 0.3, 0.3, 5, ctypes.c_void_p(chi.data_ptr()), None)
        assert st == pcs.PCS_EINVAL
        assert "weight" in pcs.last_error()
    finally:
        pcs.pcs_destroy(ctx)
