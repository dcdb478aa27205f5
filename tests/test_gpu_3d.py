"""3-D variant (pcs_solve_volume_3d) against the FP64 3-D oracle.

The volume is one unknown (slices coupled through the 3-D dipole convolution
and the z differences), so every parity case runs the oracle on the whole
volume.  tau = sigma = 1/sqrt(4/9 + 12), a valid step for every 0/1 mask
(||D|| <= 2/3, ||G||^2 <= 12), the same on both sides.
"""

import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2006_09808_gb300 as pcs  # noqa: E402
import phantoms  # noqa: E402
from oracle import pd_oracle_3d as O3  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-4
STEP = 1.0 / math.sqrt(4.0 / 9.0 + 12.0)


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


def gpu3(field, mask, lam, n_iter, tv=0, weight=None, voxel=None):
    f = torch.from_numpy(np.array(field, dtype=np.float32)).cuda()
    m = torch.from_numpy(np.array(mask, dtype=np.uint8)).cuda()
    w = None if weight is None else torch.from_numpy(np.array(weight, dtype=np.float32)).cuda()
    chi = torch.full_like(f, float("nan"))
    pcs.pcs_solve_volume_3d(f, m, lam, STEP, STEP, n_iter, chi, tv=tv, weight=w, voxel=voxel)
    torch.cuda.synchronize()
    return chi.cpu().numpy()


@pytest.mark.parametrize(
    "S,H,n_iter,lam,tv",
    [(32, 64, 100, 1.0, 0), (32, 64, 100, 1.0, 1), (64, 64, 60, 1e-3, 0), (32, 128, 50, 1.0, 0),
     (128, 128, 10, 1.0, 0),  # 128 slices: the z transform of length 128, several slices per cluster
     (64, 128, 30, 5e-4, 0), (32, 256, 20, 5e-4, 1)],  # with the above: every pencil-form instance
)
def test_parity_3d(S, H, n_iter, lam, tv):
    pb = phantoms.volume(H, H, S, seed=51, lam=lam, n_iter=n_iter)
    ref = O3.pd_solve_3d(pb.field.astype(np.float64), pb.mask, lam, STEP, STEP, n_iter, tv="iso" if tv else "aniso")
    got = gpu3(pb.field, pb.mask, lam, n_iter, tv)
    assert np.all(np.isfinite(got))
    assert rel_l2(got, ref) <= TOL
    # per slice as well (the top and bottom slices see the z boundary)
    for s in (0, S // 2, S - 1):
        assert rel_l2(got[s], ref[s]) <= 10 * TOL, s


def test_parity_3d_at_the_bench_iteration_count():
    """64 x 64 x 32 after 500 iterations (the bench's count) against the whole-volume oracle:
    the volume and every slice within 1e-4."""
    n_iter = 500
    pb = phantoms.volume(64, 64, 32, seed=54, lam=5e-4, n_iter=n_iter)
    ref = O3.pd_solve_3d(pb.field.astype(np.float64), pb.mask, pb.lam, STEP, STEP, n_iter)
    got = gpu3(pb.field, pb.mask, pb.lam, n_iter)
    assert np.all(np.isfinite(got))
    assert rel_l2(got, ref) <= TOL
    for s in range(pb.field.shape[0]):
        assert rel_l2(got[s], ref[s]) <= TOL, s


def test_weighted_3d_parity():
    pb = phantoms.volume(64, 64, 32, seed=52, lam=1.0, n_iter=80)
    w = phantoms.magnitude_weight(pb.mask, seed=53)
    ref = O3.pd_solve_3d(pb.field.astype(np.float64), pb.mask, pb.lam, STEP, STEP, 80, weight=w.astype(np.float64))
    got = gpu3(pb.field, pb.mask, pb.lam, 80, weight=w)
    assert rel_l2(got, ref) <= TOL
    unweighted = O3.pd_solve_3d(pb.field.astype(np.float64), pb.mask, pb.lam, STEP, STEP, 80)
    assert rel_l2(ref, unweighted) > 100 * TOL
    # a 0/1 weight equal to the mask reproduces the unweighted solve bit for bit
    assert np.array_equal(gpu3(pb.field, pb.mask, pb.lam, 30, weight=pb.mask.astype(np.float32)),
                          gpu3(pb.field, pb.mask, pb.lam, 30))


def test_parity_3d_full_size_volume():
    """256 x 256 x 64, the bench volume, 20 iterations against the whole-volume oracle."""
    pb = phantoms.config2()
    n = 20
    ref = O3.pd_solve_3d(pb.field.astype(np.float64), pb.mask, pb.lam, STEP, STEP, n)
    got = gpu3(pb.field, pb.mask, pb.lam, n)
    assert rel_l2(got, ref) <= TOL
    m = pb.mask.astype(bool)
    assert rel_l2(got[m], ref[m]) <= TOL


def test_parity_3d_more_slices_than_resident_clusters():
    """256 x 256 x 128: more slices than the slice kernel's resident clusters, so clusters take
    several slices per launch; against the whole-volume oracle."""
    pb = phantoms.volume(256, 256, 128, seed=55, lam=5e-4, n_iter=6)
    ref = O3.pd_solve_3d(pb.field.astype(np.float64), pb.mask, pb.lam, STEP, STEP, pb.n_iter)
    got = gpu3(pb.field, pb.mask, pb.lam, pb.n_iter)
    assert np.all(np.isfinite(got))
    assert rel_l2(got, ref) <= TOL
    for s in (0, 63, 64, 127):
        assert rel_l2(got[s], ref[s]) <= 10 * TOL, s


def test_3d_edge_cases_and_errors():
    rng = np.random.default_rng(0)
    f = rng.standard_normal((32, 64, 64)).astype(np.float32)
    ones = np.ones_like(f, dtype=np.uint8)
    assert np.all(gpu3(f, ones, 1.0, 0) == 0)  # n_iter = 0
    assert np.all(gpu3(f, np.zeros_like(ones), 1.0, 20) == 0)  # empty mask
    one = gpu3(f, ones, 1.0, 1)
    assert rel_l2(one, O3.pd_solve_3d(f.astype(np.float64), ones, 1.0, STEP, STEP, 1)) <= 1e-6
    assert pcs.pcs_supported_volume_3d(64, 256, 256) and not pcs.pcs_supported_volume_3d(48, 256, 256)
    bad = torch.zeros((48, 64, 64), device="cuda")
    with pytest.raises(pcs.PcsError) as ei:
        pcs.pcs_solve_volume_3d(bad, torch.ones((48, 64, 64), dtype=torch.uint8, device="cuda"), 1.0, STEP, STEP, 5,
                                torch.empty_like(bad))
    assert ei.value.status == pcs.PCS_EUNSUPPORTED
    g = torch.zeros((32, 64, 64), device="cuda")
    with pytest.raises(pcs.PcsError) as ei:
        pcs.pcs_solve_volume_3d(g, torch.ones((32, 64, 64), dtype=torch.uint8, device="cuda"), -1.0, STEP, STEP, 5,
                                torch.empty_like(g))
    assert ei.value.status == pcs.PCS_EINVAL


@pytest.mark.parametrize("tv,weighted", [(0, False), (1, False), (0, True)])
def test_report_3d_against_oracle(tv, weighted):
    """FP64 diagnostics of the volume at (chi_N, p_N, q_N) against the oracle's, on the oracle's
    own state after the same iterations.  Objective and residual come from chi, which agrees to
    1e-4; the gap and the stationarity are differences of nearly equal terms, so they get a
    looser bound plus an absolute floor from the terms' size."""
    S, H, n_iter, lam = 32, 64, 120, 1.0
    pb = phantoms.volume(H, H, S, seed=54, lam=lam, n_iter=n_iter)
    w = phantoms.magnitude_weight(pb.mask, seed=55) if weighted else None
    wd = None if w is None else w.astype(np.float64)
    tvs = "iso" if tv else "aniso"
    st = O3.pd_solve_3d(pb.field.astype(np.float64), pb.mask, lam, STEP, STEP, n_iter, weight=wd, tv=tvs,
                        return_state=True)
    ref = O3.diagnostics_3d(st, pb.field, pb.mask, lam, weight=wd, tv=tvs)
    f = torch.from_numpy(np.ascontiguousarray(pb.field, dtype=np.float32)).cuda()
    m = torch.from_numpy(np.ascontiguousarray(pb.mask, dtype=np.uint8)).cuda()
    wt = None if w is None else torch.from_numpy(np.ascontiguousarray(w, dtype=np.float32)).cuda()
    chi = torch.empty_like(f)
    rep = pcs.pcs_solve_volume_3d(f, m, lam, STEP, STEP, n_iter, chi, tv=tv, weight=wt, report=True)
    torch.cuda.synchronize()
    assert rel_l2(chi.cpu().numpy(), st.chi) <= TOL
    assert rep["iters"] == n_iter
    assert rep["objective"] == pytest.approx(ref.primal, rel=1e-4)
    assert rep["data_residual"] == pytest.approx(ref.data_residual, rel=1e-4)
    assert rep["gap"] >= -1e-3 * ref.primal
    assert abs(rep["gap"] - ref.gap) <= 2e-2 * ref.gap + 1e-4 * ref.primal
    assert abs(rep["stationarity"] - ref.stationarity) <= 2e-2 * ref.stationarity + 1e-3


def test_report_3d_at_zero_start():
    """n_iter = 0: chi = p = q = 0, so objective = lambda/2 ||W dB||^2, gap = ||lambda W dB||^2 / (2 lambda),
    stationarity 0, residual ||W dB|| (closed forms, no oracle)."""
    pb = phantoms.volume(64, 64, 32, seed=56, lam=1.0, n_iter=1)
    lam = 0.5
    f = torch.from_numpy(np.ascontiguousarray(pb.field, dtype=np.float32)).cuda()
    m = torch.from_numpy(np.ascontiguousarray(pb.mask, dtype=np.uint8)).cuda()
    chi = torch.empty_like(f)
    rep = pcs.pcs_solve_volume_3d(f, m, lam, STEP, STEP, 0, chi, report=True)
    torch.cuda.synchronize()
    b2 = float(np.sum((pb.mask.astype(np.float64) * pb.field.astype(np.float32).astype(np.float64)) ** 2))
    assert rep["objective"] == pytest.approx(0.5 * lam * b2, rel=1e-12)
    assert rep["gap"] == pytest.approx(lam * b2 / 2.0, rel=1e-12)
    assert rep["data_residual"] == pytest.approx(math.sqrt(b2), rel=1e-12)
    assert rep["stationarity"] == 0.0


def test_anisotropic_voxels_3d():
    """The paper's voxel shape (2 mm slices, 0.72 mm pixels) against the oracle with the same
    voxel; unit or uniformly scaled voxels reproduce the isotropic solve bit for bit."""
    pb = phantoms.volume(64, 64, 32, seed=57, lam=1.0, n_iter=80)
    vox = (2.0, 0.72, 0.72)
    ref = O3.pd_solve_3d(pb.field.astype(np.float64), pb.mask, pb.lam, STEP, STEP, 80, voxel=vox)
    got = gpu3(pb.field, pb.mask, pb.lam, 80, voxel=vox)
    assert rel_l2(got, ref) <= TOL
    iso = O3.pd_solve_3d(pb.field.astype(np.float64), pb.mask, pb.lam, STEP, STEP, 80)
    assert rel_l2(ref, iso) > 100 * TOL  # the voxel shape matters
    base = gpu3(pb.field, pb.mask, pb.lam, 20)
    assert np.array_equal(gpu3(pb.field, pb.mask, pb.lam, 20, voxel=(1.0, 1.0, 1.0)), base)
    assert np.array_equal(gpu3(pb.field, pb.mask, pb.lam, 20, voxel=(2.5, 2.5, 2.5)), base)
    g = torch.zeros((32, 64, 64), device="cuda")
    with pytest.raises(pcs.PcsError) as ei:
        pcs.pcs_solve_volume_3d(g, torch.ones((32, 64, 64), dtype=torch.uint8, device="cuda"), 1.0, STEP, STEP, 5,
                                torch.empty_like(g), voxel=(1.0, 0.0, 1.0))
    assert ei.value.status == pcs.PCS_EINVAL
