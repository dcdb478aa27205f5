"""Field-map preprocessing (pcs_field_map) against the FP64 oracle, and the
whole chain echoes -> field map -> weighted solve against the oracle chain."""

import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2006_09808_gb300 as pcs  # noqa: E402
import phantoms  # noqa: E402
from oracle import field_map as FM  # noqa: E402
from oracle import pd_oracle as O  # noqa: E402

pytestmark = pytest.mark.gpu
T_SHIFT, B0 = 0.6e-3, 3.0


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_09808_gb300 import build

    build.build()
    pcs.load_library()


def gpu_map(s0, s1, thr):
    a = torch.from_numpy(np.ascontiguousarray(s0)).cuda()
    b = torch.from_numpy(np.ascontiguousarray(s1)).cuda()
    f = torch.empty(s0.shape, dtype=torch.float32, device="cuda")
    w = torch.empty_like(f)
    m = torch.empty(s0.shape, dtype=torch.uint8, device="cuda")
    pcs.pcs_field_map(a, b, T_SHIFT, B0, thr, f, w, m)
    torch.cuda.synchronize()
    return f.cpu().numpy(), w.cpu().numpy(), m.cpu().numpy()


def check_mask(m, rm, s0, thr, max_frac=1e-4):
    """GPU mask (a float32 decision) against the oracle's FP64 decision: they may differ only at
    voxels within float32 rounding of the threshold, and those must be few.  Returns the voxels
    where the two agree."""
    diff = m != rm
    band = FM.mask_boundary_band(s0, thr)
    assert not np.any(diff & ~band), f"{int(np.sum(diff & ~band))} mask voxels differ outside the rounding band"
    assert diff.sum() <= max(1, max_frac * m.size), int(diff.sum())
    return ~diff


def phase_err(a, b):
    """Difference of two fields as a phase, folded into (-pi, pi]."""
    d = (np.asarray(a, np.float64) - np.asarray(b, np.float64)) / FM.ppm_per_radian(B0, T_SHIFT)
    return np.abs((d + np.pi) % (2 * np.pi) - np.pi)


@pytest.mark.parametrize("H,S,thr", [(64, 3, 0.3), (256, 16, 0.25)])
def test_field_map_parity(H, S, thr):
    pb = phantoms.volume(H, H, S, seed=61)
    s0, s1 = phantoms.echo_pair(pb.field, pb.mask, seed=62)
    f, w, m = gpu_map(s0, s1, thr)
    rf, rw, rm = FM.field_map(s0, s1, T_SHIFT, B0, thr)
    agree = check_mask(m, rm, s0, thr)
    assert 0 < m.sum() < m.size
    assert np.max(np.abs(w - rw)) <= 1e-6
    assert np.max(phase_err(f, rf)[agree]) <= 1e-5
    assert np.all(f[m == 0] == 0)


def test_noise_free_field_recovery():
    rng = np.random.default_rng(3)
    shape = (2, 32, 48)
    truth = rng.uniform(-5.0, 5.0, shape)  # |phase| < pi
    mag = rng.uniform(0.5, 1.0, shape)
    phi0 = rng.uniform(-np.pi, np.pi, shape)
    kappa = 1.0 / FM.ppm_per_radian(B0, T_SHIFT)
    s0 = (mag * np.exp(1j * phi0)).astype(np.complex64)
    s1 = (mag * np.exp(1j * (phi0 + kappa * truth))).astype(np.complex64)
    f, w, m = gpu_map(s0, s1, 0.0)
    assert m.all()
    assert np.max(np.abs(f - truth)) <= 2e-5
    assert w.max() == 1.0


def test_pipeline_echoes_to_chi_matches_the_oracle_chain():
    pb = phantoms.volume(64, 64, 3, seed=63, lam=1.0, n_iter=200)
    s0, s1 = phantoms.echo_pair(pb.field, pb.mask, seed=64)
    f, w, m = gpu_map(s0, s1, 0.3)
    rf, rw, rm = FM.field_map(s0, s1, T_SHIFT, B0, 0.3)
    check_mask(m, rm, s0, 0.3)
    assert np.array_equal(m, rm)  # this seeded volume has no voxel in the rounding band: the chains agree
    L = 2.832522691076350  # full-mask ||K|| of 64 x 64 (tests/golden/opnorm_full_mask.txt)
    ref = O.pd_solve(rf, rm, pb.lam, 1 / L, 1 / L, pb.n_iter, weight=rw)
    ft, mt, wt = (torch.from_numpy(a).cuda() for a in (f, m, w))
    chi = torch.empty_like(ft)
    ctx = pcs.pcs_create(64, 64, 3, kernel=pcs.KERNEL_STREAMING)
    try:
        pcs.pcs_solve_slices_weighted(ctx, ft, mt, wt, pb.lam, 1 / L, 1 / L, pb.n_iter, chi)
        torch.cuda.synchronize()
    finally:
        pcs.pcs_destroy(ctx)
    got = chi.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-4


def test_field_map_edges_and_errors():
    z = torch.zeros((0,), dtype=torch.complex64, device="cuda")
    pcs.pcs_field_map(z, z, T_SHIFT, B0, 0.1, torch.empty(0, device="cuda"), torch.empty(0, device="cuda"),
                      torch.empty(0, dtype=torch.uint8, device="cuda"))
    a = torch.ones((4, 4), dtype=torch.complex64, device="cuda")
    out = [torch.empty((4, 4), device="cuda"), torch.empty((4, 4), device="cuda"),
           torch.empty((4, 4), dtype=torch.uint8, device="cuda")]
    with pytest.raises(pcs.PcsError) as ei:
        pcs.pcs_field_map(a, a, T_SHIFT, B0, -0.1, *out)
    assert ei.value.status == pcs.PCS_EINVAL
    with pytest.raises(pcs.PcsError) as ei:
        pcs.pcs_field_map(a, a, 0.0, B0, 0.1, *out)
    assert ei.value.status == pcs.PCS_EINVAL
    pcs.pcs_field_map(a, a, T_SHIFT, B0, 0.5, *out)
    torch.cuda.synchronize()
    assert torch.all(out[2] == 1) and torch.all(out[0] == 0) and torch.all(out[1] == 1)
    # an odd voxel count (the last voxel is handled apart from the 16-byte pairs)
    rng = np.random.default_rng(5)
    shape = (3, 5, 7)
    s0 = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)
    s1 = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)
    f, w, m = gpu_map(s0, s1, 0.4)
    rf, rw, rm = FM.field_map(s0, s1, T_SHIFT, B0, 0.4)
    agree = check_mask(m, rm, s0, 0.4)
    assert np.max(np.abs(w - rw)) <= 1e-6 and np.max(phase_err(f, rf)[agree]) <= 1e-5
    # inputs off their 16-byte alignment are refused
    z1 = torch.ones(17, dtype=torch.complex64, device="cuda")[1:]
    o1 = [torch.empty(16, device="cuda"), torch.empty(16, device="cuda"), torch.empty(16, dtype=torch.uint8, device="cuda")]
    with pytest.raises(pcs.PcsError) as ei:
        pcs.pcs_field_map(z1, z1, T_SHIFT, B0, 0.1, *o1)
    assert ei.value.status == pcs.PCS_EINVAL
