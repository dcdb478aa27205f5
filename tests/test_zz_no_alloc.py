"""The allocation-free entry point pcs_solve_slices_noalloc.

Some callers may not allocate device memory once they run (a reconstruction
plug-in inside a host application that owns the GPU memory budget, code
inside another framework's memory pool).  For them the library offers one
solve entry point whose scratch lives in static device arrays.  These tests
check, through the C ABI, that it gives the same chi as the context-based
pcs_solve_slices (bit for bit: both run the same kernel on the same tables) on
two calls in a row of different slice sizes, so that the second call finds the
first call's state in the shared arrays; that a sampled slice matches the FP64
oracle; that a size used again after another size, or with the other B0 axis,
still gives its own result bit for bit (every size and axis has its own table
region); that repeated calls leave the free device memory unchanged; and that
a batch beyond the static limit is refused with a message.

This file is named to be collected last.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2006_09808_gb300 as pcs  # noqa: E402
import phantoms  # noqa: E402
from oracle import pd_oracle as O  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-4  # the relative-L2 tolerance of the parity tests
STEP = 1.0 / 2.95  # tau = sigma below 1/||K|| for every mask (||K|| <= sqrt(4/9 + 8))


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_09808_gb300 import build

    build.build()
    pcs.load_library()


def _context_solve(field, mask, lam, n_iter, b0_axis=0):
    S, H, W = field.shape
    chi = torch.empty_like(field)
    ctx = pcs.pcs_create(H, W, S, b0_axis=b0_axis)
    try:
        pcs.pcs_solve_slices(ctx, field, mask, lam, STEP, STEP, n_iter, chi)
        torch.cuda.synchronize()
    finally:
        pcs.pcs_destroy(ctx)
    return chi.cpu().numpy()


def _noalloc_solve(field, mask, lam, n_iter, b0_axis=0):
    chi = torch.full_like(field, float("nan"))
    pcs.pcs_solve_slices_noalloc(field, mask, lam, STEP, STEP, n_iter, chi, b0_axis=b0_axis)
    torch.cuda.synchronize()
    return chi.cpu().numpy()


def _problem(H, S, seed, lam, n_iter):
    pb = phantoms.volume(H, H, S, seed=seed, lam=lam, n_iter=n_iter)
    return pb, torch.from_numpy(pb.field).cuda(), torch.from_numpy(pb.mask).cuda()


def test_noalloc_matches_context_entry_point_two_calls():
    cases = [(256, 8, 1, 5e-4, 60), (64, 5, 2, 1e-2, 120)]
    for H, S, seed, lam, n_iter in cases:
        pb, field, mask = _problem(H, S, seed, lam, n_iter)
        ref = _context_solve(field, mask, lam, n_iter)
        got = _noalloc_solve(field, mask, lam, n_iter)
        assert np.all(np.isfinite(got))
        assert np.array_equal(got, ref), H  # same kernel, same tables: bit for bit
        s = S // 2  # and the FP64 oracle on a sampled slice
        want = O.pd_solve(pb.field[s].astype(np.float64), pb.mask[s], lam, STEP, STEP, n_iter)
        rel = np.linalg.norm(got[s].astype(np.float64) - want) / np.linalg.norm(want)
        assert rel <= TOL, (H, rel)


def test_noalloc_sizes_and_axes_keep_their_own_tables():
    pb256, f256, m256 = _problem(256, 3, 7, 1e-3, 40)
    _, f64, m64 = _problem(64, 4, 8, 1e-3, 40)
    first = _noalloc_solve(f256, m256, pb256.lam, 40)
    _noalloc_solve(f64, m64, pb256.lam, 40)  # another size in between
    assert np.array_equal(_noalloc_solve(f256, m256, pb256.lam, 40), first)
    # B0 along x: its own region, equal to a context created with b0_axis = 1
    along_x = _noalloc_solve(f256, m256, pb256.lam, 40, b0_axis=1)
    assert np.array_equal(along_x, _context_solve(f256, m256, pb256.lam, 40, b0_axis=1))
    assert not np.array_equal(along_x, first)
    assert np.array_equal(_noalloc_solve(f256, m256, pb256.lam, 40), first)


def test_noalloc_repeated_calls_allocate_nothing():
    pb = phantoms.volume(128, 128, 4, seed=3, lam=1e-3, n_iter=20)
    field = torch.from_numpy(pb.field).cuda()
    mask = torch.from_numpy(pb.mask).cuda()
    chi = torch.empty_like(field)
    pcs.pcs_solve_slices_noalloc(field, mask, pb.lam, STEP, STEP, pb.n_iter, chi)  # device set-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        pcs.pcs_solve_slices_noalloc(field, mask, pb.lam, STEP, STEP, pb.n_iter, chi)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_batches_beyond_the_static_limit():
    # 17 slices of 256 x 256 = 1,114,112 voxels > PCS_NOALLOC_MAX_VOXELS (1,048,576)
    field = torch.zeros((17, 256, 256), device="cuda")
    mask = torch.ones((17, 256, 256), dtype=torch.uint8, device="cuda")
    with pytest.raises(pcs.PcsError) as ei:
        pcs.pcs_solve_slices_noalloc(field, mask, 1e-3, STEP, STEP, 5, torch.empty_like(field))
    assert ei.value.status == pcs.PCS_EINVAL
    assert "exceeds the static scratch" in str(ei.value)
