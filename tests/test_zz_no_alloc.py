"""The allocation-free entry point pcs_solve_slices_noalloc.

Some callers may not allocate device memory once they run (a reconstruction
plug-in inside a host application that owns the GPU memory budget, code
inside another framework's memory pool).  For them the library offers one
solve entry point whose scratch lives in static device arrays.  These tests
check, through the C ABI, that it gives the same chi as the context-based
pcs_solve_slices on two calls in a row (different slice sizes, so the second
call finds the first call's state and tables in the shared arrays), that
repeated calls leave the free device memory unchanged, and that a batch
beyond the static limit is refused with a message.

This file is named to be collected last.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2006_09808_gb300 as pcs  # noqa: E402
import phantoms  # noqa: E402

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


def _context_solve(field, mask, lam, n_iter):
    S, H, W = field.shape
    chi = torch.empty_like(field)
    ctx = pcs.pcs_create(H, W, S)
    try:
        pcs.pcs_solve_slices(ctx, field, mask, lam, STEP, STEP, n_iter, chi)
        torch.cuda.synchronize()
    finally:
        pcs.pcs_destroy(ctx)
    return chi.cpu().numpy().astype(np.float64)


def test_noalloc_matches_context_entry_point_two_calls():
    cases = [(256, 8, 1, 5e-4, 60), (64, 5, 2, 1e-2, 120)]
    for H, S, seed, lam, n_iter in cases:
        pb = phantoms.volume(H, H, S, seed=seed, lam=lam, n_iter=n_iter)
        field = torch.from_numpy(pb.field).cuda()
        mask = torch.from_numpy(pb.mask).cuda()
        ref = _context_solve(field, mask, lam, n_iter)
        chi = torch.full_like(field, float("nan"))
        pcs.pcs_solve_slices_noalloc(field, mask, lam, STEP, STEP, n_iter, chi)
        torch.cuda.synchronize()
        got = chi.cpu().numpy().astype(np.float64)
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert np.all(np.isfinite(got))
        assert rel <= TOL, (H, rel)


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
