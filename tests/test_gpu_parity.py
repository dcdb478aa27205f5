"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerance: relative L2 error of chi_N <= 1e-4 after the same iteration count,
tau, sigma and lambda (the stated target of this solver); probes of FP32
against FP64 arithmetic put the expected error near 1e-6, so 1e-4 leaves room
for FFT rounding growth at 512 x 512.

Step sizes: tau = sigma = 1/L with L = ||K||_2 of the full-mask operator from
the oracle's FP64 power iteration, passed to both sides.
"""

import functools

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


@functools.lru_cache(maxsize=None)
def _golden_L():
    import os

    table = {}
    path = os.path.join(os.path.dirname(__file__), "golden", "opnorm_full_mask.txt")
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            H, W, ax, L = line.split()
            table[(int(H), int(W), int(ax))] = float(L)
    return table


def steps(H, W, b0_axis=0):
    """(L, tau, sigma) = (||K||, 1/L, 1/L) of the full-mask operator, from the
    oracle-written table (tests/golden/make_step_sizes.py), else the oracle."""
    L = _golden_L().get((H, W, b0_axis))
    if L is None:
        L = O.opnorm(np.ones((H, W)), b0_axis=b0_axis)
    return L, 1.0 / L, 1.0 / L


def rel_l2(a, b, mask=None):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    if mask is not None:
        a, b = a[mask], b[mask]
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def gpu_solve(field, mask, lam, tau, sigma, n_iter, **opts):
    S, H, W = field.shape
    f = torch.from_numpy(np.ascontiguousarray(field, dtype=np.float32)).cuda()
    m = torch.from_numpy(np.ascontiguousarray(mask, dtype=np.uint8)).cuda()
    chi = torch.full_like(f, float("nan"))
    ctx = pcs.pcs_create(H, W, S, **opts)
    try:
        pcs.pcs_solve_slices(ctx, f, m, lam, tau, sigma, n_iter, chi)
        torch.cuda.synchronize()
    finally:
        pcs.pcs_destroy(ctx)
    return chi.cpu().numpy()


def oracle_solve(field, mask, lam, tau, sigma, n_iter):
    return O.pd_solve(np.asarray(field, np.float64), mask, lam, tau, sigma, n_iter)


# --------------------------------------------------------------------------- configurations


def test_config1_parity():
    pb = phantoms.config1()
    L, tau, sigma = steps(64, 64)
    ref = oracle_solve(pb.field, pb.mask, pb.lam, tau, sigma, pb.n_iter)
    got = gpu_solve(pb.field, pb.mask, pb.lam, tau, sigma, pb.n_iter)
    assert np.all(np.isfinite(got))
    assert rel_l2(got, ref) <= TOL


@pytest.mark.parametrize("lam", [1e-3, 1.0, 10.0])
def test_parity_64_regimes(lam):
    pb = phantoms.volume(64, 64, 3, seed=11, lam=lam, n_iter=300)
    L, tau, sigma = steps(64, 64)
    ref = oracle_solve(pb.field, pb.mask, lam, tau, sigma, pb.n_iter)
    got = gpu_solve(pb.field, pb.mask, lam, tau, sigma, pb.n_iter)
    for s in range(3):
        assert rel_l2(got[s], ref[s]) <= TOL, s


STREAMING, RESIDENT = pcs.KERNEL_STREAMING, pcs.KERNEL_RESIDENT


@pytest.mark.parametrize("kernel,cluster_size", [(RESIDENT, 4), (STREAMING, 1), (STREAMING, 2)])
def test_parity_128(kernel, cluster_size):
    pb = phantoms.volume(128, 128, 3, seed=5, lam=5e-4, n_iter=200)
    L, tau, sigma = steps(128, 128)
    ref = oracle_solve(pb.field, pb.mask, pb.lam, tau, sigma, pb.n_iter)
    got = gpu_solve(pb.field, pb.mask, pb.lam, tau, sigma, pb.n_iter, cluster_size=cluster_size, kernel=kernel)
    for s in range(3):
        assert rel_l2(got[s], ref[s]) <= TOL, s


@pytest.mark.parametrize(
    "kernel,cluster_size,threads",
    [(RESIDENT, 8, 256), (RESIDENT, 8, 512), (STREAMING, 2, 256), (STREAMING, 4, 256), (STREAMING, 4, 512),
     (STREAMING, 8, 256)],
)
def test_parity_256_kernel_variants(kernel, cluster_size, threads):
    pb = phantoms.volume(256, 256, 2, seed=21, lam=5e-4, n_iter=100)
    L, tau, sigma = steps(256, 256)
    ref = oracle_solve(pb.field, pb.mask, pb.lam, tau, sigma, pb.n_iter)
    got = gpu_solve(pb.field, pb.mask, pb.lam, tau, sigma, pb.n_iter, cluster_size=cluster_size, kernel=kernel,
                    threads=threads)
    for s in range(2):
        assert rel_l2(got[s], ref[s]) <= TOL, s


@pytest.mark.parametrize("kernel", [RESIDENT, STREAMING])
def test_parity_64_kernels_ragged_mask(kernel):
    rng = np.random.default_rng(12)
    pb = phantoms.volume(64, 64, 3, seed=13, lam=0.5, n_iter=150)
    mask = (rng.random(pb.mask.shape) > 0.2).astype(np.uint8) * pb.mask
    L, tau, sigma = steps(64, 64)
    ref = oracle_solve(pb.field, mask, pb.lam, tau, sigma, pb.n_iter)
    got = gpu_solve(pb.field, mask, pb.lam, tau, sigma, pb.n_iter, kernel=kernel)
    for s in range(3):
        assert rel_l2(got[s], ref[s]) <= TOL, s


def test_resident_and_streaming_kernels_agree_at_full_size():
    pb = phantoms.volume(256, 256, 16, seed=31, lam=5e-4, n_iter=200)
    L, tau, sigma = steps(256, 256)
    a = gpu_solve(pb.field, pb.mask, pb.lam, tau, sigma, pb.n_iter, kernel=RESIDENT)
    b = gpu_solve(pb.field, pb.mask, pb.lam, tau, sigma, pb.n_iter, kernel=STREAMING)
    for s in range(16):
        assert rel_l2(a[s], b[s]) <= 1e-5, s


@pytest.mark.parametrize("H,S,cluster_size", [(128, 48, 4), (64, 200, 1)])
def test_resident_kernel_with_more_slices_than_resident_clusters(H, S, cluster_size):
    """The resident kernel's slice loop, with more slices than clusters on the GPU at
    once: every cluster solves several slices in turn, each from a zero start.  Each
    sampled slice must equal, bit for bit, the same slice solved alone, and the oracle
    within the tolerance."""
    pb = phantoms.volume(H, H, S, seed=37, lam=5e-4, n_iter=60)
    L, tau, sigma = steps(H, H)
    opts = dict(kernel=RESIDENT, cluster_size=cluster_size)
    got = gpu_solve(pb.field, pb.mask, pb.lam, tau, sigma, pb.n_iter, **opts)
    assert np.all(np.isfinite(got))
    for s in (0, S // 2, S - 1):
        alone = gpu_solve(pb.field[s:s + 1], pb.mask[s:s + 1], pb.lam, tau, sigma, pb.n_iter, **opts)
        assert np.array_equal(got[s], alone[0]), s
    for s in (0, S - 1):
        ref = oracle_solve(pb.field[s], pb.mask[s], pb.lam, tau, sigma, pb.n_iter)
        assert rel_l2(got[s], ref) <= TOL, s


def test_config2_full_size_sampled_slices():
    """256 x 256 x 64, 500 iterations, in the bench's launch configuration; the
    oracle solves three sampled slices (first, middle, last)."""
    pb = phantoms.config2()
    L, tau, sigma = steps(256, 256)
    got = gpu_solve(pb.field, pb.mask, pb.lam, tau, sigma, pb.n_iter)
    assert np.all(np.isfinite(got))
    for s in (0, 31, 63):
        ref = oracle_solve(pb.field[s], pb.mask[s], pb.lam, tau, sigma, pb.n_iter)
        assert rel_l2(got[s], ref) <= TOL, s
        assert rel_l2(got[s], ref, pb.mask[s].astype(bool)) <= TOL, s


def test_parity_512():
    pb = phantoms.volume(512, 512, 2, seed=3, lam=1e-3, n_iter=60)
    L, tau, sigma = steps(512, 512)
    ref = oracle_solve(pb.field, pb.mask, pb.lam, tau, sigma, pb.n_iter)
    got = gpu_solve(pb.field, pb.mask, pb.lam, tau, sigma, pb.n_iter)
    for s in range(2):
        assert rel_l2(got[s], ref[s]) <= TOL, s


@pytest.mark.parametrize("H,S,n_iter", [(192, 3, 120), (384, 2, 60)])
def test_parity_radix3_sizes(H, S, n_iter):
    pb = phantoms.volume(H, H, S, seed=H, lam=5e-4, n_iter=n_iter)
    L, tau, sigma = steps(H, H)
    ref = oracle_solve(pb.field, pb.mask, pb.lam, tau, sigma, pb.n_iter)
    got = gpu_solve(pb.field, pb.mask, pb.lam, tau, sigma, pb.n_iter)
    for s in range(S):
        assert rel_l2(got[s], ref[s]) <= TOL, s


def test_graph_replay_matches_direct_launch():
    pb = phantoms.volume(128, 128, 4, seed=41, lam=1e-3, n_iter=60)
    L, tau, sigma = steps(128, 128)
    direct = gpu_solve(pb.field, pb.mask, pb.lam, tau, sigma, pb.n_iter)
    stream = torch.cuda.Stream()
    f = torch.from_numpy(pb.field).cuda()
    m = torch.from_numpy(pb.mask).cuda()
    chi = torch.empty_like(f)
    ctx = pcs.pcs_create(128, 128, 4, use_graph=True, stream=stream)
    try:
        for n_iter in (pb.n_iter, pb.n_iter, 7, pb.n_iter):  # replay, re-capture, re-capture
            with torch.cuda.stream(stream):
                chi.fill_(float("nan"))
                pcs.pcs_solve_slices(ctx, f, m, pb.lam, tau, sigma, n_iter, chi)
            stream.synchronize()
            if n_iter == pb.n_iter:
                assert np.array_equal(chi.cpu().numpy(), direct)
    finally:
        pcs.pcs_destroy(ctx)
    with pytest.raises(pcs.PcsError) as ei:  # the legacy stream cannot be captured
        lib = pcs.load_library()
        opt = pcs.pcs_options()
        lib.pcs_options_default(opt)
        opt.use_graph = 1
        h = __import__("ctypes").c_void_p()
        pcs._check(lib.pcs_create(h, 128, 128, 1, opt, None), "pcs_create")
    assert ei.value.status == pcs.PCS_EINVAL


def test_b0_along_columns():
    pb = phantoms.volume(64, 64, 2, seed=8, lam=1.0, n_iter=120)
    L, _, _ = steps(64, 64, b0_axis=1)
    ref = O.pd_solve(pb.field.astype(np.float64), pb.mask, pb.lam, 1 / L, 1 / L, pb.n_iter, b0_axis=1)
    got = gpu_solve(pb.field, pb.mask, pb.lam, 1 / L, 1 / L, pb.n_iter, b0_axis=1)
    assert rel_l2(got, ref) <= TOL


# --------------------------------------------------------------------------- structure and edge cases


@pytest.mark.parametrize("kernel", [RESIDENT, STREAMING])
def test_batch_invariance_bitwise(kernel):
    """A slice gives bit-identical chi alone, inside a batch, and at another batch position."""
    pb = phantoms.volume(256, 256, 6, seed=2, lam=5e-4, n_iter=40)
    L, tau, sigma = steps(256, 256)
    batch = gpu_solve(pb.field, pb.mask, pb.lam, tau, sigma, pb.n_iter, kernel=kernel)
    alone = gpu_solve(pb.field[4:5], pb.mask[4:5], pb.lam, tau, sigma, pb.n_iter, kernel=kernel)
    assert np.array_equal(batch[4], alone[0])
    perm = [4, 0, 1, 2, 3, 5]
    shuffled = gpu_solve(pb.field[perm], pb.mask[perm], pb.lam, tau, sigma, pb.n_iter, kernel=kernel)
    assert np.array_equal(shuffled[0], batch[4])
    few = gpu_solve(pb.field, pb.mask, pb.lam, tau, sigma, pb.n_iter, max_clusters=1, kernel=kernel)
    assert np.array_equal(few, batch)


def test_edge_cases():
    L, tau, sigma = steps(64, 64)
    rng = np.random.default_rng(0)
    f = rng.standard_normal((2, 64, 64)).astype(np.float32)
    ones = np.ones((2, 64, 64), np.uint8)
    assert np.all(gpu_solve(f, ones, 0.1, tau, sigma, 0) == 0)  # n_iter = 0
    assert np.all(gpu_solve(np.zeros_like(f), ones, 0.1, tau, sigma, 25) == 0)  # f = 0
    assert np.all(gpu_solve(f, np.zeros_like(ones), 0.1, tau, sigma, 25) == 0)  # empty mask
    one = gpu_solve(f, ones, 0.1, tau, sigma, 1)
    assert rel_l2(one, oracle_solve(f, ones, 0.1, tau, sigma, 1)) <= 1e-6
    # ragged masks: holes and a mask touching the slice border
    m = (rng.random((2, 64, 64)) > 0.3).astype(np.uint8)
    m[:, 0, :] = 1
    m[:, :, -1] = 1
    got = gpu_solve(f, m, 0.5, tau, sigma, 80)
    assert rel_l2(got, oracle_solve(f, m, 0.5, tau, sigma, 80)) <= TOL
    # empty batch is a no-op
    ctx = pcs.pcs_create(64, 64, 4)
    try:
        e = torch.empty((0, 64, 64), device="cuda")
        pcs.pcs_solve_slices(ctx, e, torch.empty((0, 64, 64), dtype=torch.uint8, device="cuda"), 0.1, tau,
                             sigma, 5, torch.empty((0, 64, 64), device="cuda"))
    finally:
        pcs.pcs_destroy(ctx)


def test_error_codes_on_gpu():
    ctx = pcs.pcs_create(64, 64, 2)
    try:
        f = torch.zeros((3, 64, 64), device="cuda")
        m = torch.ones((3, 64, 64), dtype=torch.uint8, device="cuda")
        with pytest.raises(pcs.PcsError) as ei:
            pcs.pcs_solve_slices(ctx, f, m, 0.1, 0.3, 0.3, 5, torch.empty_like(f))
        assert ei.value.status == pcs.PCS_EINVAL
        f2, m2 = f[:2], m[:2]
        for lam, tau, sigma, n in [(0.0, 0.3, 0.3, 5), (0.1, -1.0, 0.3, 5), (0.1, 0.3, 0.3, -1)]:
            with pytest.raises(pcs.PcsError) as ei:
                pcs.pcs_solve_slices(ctx, f2, m2, lam, tau, sigma, n, torch.empty_like(f2))
            assert ei.value.status == pcs.PCS_EINVAL
        buf = torch.zeros(2 * 64 * 64 + 1, device="cuda")
        mis = buf[1:].view(2, 64, 64)  # 4-byte offset: misaligned
        with pytest.raises(pcs.PcsError) as ei:
            pcs.pcs_solve_slices(ctx, mis, m2, 0.1, 0.3, 0.3, 5, torch.empty_like(f2))
        assert ei.value.status == pcs.PCS_EINVAL
    finally:
        pcs.pcs_destroy(ctx)
    with pytest.raises(pcs.PcsError) as ei:  # no compiled kernel, and 134 = 2 x 67 outside the any-size rule
        pcs.pcs_create(96, 134, 1)
    assert ei.value.status == pcs.PCS_EUNSUPPORTED


# --------------------------------------------------------------------------- diagnostics, step size, host path


def test_report_matches_oracle_diagnostics():
    pb = phantoms.volume(64, 64, 2, seed=4, lam=10.0, n_iter=200)
    L, tau, sigma = steps(64, 64)
    f = torch.from_numpy(pb.field).cuda()
    m = torch.from_numpy(pb.mask).cuda()
    chi = torch.empty_like(f)
    ctx = pcs.pcs_create(64, 64, 2)
    try:
        rep = pcs.pcs_solve_slices(ctx, f, m, pb.lam, tau, sigma, pb.n_iter, chi, report=True)
    finally:
        pcs.pcs_destroy(ctx)
    for s in range(2):
        st = O.pd_solve(pb.field[s].astype(np.float64), pb.mask[s], pb.lam, tau, sigma, pb.n_iter,
                        return_state=True)
        d = O.diagnostics(st, pb.field[s].astype(np.float64), pb.mask[s], pb.lam)
        r = rep[s]
        assert r["iters"] == pb.n_iter
        assert r["objective"] == pytest.approx(d.primal, rel=1e-4)
        assert r["data_residual"] == pytest.approx(d.data_residual, rel=1e-4)
        assert r["gap"] == pytest.approx(d.gap, rel=2e-2, abs=1e-4 * d.primal)
        assert r["stationarity"] == pytest.approx(d.stationarity, rel=2e-2, abs=1e-4)
        assert r["gap"] >= 0


# --------------------------------------------------------------------------- isotropic TV


@pytest.mark.parametrize(
    "H,S,n_iter,kernel,cluster_size",
    [(64, 3, 300, RESIDENT, 0), (64, 3, 300, STREAMING, 1), (128, 2, 150, RESIDENT, 4),
     (256, 2, 100, STREAMING, 4), (256, 2, 100, RESIDENT, 8)],
)
def test_isotropic_tv_parity(H, S, n_iter, kernel, cluster_size):
    """tv = 1: the dual TV prox projects each pixel's (qx, qy) onto the unit
    disc; against the oracle's isotropic reading of Eq. (1)."""
    pb = phantoms.volume(H, H, S, seed=31, lam=1.0, n_iter=n_iter)  # lambda large enough for |q| to reach 1
    L, tau, sigma = steps(H, H)
    ref = O.pd_solve(pb.field.astype(np.float64), pb.mask, pb.lam, tau, sigma, n_iter, tv="iso")
    got = gpu_solve(pb.field, pb.mask, pb.lam, tau, sigma, n_iter, kernel=kernel, cluster_size=cluster_size, tv=1)
    aniso = gpu_solve(pb.field, pb.mask, pb.lam, tau, sigma, n_iter, kernel=kernel, cluster_size=cluster_size)
    for s in range(S):
        assert rel_l2(got[s], ref[s]) <= TOL, s
        # the two readings give different minimisers on these phantoms
        assert rel_l2(got[s], aniso[s]) > 100 * TOL, s


def test_isotropic_tv_report_matches_oracle_diagnostics():
    pb = phantoms.volume(64, 64, 2, seed=4, lam=10.0, n_iter=200)
    L, tau, sigma = steps(64, 64)
    f = torch.from_numpy(pb.field).cuda()
    m = torch.from_numpy(pb.mask).cuda()
    chi = torch.empty_like(f)
    ctx = pcs.pcs_create(64, 64, 2, tv=1)
    try:
        rep = pcs.pcs_solve_slices(ctx, f, m, pb.lam, tau, sigma, pb.n_iter, chi, report=True)
    finally:
        pcs.pcs_destroy(ctx)
    for s in range(2):
        st = O.pd_solve(pb.field[s].astype(np.float64), pb.mask[s], pb.lam, tau, sigma, pb.n_iter,
                        return_state=True, tv="iso")
        d = O.diagnostics(st, pb.field[s].astype(np.float64), pb.mask[s], pb.lam, tv="iso")
        r = rep[s]
        assert r["objective"] == pytest.approx(d.primal, rel=1e-4)
        assert r["gap"] == pytest.approx(d.gap, rel=2e-2, abs=1e-4 * d.primal)
        assert r["stationarity"] == pytest.approx(d.stationarity, rel=2e-2, abs=1e-4)
        assert r["gap"] >= 0


@pytest.mark.parametrize("H,kind", [(64, "full"), (256, "full"), (128, "ellipse")])
def test_opnorm_matches_oracle(H, kind):
    mask = np.ones((H, H), np.uint8) if kind == "full" else phantoms.ellipse_mask(H, H)
    ref = O.opnorm(mask)
    ctx = pcs.pcs_create(H, H, 2)
    try:
        m = torch.from_numpy(np.stack([mask, mask])).cuda()
        got = pcs.pcs_opnorm(ctx, m, 400)
    finally:
        pcs.pcs_destroy(ctx)
    for g in got:
        # a Rayleigh quotient never exceeds the top eigenvalue; 400 steps get within 0.2%
        assert ref * (1 - 2e-3) <= g <= ref * (1 + 1e-5)


def test_host_buffer_entry_point_matches_device_path():
    pb = phantoms.volume(128, 128, 4, seed=9, lam=1e-3, n_iter=50)
    L, tau, sigma = steps(128, 128)
    dev = gpu_solve(pb.field, pb.mask, pb.lam, tau, sigma, pb.n_iter)
    out = np.empty_like(pb.field)
    ctx = pcs.pcs_create(128, 128, 4)
    try:
        pcs.pcs_solve_slices_host(ctx, pb.field, pb.mask, pb.lam, tau, sigma, pb.n_iter, out)
    finally:
        pcs.pcs_destroy(ctx)
    assert np.array_equal(out, dev)


@pytest.mark.parametrize("H", [64, 128, 192, 256, 384, 512])
def test_every_compiled_variant_matches_the_oracle(H):
    """Every compiled variant of a slice size (cluster shape, kernel kind, threads per CTA, FFT
    tile shape), listed by the autotuner's candidate record, against the FP64 oracle."""
    pb = phantoms.volume(H, H, 2, seed=40 + H, lam=5e-4, n_iter=60)
    batch = pcs.pcs_batch_create(autotune=True)
    try:
        f = torch.from_numpy(pb.field).cuda()
        m = torch.from_numpy(pb.mask).cuda()
        pcs.pcs_batch_solve(batch, [(f, m, pb.lam, torch.empty_like(f))], 2)
        pcs.pcs_batch_check(batch)
        cands = pcs.pcs_batch_tuning(batch, H, H)["candidates"]
    finally:
        pcs.pcs_batch_destroy(batch)
    assert len(cands) >= 1
    L, tau, sigma = steps(H, H)
    ref = oracle_solve(pb.field, pb.mask, pb.lam, tau, sigma, pb.n_iter)
    for c in cands:
        got = gpu_solve(pb.field, pb.mask, pb.lam, tau, sigma, pb.n_iter, cluster_size=c["cluster_size"],
                        kernel=c["kernel"], threads=c["threads"], tile=c["tile"])
        assert np.all(np.isfinite(got)), c
        for s in range(2):
            assert rel_l2(got[s], ref[s]) <= TOL, (c, s)
