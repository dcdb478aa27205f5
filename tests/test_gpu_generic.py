"""Any-size per-slice solver (pcs_solve_slices_generic) against the FP64 oracle.

Sizes include the paper's own slices, 256 x 258 and 128 x 132 (FFT lengths with the
prime factors 43 and 11), rectangles, and the smallest accepted size; H in {64·2^k, 3·2^k}
takes the register-FFT column kernel, other H the shared-memory DFT column kernel.  tau = sigma =
1/sqrt(4/9 + 8), a valid step for every 0/1 mask (||D|| <= 2/3, ||G||^2 <= 8).
"""

import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2006_09808_gb300 as pcs  # noqa: E402
import phantoms  # noqa: E402
from oracle import pd_oracle as O  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-4
STEP = 1.0 / math.sqrt(4.0 / 9.0 + 8.0)


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


def gpu_generic(field, mask, lam, n_iter, tv=0, weight=None, b0_axis=0):
    f = torch.from_numpy(np.array(field, dtype=np.float32)).cuda()
    m = torch.from_numpy(np.array(mask, dtype=np.uint8)).cuda()
    w = None if weight is None else torch.from_numpy(np.array(weight, dtype=np.float32)).cuda()
    chi = torch.full_like(f, float("nan"))
    pcs.pcs_solve_slices_generic(f, m, lam, STEP, STEP, n_iter, chi, tv=tv, weight=w, b0_axis=b0_axis)
    torch.cuda.synchronize()
    return chi.cpu().numpy()


def oracle(field, mask, lam, n_iter, tv=0, weight=None, b0_axis=0):
    return O.pd_solve(np.asarray(field, np.float64), mask, lam, STEP, STEP, n_iter, b0_axis=b0_axis,
                      weight=None if weight is None else np.asarray(weight, np.float64),
                      tv="iso" if tv else "aniso")


@pytest.mark.parametrize(
    "S,H,W,n_iter,lam,tv,b0",
    [
        (4, 256, 258, 60, 1.0, 0, 0),   # the stent slices' shape
        (6, 128, 132, 100, 1.0, 0, 0),  # the seed / needle slices' shape
        (3, 128, 132, 100, 1.0, 1, 0),
        (3, 128, 132, 80, 5e-4, 0, 1),
        (2, 90, 98, 80, 1.0, 0, 0),     # 2·3²·5 x 2·7²
        (5, 30, 42, 150, 1.0, 1, 1),
        (2, 64, 64, 80, 1.0, 0, 0),     # power of two: the same problem as the compiled variants
        (2, 192, 198, 60, 1.0, 0, 0),   # register-FFT column pass at H = 3·2^6; 198 = 2·3²·11
        (1, 512, 46, 60, 1.0, 1, 0),    # H = 512, W = 2·23
        (1, 384, 130, 40, 1.0, 0, 1),   # H = 3·2^7, W = 2·5·13
    ],
)
def test_parity_generic(S, H, W, n_iter, lam, tv, b0):
    pb = phantoms.volume(H, W, S, seed=61 + H + W, lam=lam, n_iter=n_iter)
    ref = oracle(pb.field, pb.mask, lam, n_iter, tv=tv, b0_axis=b0)
    got = gpu_generic(pb.field, pb.mask, lam, n_iter, tv=tv, b0_axis=b0)
    assert np.all(np.isfinite(got))
    assert rel_l2(got, ref) <= TOL
    for s in range(S):
        assert rel_l2(got[s], ref[s]) <= 10 * TOL, s
    m = pb.mask.astype(bool)
    assert rel_l2(got[m], ref[m]) <= TOL


def test_generic_weighted_and_batch_independence():
    pb = phantoms.volume(128, 132, 4, seed=71, lam=1.0, n_iter=60)
    w = phantoms.magnitude_weight(pb.mask, seed=72)
    ref = oracle(pb.field, pb.mask, 1.0, 60, weight=w)
    got = gpu_generic(pb.field, pb.mask, 1.0, 60, weight=w)
    assert rel_l2(got, ref) <= TOL
    # a slice alone equals the same slice inside the batch, bit for bit
    alone = gpu_generic(pb.field[2:3], pb.mask[2:3], 1.0, 60, weight=w[2:3])
    assert np.array_equal(alone[0], got[2])


def test_generic_stent_shape_at_the_bench_iteration_count():
    """256 x 258 x 25 solved in the bench's launch (all slices, 500 iterations, lambda 5e-4);
    three sampled slices against the oracle after the same 500 iterations, each within 1e-4."""
    n_iter = 500
    pb = phantoms.volume(256, 258, 25, seed=0, lam=5e-4, n_iter=n_iter, name="bench258")
    got = gpu_generic(pb.field, pb.mask, pb.lam, n_iter)
    assert np.all(np.isfinite(got))
    for s in (0, 12, 24):
        ref = oracle(pb.field[s], pb.mask[s], pb.lam, n_iter)
        assert rel_l2(got[s], ref) <= TOL, s
        m = pb.mask[s].astype(bool)
        assert rel_l2(got[s][m], ref[m]) <= TOL, s


def test_generic_full_stent_shape():
    """256 x 258 x 25, the stent acquisition's shape, 20 iterations against the oracle."""
    pb = phantoms.volume(256, 258, 25, seed=73, lam=5e-4, n_iter=20)
    ref = oracle(pb.field, pb.mask, pb.lam, 20)
    got = gpu_generic(pb.field, pb.mask, pb.lam, 20)
    assert rel_l2(got, ref) <= TOL


def test_generic_matches_compiled_variant_at_64():
    """At 64 x 64 both solvers take the same problem: results agree to rounding."""
    pb = phantoms.volume(64, 64, 3, seed=74, lam=1.0, n_iter=50)
    got = gpu_generic(pb.field, pb.mask, 1.0, 50)
    f = torch.from_numpy(pb.field.astype(np.float32)).cuda()
    m = torch.from_numpy(pb.mask.astype(np.uint8)).cuda()
    chi = torch.empty_like(f)
    ctx = pcs.pcs_create(64, 64, 3)
    try:
        pcs.pcs_solve_slices(ctx, f, m, 1.0, STEP, STEP, 50, chi)
        torch.cuda.synchronize()
    finally:
        pcs.pcs_destroy(ctx)
    assert rel_l2(got, chi.cpu().numpy()) <= 1e-5


def test_generic_edge_cases_and_errors():
    rng = np.random.default_rng(3)
    f = rng.standard_normal((2, 8, 12)).astype(np.float32)
    ones = np.ones_like(f, dtype=np.uint8)
    assert np.all(gpu_generic(f, ones, 1.0, 0) == 0)                   # n_iter = 0
    assert np.all(gpu_generic(f, np.zeros_like(ones), 1.0, 30) == 0)   # empty mask
    one = gpu_generic(f, ones, 1.0, 1)                                  # smallest size, one iteration
    assert rel_l2(one, oracle(f, ones, 1.0, 1)) <= 1e-6
    assert rel_l2(gpu_generic(f, ones, 1.0, 200), oracle(f, ones, 1.0, 200)) <= TOL
    assert pcs.pcs_supported_generic(256, 258) and pcs.pcs_supported_generic(128, 132)
    e0 = torch.zeros((0, 8, 12), device="cuda")
    pcs.pcs_solve_slices_generic(e0, torch.zeros((0, 8, 12), dtype=torch.uint8, device="cuda"), 1.0, STEP, STEP,
                                 5, torch.empty_like(e0))  # S = 0: no-op
    for shape, status in (((2, 8, 134), pcs.PCS_EUNSUPPORTED), ((2, 9, 12), pcs.PCS_EUNSUPPORTED),
                          ((1, 8, 514), pcs.PCS_EUNSUPPORTED)):
        g = torch.zeros(shape, device="cuda")
        with pytest.raises(pcs.PcsError) as ei:
            pcs.pcs_solve_slices_generic(g, torch.ones(shape, dtype=torch.uint8, device="cuda"), 1.0, STEP, STEP,
                                         5, torch.empty_like(g))
        assert ei.value.status == status, shape
    g = torch.zeros((1, 8, 12), device="cuda")
    mk = torch.ones((1, 8, 12), dtype=torch.uint8, device="cuda")
    for kw in (dict(lam=-1.0), dict(tv=2), dict(b0_axis=2)):
        args = dict(lam=1.0, tv=0, b0_axis=0)
        args.update(kw)
        with pytest.raises(pcs.PcsError) as ei:
            pcs.pcs_solve_slices_generic(g, mk, args["lam"], STEP, STEP, 5, torch.empty_like(g), tv=args["tv"],
                                         b0_axis=args["b0_axis"])
        assert ei.value.status == pcs.PCS_EINVAL


def test_any_size_context():
    """pcs_create for a size without a compiled kernel makes an any-size context: the same
    results and reports as pcs_solve_slices_generic, bit for bit, with the context's scratch
    and stream; repeated solves reuse it."""
    pb = phantoms.volume(128, 132, 5, seed=75, lam=1.0, n_iter=40)
    direct = gpu_generic(pb.field, pb.mask, 1.0, 40, tv=1)
    f = torch.from_numpy(np.array(pb.field, dtype=np.float32)).cuda()
    m = torch.from_numpy(np.array(pb.mask, dtype=np.uint8)).cuda()
    stream = torch.cuda.Stream()
    assert not pcs.pcs_supported_size(128, 132)
    ctx = pcs.pcs_create(128, 132, 8, tv=1, stream=stream)
    try:
        for S in (5, 3):  # fewer slices than the capacity, then again on the same scratch
            chi = torch.full_like(f[:S], float("nan"))
            with torch.cuda.stream(stream):
                pcs.pcs_solve_slices(ctx, f[:S].contiguous(), m[:S].contiguous(), 1.0, STEP, STEP, 40, chi)
            stream.synchronize()
            assert np.array_equal(chi.cpu().numpy(), direct[:S])
        w = torch.from_numpy(np.array(phantoms.magnitude_weight(pb.mask, seed=76), dtype=np.float32)).cuda()
        chi = torch.empty_like(f)
        torch.cuda.synchronize()  # inputs made on the current stream; the context runs on its own
        pcs.pcs_solve_slices_weighted(ctx, f, m, w, 1.0, STEP, STEP, 40, chi)
        stream.synchronize()
        assert rel_l2(chi.cpu().numpy(), oracle(pb.field, pb.mask, 1.0, 40, tv=1, weight=w.cpu().numpy())) <= TOL
        # the context's FP64 report equals the standalone call's
        rep = pcs.pcs_solve_slices(ctx, f, m, 1.0, STEP, STEP, 40, chi, report=True)
        chi2 = torch.empty_like(f)
        ref = pcs.pcs_solve_slices_generic(f, m, 1.0, STEP, STEP, 40, chi2, tv=1, report=True)
        assert rep == ref
        pcs.pcs_check(ctx)
    finally:
        pcs.pcs_destroy(ctx)
    with pytest.raises(pcs.PcsError) as ei:  # a compiled-kernel option cannot apply
        pcs.pcs_create(128, 132, 8, cluster_size=2)
    assert ei.value.status == pcs.PCS_EUNSUPPORTED


def test_any_size_solve_captured_in_a_cuda_graph():
    """The any-size iteration loop (every launch after the first a programmatic dependent
    launch) captured by the caller in a CUDA graph: each replay equals the direct solve bit for
    bit, and the oracle within the tolerance."""
    pb = phantoms.volume(128, 132, 3, seed=81, lam=5e-4, n_iter=30)
    f = torch.from_numpy(np.array(pb.field, dtype=np.float32)).cuda()
    m = torch.from_numpy(np.array(pb.mask, dtype=np.uint8)).cuda()
    stream = torch.cuda.Stream()
    ctx = pcs.pcs_create(128, 132, 3, stream=stream)
    try:
        torch.cuda.synchronize()
        direct = torch.empty_like(f)
        with torch.cuda.stream(stream):
            pcs.pcs_solve_slices(ctx, f, m, pb.lam, STEP, STEP, pb.n_iter, direct)
        stream.synchronize()
        captured = torch.full_like(f, float("nan"))
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            pcs.pcs_solve_slices(ctx, f, m, pb.lam, STEP, STEP, pb.n_iter, captured)
        for _ in range(2):
            captured.fill_(float("nan"))
            torch.cuda.synchronize()
            graph.replay()
            torch.cuda.synchronize()
            assert torch.equal(captured, direct)
        pcs.pcs_check(ctx)
    finally:
        pcs.pcs_destroy(ctx)
    assert rel_l2(direct.cpu().numpy(), oracle(pb.field, pb.mask, pb.lam, pb.n_iter)) <= TOL


@pytest.mark.parametrize("H,W,tv,weighted,b0", [(128, 132, 0, False, 0), (256, 258, 1, False, 0),
                                                (90, 98, 0, True, 1)])
def test_generic_report_against_oracle(H, W, tv, weighted, b0):
    """Per-slice FP64 report at (chi_N, p_N, q_N) against the oracle's diagnostics on its own state
    after the same iterations (gap and stationarity are differences of nearly equal terms: a
    relative bound plus a floor from the terms' size)."""
    S, n_iter, lam = 3, 120, 1.0
    pb = phantoms.volume(H, W, S, seed=81 + H, lam=lam, n_iter=n_iter)
    w = phantoms.magnitude_weight(pb.mask, seed=82) if weighted else None
    f = torch.from_numpy(np.array(pb.field, dtype=np.float32)).cuda()
    m = torch.from_numpy(np.array(pb.mask, dtype=np.uint8)).cuda()
    wt = None if w is None else torch.from_numpy(np.array(w, dtype=np.float32)).cuda()
    chi = torch.empty_like(f)
    rep = pcs.pcs_solve_slices_generic(f, m, lam, STEP, STEP, n_iter, chi, tv=tv, weight=wt, b0_axis=b0,
                                       report=True)
    torch.cuda.synchronize()
    tvs = "iso" if tv else "aniso"
    wd = None if w is None else w.astype(np.float64)
    for s in range(S):
        st = O.pd_solve(pb.field[s].astype(np.float64), pb.mask[s], lam, STEP, STEP, n_iter, b0_axis=b0,
                        weight=None if wd is None else wd[s], tv=tvs, return_state=True)
        ref = O.diagnostics(st, pb.field[s], pb.mask[s], lam, b0_axis=b0, weight=None if wd is None else wd[s],
                            tv=tvs)
        r = rep[s]
        assert r["iters"] == n_iter
        assert r["objective"] == pytest.approx(ref.primal, rel=1e-4)
        assert r["data_residual"] == pytest.approx(ref.data_residual, rel=1e-4)
        assert abs(r["gap"] - ref.gap) <= 2e-2 * ref.gap + 1e-4 * ref.primal
        assert abs(r["stationarity"] - ref.stationarity) <= 2e-2 * ref.stationarity + 1e-3


def test_generic_report_zero_start_closed_form():
    """N = 0: chi = p = q = 0, so objective = lambda/2 ||W dB||^2, gap = lambda ||W dB||^2 / 2,
    stationarity 0 and residual ||W dB|| (per slice; no oracle)."""
    pb = phantoms.volume(128, 132, 2, seed=83, lam=1.0, n_iter=1)
    lam = 0.25
    f = torch.from_numpy(np.array(pb.field, dtype=np.float32)).cuda()
    m = torch.from_numpy(np.array(pb.mask, dtype=np.uint8)).cuda()
    rep = pcs.pcs_solve_slices_generic(f, m, lam, STEP, STEP, 0, torch.empty_like(f), report=True)
    for s in range(2):
        b2 = float(np.sum((pb.mask[s].astype(np.float64) * pb.field[s].astype(np.float32).astype(np.float64)) ** 2))
        assert rep[s]["objective"] == pytest.approx(0.5 * lam * b2, rel=1e-12)
        assert rep[s]["gap"] == pytest.approx(lam * b2 / 2.0, rel=1e-12)
        assert rep[s]["data_residual"] == pytest.approx(math.sqrt(b2), rel=1e-12)
        assert rep[s]["stationarity"] == 0.0


@pytest.mark.parametrize("H,W,kind", [(128, 132, "full"), (256, 258, "ellipse"), (90, 98, "full")])
def test_generic_opnorm_matches_oracle(H, W, kind):
    """L = ||K|| by the any-size power iteration against the oracle's converged power iteration
    (a Rayleigh quotient never exceeds the top eigenvalue; 400 steps get within 0.2%)."""
    mask = np.ones((H, W), np.uint8) if kind == "full" else phantoms.ellipse_mask(H, W)
    ref = O.opnorm(mask)
    ctx = pcs.pcs_create(H, W, 2)
    try:
        got = pcs.pcs_opnorm(ctx, torch.from_numpy(np.stack([mask, mask])).cuda(), 400)
    finally:
        pcs.pcs_destroy(ctx)
    for g in got:  # each slice starts from its own pseudo-random vector
        assert ref * (1 - 2e-3) <= g <= ref * (1 + 1e-5)
        assert g <= math.sqrt(4.0 / 9.0 + 8.0)


def test_solver_on_a_native_size():
    """The convenience Solver on 128 x 132 slices: steps 1/L from the device power iteration,
    the same result as the standalone call with those steps."""
    pb = phantoms.volume(128, 132, 2, seed=84, lam=1.0, n_iter=30)
    f = torch.from_numpy(np.array(pb.field, dtype=np.float32)).cuda()
    m = torch.from_numpy(np.array(pb.mask, dtype=np.uint8)).cuda()
    with pcs.Solver(128, 132, 2) as s:
        L, tau, sigma = s.step_sizes()
        assert L == pytest.approx(O.opnorm(np.ones((128, 132))), rel=2e-3) and tau == sigma
        chi = s.solve(f, m, 1.0, 30)
        torch.cuda.synchronize()
    chi2 = torch.empty_like(f)
    pcs.pcs_solve_slices_generic(f, m, 1.0, tau, sigma, 30, chi2)
    torch.cuda.synchronize()
    assert np.array_equal(chi.cpu().numpy(), chi2.cpu().numpy())


def test_generic_monitored_resume_and_early_stop():
    """Monitored solves on an any-size context: chunks of 25 iterations resume exactly (equal bit
    for bit to one straight solve, reports included), and a slice whose gap is already zero (zero
    field) freezes at the first check while the others run on."""
    pb = phantoms.volume(128, 132, 3, seed=85, lam=1.0, n_iter=75)
    field = np.array(pb.field, dtype=np.float32)
    field[1] = 0.0  # chi stays 0: gap 0 at every check
    f = torch.from_numpy(field).cuda()
    m = torch.from_numpy(np.array(pb.mask, dtype=np.uint8)).cuda()
    ctx = pcs.pcs_create(128, 132, 3)
    try:
        straight = torch.empty_like(f)
        rep_s = pcs.pcs_solve_slices(ctx, f, m, 1.0, STEP, STEP, 75, straight, report=True)
        chunked = torch.full_like(f, float("nan"))
        rep_c = pcs.pcs_solve_slices_monitored(ctx, f, m, 1.0, STEP, STEP, 75, 25, 0.0, chunked)
        torch.cuda.synchronize()
        assert np.array_equal(chunked.cpu().numpy(), straight.cpu().numpy())
        for a, b in zip(rep_c, rep_s):
            assert a == b
        stop = torch.full_like(f, float("nan"))
        rep_e = pcs.pcs_solve_slices_monitored(ctx, f, m, 1.0, STEP, STEP, 75, 25, 1e-12, stop)
        torch.cuda.synchronize()
    finally:
        pcs.pcs_destroy(ctx)
    assert rep_e[1]["iters"] == 25 and rep_e[1]["gap"] == 0.0
    assert rep_e[0]["iters"] == 75 and rep_e[2]["iters"] == 75
    got = stop.cpu().numpy()
    assert np.all(got[1] == 0.0)
    assert np.array_equal(got[0], straight.cpu().numpy()[0]) and np.array_equal(got[2], straight.cpu().numpy()[2])


def test_generic_sizes_in_an_uneven_batch():
    """An uneven batch mixing the paper's 256 x 258 and 128 x 132 slices (two lambdas in one size
    class) with a compiled 128 x 128 volume: every slice against the oracle with the class's
    tau = sigma = 1/L; a volume alone equal bit for bit to the same volume inside the mix."""
    specs = [(128, 132, 3, 1.0, 91), (256, 258, 2, 0.5, 92), (128, 128, 2, 1.0, 93), (128, 132, 2, 0.25, 94)]
    probs = [phantoms.volume(H, W, S, seed=sd, lam=lam, n_iter=60) for H, W, S, lam, sd in specs]

    def run(pbs):
        batch = pcs.pcs_batch_create(autotune=False)
        vols, outs = [], []
        for pb in pbs:
            f = torch.from_numpy(np.array(pb.field, dtype=np.float32)).cuda()
            m = torch.from_numpy(np.array(pb.mask, dtype=np.uint8)).cuda()
            chi = torch.full_like(f, float("nan"))
            vols.append((f, m, pb.lam, chi))
            outs.append(chi)
        try:
            pcs.pcs_batch_solve(batch, vols, 60)
            torch.cuda.synchronize()
            Ls = {(pb.field.shape[1], pb.field.shape[2]):
                  pcs.pcs_batch_tuning(batch, pb.field.shape[1], pb.field.shape[2])["L"] for pb in pbs}
        finally:
            pcs.pcs_batch_destroy(batch)
        return [o.cpu().numpy() for o in outs], Ls

    got, Ls = run(probs)
    for pb, g in zip(probs, got):
        S, H, W = pb.field.shape
        L = Ls[(H, W)]
        assert 2.5 < L <= math.sqrt(4.0 / 9.0 + 8.0)
        ref = O.pd_solve(pb.field.astype(np.float64), pb.mask, pb.lam, 1.0 / L, 1.0 / L, 60)
        assert rel_l2(g, ref) <= TOL, (H, W, pb.lam)
    alone, _ = run([probs[3]])
    assert np.array_equal(alone[0], got[3])


def test_solvers_of_several_sizes_coexist():
    """A larger any-size solver made before a smaller one (and the shared-memory column kernel's
    H = 90 before H = 30) still launches: the kernels' shared-memory limits do not depend on the
    order in which sizes are set up."""
    big = phantoms.volume(256, 258, 1, seed=95, lam=1.0, n_iter=10)
    small = phantoms.volume(128, 132, 1, seed=96, lam=1.0, n_iter=10)
    odd_big = phantoms.volume(90, 98, 1, seed=97, lam=1.0, n_iter=10)
    odd_small = phantoms.volume(30, 42, 1, seed=98, lam=1.0, n_iter=10)
    ctxs = []
    try:
        for pb in (big, odd_big, small, odd_small):  # larger sizes first
            ctxs.append(pcs.pcs_create(pb.field.shape[1], pb.field.shape[2], 1))
        for ctx, pb in zip(ctxs, (big, odd_big, small, odd_small)):
            f = torch.from_numpy(np.array(pb.field, dtype=np.float32)).cuda()
            m = torch.from_numpy(np.array(pb.mask, dtype=np.uint8)).cuda()
            chi = torch.empty_like(f)
            pcs.pcs_solve_slices(ctx, f, m, 1.0, STEP, STEP, 10, chi)
            torch.cuda.synchronize()
            assert rel_l2(chi.cpu().numpy(), oracle(pb.field, pb.mask, 1.0, 10)) <= TOL
    finally:
        for c in ctxs:
            pcs.pcs_destroy(c)
