"""Uneven batches (volumes of different slice sizes and lambdas in one call).

The batch path packs volumes per slice size, runs one persistent launch per
size (the autotuner's variant), and uses tau = sigma = 1/L with L the
full-mask operator norm it computed on the GPU; the oracle is given that
same L.
"""

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


def _batch_solve(problems, n_iter, autotune=True, batch=None):
    own = batch is None
    if own:
        batch = pcs.pcs_batch_create(autotune=autotune)
    vols, outs = [], []
    for pb in problems:
        f = torch.from_numpy(pb.field).cuda()
        m = torch.from_numpy(pb.mask).cuda()
        chi = torch.full_like(f, float("nan"))
        vols.append((f, m, pb.lam, chi))
        outs.append(chi)
    try:
        pcs.pcs_batch_solve(batch, vols, n_iter)
        pcs.pcs_batch_check(batch)  # synchronises; PCS_ETIMEOUT if a schedule wait gave up
        tunings = {pb.field.shape[1]: pcs.pcs_batch_tuning(batch, pb.field.shape[1], pb.field.shape[2])
                   for pb in problems}
    finally:
        if own:
            pcs.pcs_batch_destroy(batch)
    return [o.cpu().numpy() for o in outs], tunings


def test_batch_matches_per_volume_solves():
    probs = [
        phantoms.volume(128, 128, 3, seed=1, lam=2e-4, n_iter=60),
        phantoms.volume(256, 256, 2, seed=2, lam=1e-3, n_iter=60),
        phantoms.volume(128, 128, 2, seed=3, lam=5e-4, n_iter=60),
        phantoms.volume(192, 192, 2, seed=4, lam=5e-4, n_iter=60),
    ]
    got, tun = _batch_solve(probs, 60)
    for pb, g in zip(probs, got):
        S, H, W = pb.field.shape
        L = tun[H]["L"]
        f = torch.from_numpy(pb.field).cuda()
        m = torch.from_numpy(pb.mask).cuda()
        chi = torch.empty_like(f)
        t = tun[H]
        ctx = pcs.pcs_create(H, W, S, cluster_size=t["cluster_size"], kernel=t["kernel"], threads=t["threads"],
                             tile=t["tile"])
        try:
            pcs.pcs_solve_slices(ctx, f, m, pb.lam, 1.0 / L, 1.0 / L, 60, chi)
            torch.cuda.synchronize()
        finally:
            pcs.pcs_destroy(ctx)
        assert np.array_equal(g, chi.cpu().numpy())


def test_batch_invariance_alone_vs_mix():
    a = phantoms.volume(256, 256, 2, seed=7, lam=5e-4, n_iter=40)
    b = phantoms.volume(384, 384, 2, seed=8, lam=2e-4, n_iter=40)
    c = phantoms.volume(256, 256, 3, seed=9, lam=1e-3, n_iter=40)
    mix, _ = _batch_solve([a, b, c], 40, autotune=False)
    alone, _ = _batch_solve([c], 40, autotune=False)
    assert np.array_equal(mix[2], alone[0])


def test_autotuner_record():
    pb = phantoms.volume(256, 256, 8, seed=5, lam=5e-4, n_iter=10)
    _, tun = _batch_solve([pb], 10, autotune=True)
    t = tun[256]
    assert len(t["candidates"]) >= 2
    times = [c["ns_per_voxel_iter"] for c in t["candidates"]]
    assert all(x > 0 for x in times)
    best = t["candidates"][int(np.argmin(times))]
    assert (t["cluster_size"], t["kernel"], t["threads"]) == (best["cluster_size"], best["kernel"], best["threads"])
    assert 2.7 < t["L"] < 2.91


def test_uneven_batch_recipe_subset_vs_oracle():
    """One volume of each slice size from the uneven-batch recipe (full slice
    counts, its lambda, 400 iterations), solved in one batch call; one sampled
    slice per volume against the FP64 oracle."""
    specs = phantoms.config4_volumes()
    chosen, seen = [], set()
    for sp in specs:
        if sp["size"] not in seen:
            seen.add(sp["size"])
            chosen.append(sp)
    probs = [phantoms.volume(sp["size"], sp["size"], sp["slices"], seed=sp["seed"], lam=sp["lam"],
                             n_iter=sp["n_iter"]) for sp in chosen]
    got, tun = _batch_solve(probs, 400)
    rng = np.random.default_rng(0)
    for pb, g in zip(probs, got):
        S, H, W = pb.field.shape
        assert np.all(np.isfinite(g))
        s = int(rng.integers(0, S))
        L = tun[H]["L"]
        ref = O.pd_solve(pb.field[s].astype(np.float64), pb.mask[s], pb.lam, 1.0 / L, 1.0 / L, 400)
        assert rel_l2(g[s], ref) <= TOL, (H, s)


def test_uneven_batch_full_recipe_vs_oracle():
    """All 48 volumes of the uneven-batch recipe (about 2.7e8 voxels, 400 iterations) in one batch
    call, the bench's launch; one sampled slice of every volume against the FP64 oracle (rel-L2
    1e-4), the oracle solves spread over the host cores."""
    import oracle_workers as OW

    specs = phantoms.config4_volumes()
    with OW.spawn_pool() as ex:
        data = list(ex.map(OW.gen_volume, specs))
        batch = pcs.pcs_batch_create(autotune=True)
        vols, outs = [], []
        for (f, m), sp in zip(data, specs):
            ft = torch.from_numpy(f).cuda()
            mt = torch.from_numpy(m).cuda()
            chi = torch.full_like(ft, float("nan"))
            vols.append((ft, mt, sp["lam"], chi))
            outs.append(chi)
        try:
            pcs.pcs_batch_solve(batch, vols, 400)
            pcs.pcs_batch_check(batch)
            tun = {n: pcs.pcs_batch_tuning(batch, n, n) for n in {sp["size"] for sp in specs}}
        finally:
            pcs.pcs_batch_destroy(batch)
        rng = np.random.default_rng(48)
        picks = [int(rng.integers(0, sp["slices"])) for sp in specs]
        jobs = []
        for (f, m), sp, s in zip(data, specs, picks):
            L = tun[sp["size"]]["L"]
            jobs.append((f[s], m[s], sp["lam"], 1.0 / L, 1.0 / L, 400))
        refs = list(ex.map(OW.oracle_slice, jobs))
    for k, (sp, s, ref) in enumerate(zip(specs, picks, refs)):
        got = outs[k][s].cpu().numpy()
        assert np.all(np.isfinite(got)), k
        assert rel_l2(got, ref) <= TOL, (k, sp["size"], s)
