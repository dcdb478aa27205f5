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
        torch.cuda.synchronize()
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
        ctx = pcs.pcs_create(H, W, S, cluster_size=t["cluster_size"], kernel=t["kernel"], threads=t["threads"])
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
