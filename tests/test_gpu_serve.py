"""Serving loop: continuous batching of slice-streamed volume requests.

Requests of different slice sizes are opened and their slices pushed in
chunks while other requests run; each result must equal (bitwise) the same
volume served alone, and the plain solve with the server's kernel variant and
step size, and a sampled slice of every served request must match the FP64
oracle after the same iterations at the server's step size (rel-L2 1e-4).
Admission respects the memory budget.
"""

import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2006_09808_gb300 as pcs  # noqa: E402
import phantoms  # noqa: E402
from oracle import pd_oracle as O  # noqa: E402

pytestmark = pytest.mark.gpu
N_ITER = 80
TOL = 1e-4  # relative L2 on chi against the FP64 oracle


def check_against_oracle(served, pb, L, k):
    """The middle slice of a served request against the oracle at the server's tau = sigma = 1/L."""
    s = pb.field.shape[0] // 2
    ref = O.pd_solve(pb.field[s].astype(np.float64), pb.mask[s], pb.lam, 1 / L, 1 / L, N_ITER)
    got = served[s].astype(np.float64)
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel <= TOL, (k, rel)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_09808_gb300 import build

    build.build()
    pcs.load_library()


def pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()


def _wait_all(sv, ids, timeout=120.0, expect_ok=True):
    done, status, t0 = {}, {}, time.time()
    while len(done) < len(ids):
        for rid, lat, st in pcs.pcs_serve_poll(sv):
            done[rid] = lat
            status[rid] = st
        assert time.time() - t0 < timeout, "requests did not complete"
        time.sleep(0.002)
    if expect_ok:
        assert all(v == pcs.PCS_OK for v in status.values()), status
        return done
    return done, status


def _serve(sv, probs, chunks=3, gap_s=0.003):
    outs, keep, ids = [], [], []
    for pb in probs:
        S, H, W = pb.field.shape
        f, m = pinned(pb.field), pinned(pb.mask)
        chi = pinned(np.full(pb.field.shape, np.nan, np.float32))
        rid = pcs.pcs_serve_open(sv, H, W, S, pb.lam, chi)
        keep += [f, m]
        outs.append(chi)
        ids.append((rid, f, m, S))
    # push the slices of all requests interleaved, in chunks, as a scanner would
    pos = [0] * len(ids)
    while any(p < S for p, (_, _, _, S) in zip(pos, ids)):
        for k, (rid, f, m, S) in enumerate(ids):
            if pos[k] < S:
                n = max(1, -(-S // chunks))
                n = min(n, S - pos[k])
                pcs.pcs_serve_push(sv, rid, pos[k], f[pos[k]:pos[k] + n], m[pos[k]:pos[k] + n])
                pos[k] += n
                time.sleep(gap_s)
    lat = _wait_all(sv, [r for r, *_ in ids])
    return outs, lat


PROBS = [
    (128, 4, 1, 2e-4), (256, 3, 2, 5e-4), (192, 5, 3, 1e-3), (128, 3, 4, 5e-4), (384, 2, 5, 2e-4), (256, 4, 6, 1e-3),
]


def _probs():
    return [phantoms.volume(H, H, S, seed=sd, lam=lam, n_iter=N_ITER) for H, S, sd, lam in PROBS]


def test_mix_equals_alone_and_plain():
    probs = _probs()
    sv = pcs.pcs_serve_start(hbm_budget_bytes=8 << 30, slots=4, n_iter=N_ITER, autotune=True)
    try:
        tun = {H: pcs.pcs_serve_prepare_size(sv, H, H) for H, *_ in PROBS}
        mix, lat = _serve(sv, probs)
        st = pcs.pcs_serve_stats(sv)
        assert st["completed"] == len(probs) and st["peak_inflight"] >= 2  # work overlapped
        assert all(v > 0 for v in lat.values())
        for k, pb in enumerate(probs):
            alone, _ = _serve(sv, [pb], chunks=1)
            assert np.array_equal(mix[k], alone[0]), k
    finally:
        pcs.pcs_serve_stop(sv)
    for k, pb in enumerate(probs):
        check_against_oracle(mix[k], pb, tun[pb.field.shape[1]]["L"], k)
    for k, pb in enumerate(probs):
        S, H, W = pb.field.shape
        t = tun[H]
        f = torch.from_numpy(pb.field).cuda()
        m = torch.from_numpy(pb.mask).cuda()
        chi = torch.empty_like(f)
        ctx = pcs.pcs_create(H, W, S, cluster_size=t["cluster_size"], kernel=t["kernel"], threads=t["threads"],
                             tile=t["tile"])
        try:
            pcs.pcs_solve_slices(ctx, f, m, pb.lam, 1 / t["L"], 1 / t["L"], N_ITER, chi)
            torch.cuda.synchronize()
        finally:
            pcs.pcs_destroy(ctx)
        assert np.array_equal(mix[k], chi.cpu().numpy()), k


def test_budget_limits_admission():
    probs = _probs()[:3]
    need = [pcs.pcs_serve_request_bytes(pb.field.shape[1], pb.field.shape[2], pb.field.shape[0]) for pb in probs]
    assert all(n >= 25 * pb.voxels for n, pb in zip(need, probs))  # field, mask, chi, four state arrays
    # room for the biggest request alone, never for two of them
    budget = max(need) + 1024
    assert budget < min(a + b for k, a in enumerate(need) for b in need[k + 1:])
    sv = pcs.pcs_serve_start(hbm_budget_bytes=budget, slots=4, n_iter=20, autotune=False)
    try:
        outs, _ = _serve(sv, probs)
        st = pcs.pcs_serve_stats(sv)
        assert st["peak_inflight"] == 1 and st["peak_bytes"] <= budget
        assert all(np.all(np.isfinite(o)) for o in outs)
    finally:
        pcs.pcs_serve_stop(sv)


def test_serving_allocates_no_device_memory_while_it_runs():
    """The budget is one arena allocated at start: serving requests of every size leaves the free
    device memory unchanged (the scheduler thread never allocates)."""
    probs = _probs()
    sv = pcs.pcs_serve_start(hbm_budget_bytes=2 << 30, slots=3, n_iter=20, autotune=False)
    try:
        for H, *_ in PROBS:
            pcs.pcs_serve_prepare_size(sv, H, H)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        outs, _ = _serve(sv, probs)
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0
        assert all(np.all(np.isfinite(o)) for o in outs)
    finally:
        pcs.pcs_serve_stop(sv)


def test_failed_request_is_isolated():
    """A launch failure injected on the host into one request finishes that request alone with an
    error status; the requests around it complete with their correct chi, and the server keeps
    serving."""
    probs = [phantoms.volume(128, 128, 4, seed=21 + k, lam=5e-4, n_iter=N_ITER) for k in range(3)]
    sv = pcs.pcs_serve_start(hbm_budget_bytes=1 << 30, slots=3, n_iter=N_ITER, autotune=False)
    try:
        L = pcs.pcs_serve_prepare_size(sv, 128, 128)["L"]
        outs, keep, ids = [], [], []
        for k, pb in enumerate(probs):
            f, m = pinned(pb.field), pinned(pb.mask)
            chi = pinned(np.full(pb.field.shape, np.nan, np.float32))
            rid = pcs.pcs_serve_open(sv, 128, 128, 4, pb.lam, chi)
            if k == 1:
                pcs.pcs_serve_fail_next_launch(sv, rid)
            keep += [f, m]
            outs.append(chi)
            ids.append(rid)
            pcs.pcs_serve_push(sv, rid, 0, f, m)
        _, status = _wait_all(sv, ids, expect_ok=False)
        assert status[ids[1]] == pcs.PCS_ECUDA
        assert status[ids[0]] == pcs.PCS_OK and status[ids[2]] == pcs.PCS_OK
        st = pcs.pcs_serve_stats(sv)
        assert st["failed"] == 1 and st["completed"] == 2
        again, _ = _serve(sv, [probs[1]])  # the server goes on after the failure
        for k, got in ((0, outs[0]), (2, outs[2]), (1, again[0])):
            check_against_oracle(got, probs[k], L, k)
    finally:
        pcs.pcs_serve_stop(sv)


def test_rejections():
    sv = pcs.pcs_serve_start(hbm_budget_bytes=1 << 20, slots=1, n_iter=5, autotune=False)
    try:
        chi = np.zeros((4, 256, 256), np.float32)
        with pytest.raises(pcs.PcsError) as ei:  # 4 x 256 x 256 x 25 B > 1 MiB
            pcs.pcs_serve_open(sv, 256, 256, 4, 1e-3, chi)
        assert ei.value.status == pcs.PCS_ENOMEM
        with pytest.raises(pcs.PcsError) as ei:  # no compiled kernel; 134 = 2 x 67 outside the any-size rule
            pcs.pcs_serve_open(sv, 100, 134, 1, 1e-3, np.zeros((1, 100, 134), np.float32))
        assert ei.value.status == pcs.PCS_EUNSUPPORTED
    finally:
        pcs.pcs_serve_stop(sv)


def test_native_sizes_served_with_the_rest():
    """Requests of the paper's 128 x 132 and 256 x 258 slices (the any-size kernels, each slot with
    its own spectrum) served among a compiled 128 x 128 request: mix == alone, and equal to the
    plain solves with the server's step size, bit for bit."""
    specs = [(128, 132, 4, 11, 5e-4), (256, 258, 3, 12, 1e-3), (128, 128, 3, 13, 5e-4)]
    probs = [phantoms.volume(H, W, S, seed=sd, lam=lam, n_iter=N_ITER) for H, W, S, sd, lam in specs]
    sv = pcs.pcs_serve_start(hbm_budget_bytes=8 << 30, slots=3, n_iter=N_ITER, autotune=False)
    try:
        tun = {(H, W): pcs.pcs_serve_prepare_size(sv, H, W) for H, W, *_ in specs}
        mix, _ = _serve(sv, probs)
        for k, pb in enumerate(probs):
            alone, _ = _serve(sv, [pb], chunks=1)
            assert np.array_equal(mix[k], alone[0]), k
    finally:
        pcs.pcs_serve_stop(sv)
    for k, pb in enumerate(probs):
        S, H, W = pb.field.shape
        check_against_oracle(mix[k], pb, tun[(H, W)]["L"], k)
    for k, pb in enumerate(probs[:2]):
        S, H, W = pb.field.shape
        L = tun[(H, W)]["L"]
        f = torch.from_numpy(pb.field).cuda()
        m = torch.from_numpy(pb.mask).cuda()
        chi = torch.empty_like(f)
        pcs.pcs_solve_slices_generic(f, m, pb.lam, 1 / L, 1 / L, N_ITER, chi)
        torch.cuda.synchronize()
        assert np.array_equal(mix[k], chi.cpu().numpy()), k
