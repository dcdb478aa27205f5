"""Precision modes on the one-slice 64 x 64 phantom (config-1 inputs).

FP32 state and transforms (the production path, FP64 reductions in its
diagnostics) against the all-FP64 instantiation of the same kernel, both
against the FP64 CPU oracle after 100, 300 and 500 iterations: relative L2
error of chi and of the field residual W(D chi - dB).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2006_09808_gb300 as pcs  # noqa: E402
import phantoms  # noqa: E402
from oracle import pd_oracle as O  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_09808_gb300 import build

    build.build()
    pcs.load_library()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def precision_table(pb, L, iters=(100, 300, 500), lam=None):
    lam = pb.lam if lam is None else lam
    f64 = pb.field.astype(np.float64)
    Dk = O.dipole_kernel(*pb.field.shape[1:])
    m = pb.mask.astype(np.float64)
    rows = []
    for n in iters:
        ref = O.pd_solve(f64, pb.mask, lam, 1 / L, 1 / L, n)
        res_ref = m * (O.apply_D(ref, Dk) - f64)
        ft = torch.from_numpy(pb.field).cuda()
        mt = torch.from_numpy(pb.mask).cuda()
        c32 = torch.empty_like(ft)
        ctx = pcs.pcs_create(64, 64, 1)
        try:
            pcs.pcs_solve_slices(ctx, ft, mt, lam, 1 / L, 1 / L, n, c32)
        finally:
            torch.cuda.synchronize()
            pcs.pcs_destroy(ctx)
        c64 = torch.empty(pb.field.shape, dtype=torch.float64, device="cuda")
        pcs.pcs_solve_slices_f64(torch.from_numpy(f64).cuda(), mt, lam, 1 / L, 1 / L, n, c64)
        g32 = c32.cpu().numpy().astype(np.float64)
        g64 = c64.cpu().numpy()
        rows.append({
            "iters": n,
            "chi_rel_fp32": rel(g32, ref),
            "chi_rel_fp64": rel(g64, ref),
            "residual_rel_fp32": rel(m * (O.apply_D(g32, Dk) - f64), res_ref),
            "residual_rel_fp64": rel(m * (O.apply_D(g64, Dk) - f64), res_ref),
        })
    return rows


@pytest.mark.parametrize("lam", [None, 10.0])
def test_precision_modes_config1(lam):
    pb = phantoms.config1()
    L = 2.832522691076350  # full-mask ||K|| for 64 x 64 (tests/golden/opnorm_full_mask.txt)
    rows = precision_table(pb, L, lam=lam)
    for r in rows:
        print(r)
        assert r["chi_rel_fp64"] < 1e-11
        assert r["residual_rel_fp64"] < 1e-10
        assert r["chi_rel_fp32"] < 1e-4
        assert r["chi_rel_fp64"] < 1e-3 * r["chi_rel_fp32"]


def test_fp64_kernel_256_and_unsupported_size():
    pb = phantoms.volume(256, 256, 2, seed=3, lam=1e-3, n_iter=30)
    L = 2.833285229534487
    ref = O.pd_solve(pb.field.astype(np.float64), pb.mask, pb.lam, 1 / L, 1 / L, pb.n_iter)
    c64 = torch.empty(pb.field.shape, dtype=torch.float64, device="cuda")
    pcs.pcs_solve_slices_f64(torch.from_numpy(pb.field.astype(np.float64)).cuda(), torch.from_numpy(pb.mask).cuda(),
                             pb.lam, 1 / L, 1 / L, pb.n_iter, c64)
    assert rel(c64.cpu().numpy(), ref) < 1e-11
    bad = torch.zeros((1, 128, 128), dtype=torch.float64, device="cuda")
    with pytest.raises(pcs.PcsError) as ei:
        pcs.pcs_solve_slices_f64(bad, torch.ones((1, 128, 128), dtype=torch.uint8, device="cuda"), 1.0, 0.3, 0.3, 5,
                                 torch.empty_like(bad))
    assert ei.value.status == pcs.PCS_EUNSUPPORTED
