"""The C ABI without a GPU: the library builds, loads, exports every declared
symbol, and rejects bad arguments with status codes (no compute calls)."""

import ctypes
import os
import shutil
import subprocess

import pytest

import paper_2006_09808_gb300 as pcs

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists(pcs.LIB_PATH),
                                reason="needs nvcc or a built libpcs.so")


@pytest.fixture(scope="module")
def lib():
    from paper_2006_09808_gb300 import build

    build.build()
    return pcs.load_library()


def test_header_declares_the_boundary():
    names = pcs.declared_functions()
    for n in ("pcs_create", "pcs_solve_slices", "pcs_destroy", "pcs_opnorm", "pcs_report",
              "pcs_solve_slices_host", "pcs_last_error"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", pcs.LIB_PATH], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    for name in pcs.declared_functions():
        assert name in exported, name
        assert getattr(lib, name) is not None


def test_only_the_c_abi_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", pcs.LIB_PATH], capture_output=True, text=True).stdout
    ours = {line.split()[-1] for line in out.splitlines() if " T " in line and "pcs" in line}
    assert ours == set(pcs.declared_functions())


def test_host_side_argument_checks(lib):
    opt = pcs.pcs_options()
    assert lib.pcs_options_default(ctypes.byref(opt)) == pcs.PCS_OK
    assert (opt.b0_axis, opt.cluster_size, opt.max_clusters) == (0, 0, 0)
    assert lib.pcs_options_default(None) == pcs.PCS_EINVAL
    assert lib.pcs_supported_size(256, 256) == 1
    assert lib.pcs_supported_size(64, 64) == 1
    assert lib.pcs_supported_size(100, 100) == 0
    h = ctypes.c_void_p()
    assert lib.pcs_create(None, 64, 64, 1, None, None) == pcs.PCS_EINVAL
    assert lib.pcs_create(ctypes.byref(h), 64, 64, 0, None, None) == pcs.PCS_EINVAL
    assert h.value is None
    # 100 x 134: no compiled kernel, and 134 = 2 x 67 is outside the any-size rule (primes <= 61)
    assert lib.pcs_create(ctypes.byref(h), 100, 134, 4, None, None) == pcs.PCS_EUNSUPPORTED
    assert "100 x 134" in pcs.last_error()
    bad = pcs.pcs_options()
    bad.b0_axis = 3
    assert lib.pcs_create(ctypes.byref(h), 64, 64, 4, ctypes.byref(bad), None) == pcs.PCS_EINVAL
    bad = pcs.pcs_options()
    bad.tv = 2
    assert lib.pcs_create(ctypes.byref(h), 64, 64, 4, ctypes.byref(bad), None) == pcs.PCS_EINVAL
    assert "tv" in pcs.last_error()
    assert lib.pcs_solve_slices(None, None, None, 1, 1.0, 1.0, 1.0, 1, None, None) == pcs.PCS_EINVAL
    assert lib.pcs_opnorm(None, None, 1, 10, None) == pcs.PCS_EINVAL
    lib.pcs_destroy(None)  # NULL-safe


def test_generic_size_rule(lib):
    # even H and W in [8, 512] whose prime factors are <= 61 (the paper's 256 x 258, 128 x 132)
    for H, W in ((256, 258), (128, 132), (8, 8), (512, 512), (90, 98), (122, 8)):
        assert lib.pcs_supported_generic(H, W) == 1, (H, W)
    for H, W in ((256, 134), (9, 12), (6, 12), (514, 8), (8, 2 * 67), (0, 8)):
        assert lib.pcs_supported_generic(H, W) == 0, (H, W)
    gs = lib.pcs_solve_slices_generic
    assert gs(None, None, None, 2, 256, 134, 0, 1.0, 0.3, 0.3, 5, 0, None, None, None) == pcs.PCS_EUNSUPPORTED
    assert gs(None, None, None, 2, 256, 258, 0, 1.0, 0.3, 0.3, 5, 0, None, None, None) == pcs.PCS_EINVAL  # NULL
    assert gs(None, None, None, 0, 256, 258, 0, 1.0, 0.3, 0.3, 5, 0, None, None, None) == pcs.PCS_OK  # S = 0
    assert gs(None, None, None, 1, 256, 258, 2, 1.0, 0.3, 0.3, 5, 0, None, None, None) == pcs.PCS_EINVAL  # b0_axis
    assert gs(None, None, None, 1, 256, 258, 0, 0.0, 0.3, 0.3, 5, 0, None, None, None) == pcs.PCS_EINVAL  # lambda


def test_volume_3d_shape_rule(lib):
    """The 3-D variant's shapes (a host query, no GPU): square slices of 64, 128 and 256 with
    32 or 64 slices, and 128 slices for 128^2 and 256^2 -- each either in the pencil form or,
    256x256x128, in the slice form; everything else is refused."""
    accepted = [(32, 64), (64, 64), (32, 128), (64, 128), (128, 128), (32, 256), (64, 256), (128, 256)]
    for S, H in accepted:
        assert lib.pcs_supported_volume_3d(S, H, H) == 1, (S, H)
    for S, H, W in [(128, 64, 64), (16, 64, 64), (48, 128, 128), (64, 256, 128), (64, 512, 512), (64, 192, 192),
                    (0, 64, 64)]:
        assert lib.pcs_supported_volume_3d(S, H, W) == 0, (S, H, W)


def test_create_without_gpu_reports_cuda_error(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = lib.pcs_create(ctypes.byref(h), 64, 64, 1, None, None)
    assert st == pcs.PCS_ECUDA and h.value is None
    assert pcs.last_error() != ""


def test_binding_fails_loudly_without_library(tmp_path):
    import importlib

    mod = importlib.reload(pcs)
    saved = mod._lib
    try:
        mod._lib = None
        with pytest.raises(RuntimeError, match="libpcs.so not found"):
            mod.load_library(str(tmp_path / "missing.so"))
    finally:
        mod._lib = saved


def test_bindings_refuse_host_tensors():
    """No CPU path: the device entry points reject CPU tensors before anything runs."""
    torch = pytest.importorskip("torch")
    f = torch.zeros((2, 128, 132))
    m = torch.ones((2, 128, 132), dtype=torch.uint8)
    chi = torch.empty_like(f)
    calls = [
        lambda: pcs.pcs_solve_slices_generic(f, m, 1.0, 0.3, 0.3, 5, chi),
        lambda: pcs.pcs_solve_volume_3d(torch.zeros((32, 64, 64)), torch.ones((32, 64, 64), dtype=torch.uint8),
                                        1.0, 0.3, 0.3, 5, torch.empty((32, 64, 64))),
        lambda: pcs.pcs_field_map(torch.zeros((4, 8), dtype=torch.complex64), torch.zeros((4, 8), dtype=torch.complex64),
                                  0.6e-3, 3.0, 0.1, torch.empty((4, 8)), torch.empty((4, 8)),
                                  torch.empty((4, 8), dtype=torch.uint8)),
    ]
    for call in calls:
        with pytest.raises(ValueError, match="CUDA device"):
            call()
