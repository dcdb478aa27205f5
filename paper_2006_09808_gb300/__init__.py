"""Python binding of libpcs (GB300 primal-dual positive-contrast susceptibility solver).

Argument marshalling only: every step of the solve runs in the CUDA kernels of
``libpcs.so`` (built from ``csrc/`` by ``build.py``).  The functions keep the
C names of ``include/pcs.h`` and take torch tensors (device memory) or numpy
arrays (host memory); PyTorch is used only for device memory and streams.
There is no CPU fallback: if the library is missing, importing works but the
first call raises.
"""

from __future__ import annotations

import ctypes
import os
import re

PKG = os.path.dirname(os.path.abspath(__file__))
# PCS_LIBRARY overrides the library path (e.g. a build of another configuration)
LIB_PATH = os.environ.get("PCS_LIBRARY") or os.path.join(PKG, "libpcs.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "pcs.h")

PCS_OK, PCS_EINVAL, PCS_EUNSUPPORTED, PCS_ENOMEM, PCS_ECUDA, PCS_ETIMEOUT, PCS_EBUSY = range(7)
STATUS_NAMES = ["PCS_OK", "PCS_EINVAL", "PCS_EUNSUPPORTED", "PCS_ENOMEM", "PCS_ECUDA", "PCS_ETIMEOUT", "PCS_EBUSY"]


class PcsError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{where}: {name}: {message}")


class pcs_options(ctypes.Structure):
    _fields_ = [
        ("b0_axis", ctypes.c_int),
        ("cluster_size", ctypes.c_int),
        ("max_clusters", ctypes.c_int),
        ("kernel", ctypes.c_int),
        ("threads", ctypes.c_int),
        ("use_graph", ctypes.c_int),
        ("tv", ctypes.c_int),
        ("tile", ctypes.c_int),
    ]


class pcs_slice_report(ctypes.Structure):
    _fields_ = [
        ("objective", ctypes.c_double),
        ("gap", ctypes.c_double),
        ("stationarity", ctypes.c_double),
        ("data_residual", ctypes.c_double),
        ("iters", ctypes.c_int),
        ("pad", ctypes.c_int),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k in ("objective", "gap", "stationarity", "data_residual", "iters")}


class pcs_volume(ctypes.Structure):
    _fields_ = [
        ("H", ctypes.c_int),
        ("W", ctypes.c_int),
        ("S", ctypes.c_int),
        ("pad", ctypes.c_int),
        ("lam", ctypes.c_double),
        ("field", ctypes.c_void_p),
        ("mask", ctypes.c_void_p),
        ("chi_out", ctypes.c_void_p),
    ]


class pcs_tuning(ctypes.Structure):
    _fields_ = [
        ("H", ctypes.c_int),
        ("W", ctypes.c_int),
        ("cluster_size", ctypes.c_int),
        ("kernel", ctypes.c_int),
        ("threads", ctypes.c_int),
        ("n_candidates", ctypes.c_int),
        ("L", ctypes.c_double),
        ("ns_per_voxel_iter", ctypes.c_double * 8),
        ("cand_cluster_size", ctypes.c_int * 8),
        ("cand_kernel", ctypes.c_int * 8),
        ("cand_threads", ctypes.c_int * 8),
        ("tile", ctypes.c_int),
        ("cand_tile", ctypes.c_int * 8),
        ("pad", ctypes.c_int),
    ]

    def as_dict(self):
        n = self.n_candidates
        return {
            "H": self.H, "W": self.W, "cluster_size": self.cluster_size, "kernel": self.kernel,
            "threads": self.threads, "tile": self.tile, "L": self.L,
            "candidates": [
                {"cluster_size": self.cand_cluster_size[k], "kernel": self.cand_kernel[k],
                 "threads": self.cand_threads[k], "tile": self.cand_tile[k],
                 "ns_per_voxel_iter": self.ns_per_voxel_iter[k]}
                for k in range(n)
            ],
        }


class pcs_server_config(ctypes.Structure):
    _fields_ = [
        ("hbm_budget_bytes", ctypes.c_size_t),
        ("slots", ctypes.c_int),
        ("n_iter", ctypes.c_int),
        ("autotune", ctypes.c_int),
        ("b0_axis", ctypes.c_int),
        ("reserved", ctypes.c_int * 4),
    ]


class pcs_serve_summary(ctypes.Structure):
    _fields_ = [
        ("completed", ctypes.c_longlong),
        ("pending", ctypes.c_longlong),
        ("voxel_iters", ctypes.c_double),
        ("span_s", ctypes.c_double),
        ("p50_s", ctypes.c_double),
        ("p99_s", ctypes.c_double),
        ("max_s", ctypes.c_double),
        ("peak_bytes", ctypes.c_double),
        ("peak_inflight", ctypes.c_int),
        ("pad", ctypes.c_int),
        ("failed", ctypes.c_longlong),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libpcs.so (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"libpcs.so not found at {path}: build it first "
            "(python -c 'import __graft_entry__ as g; g.build()')"
        )
    lib = ctypes.CDLL(path)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "pcs_options_default": (i, [ctypes.POINTER(pcs_options)]),
        "pcs_supported_size": (i, [i, i]),
        "pcs_create": (i, [ctypes.POINTER(vp), i, i, i, ctypes.POINTER(pcs_options), vp]),
        "pcs_set_stream": (i, [vp, vp]),
        "pcs_solve_slices": (i, [vp, vp, vp, i, d, d, d, i, vp, ctypes.POINTER(pcs_slice_report)]),
        "pcs_solve_slices_host": (i, [vp, vp, vp, i, d, d, d, i, vp, ctypes.POINTER(pcs_slice_report)]),
        "pcs_solve_slices_weighted": (i, [vp, vp, vp, vp, i, d, d, d, i, vp, ctypes.POINTER(pcs_slice_report)]),
        "pcs_solve_volume_3d": (i, [vp, vp, vp, i, i, i, d, d, d, i, i, ctypes.POINTER(d), vp,
                                    ctypes.POINTER(pcs_slice_report), vp]),
        "pcs_supported_volume_3d": (i, [i, i, i]),
        "pcs_solve_slices_generic": (i, [vp, vp, vp, i, i, i, i, d, d, d, i, i, vp, ctypes.POINTER(pcs_slice_report),
                                         vp]),
        "pcs_supported_generic": (i, [i, i]),
        "pcs_field_map": (i, [vp, vp, ctypes.c_size_t, d, d, d, vp, vp, vp, vp]),
        "pcs_check": (i, [vp]),
        "pcs_schedule_plan": (i, [i, i, i, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                  ctypes.POINTER(ctypes.c_int)]),
        "pcs_selftest_wait": (i, [vp, ctypes.c_longlong, ctypes.POINTER(ctypes.c_int)]),
        "pcs_report": (i, [vp, vp, vp, i, d, vp, ctypes.POINTER(pcs_slice_report)]),
        "pcs_solve_slices_monitored": (i, [vp, vp, vp, i, d, d, d, i, i, d, vp, ctypes.POINTER(pcs_slice_report)]),
        "pcs_opnorm": (i, [vp, vp, i, i, ctypes.POINTER(d)]),
        "pcs_solve_slices_noalloc": (i, [vp, vp, i, i, i, d, d, d, i, vp, i, vp]),
        "pcs_destroy": (None, [vp]),
        "pcs_solve_slices_f64": (i, [vp, vp, i, i, i, d, d, d, i, vp, i, vp]),
        "pcs_batch_create": (i, [ctypes.POINTER(vp), ctypes.POINTER(pcs_options), i, vp]),
        "pcs_batch_solve": (i, [vp, ctypes.POINTER(pcs_volume), i, i]),
        "pcs_batch_tuning": (i, [vp, i, i, ctypes.POINTER(pcs_tuning)]),
        "pcs_batch_check": (i, [vp]),
        "pcs_batch_destroy": (None, [vp]),
        "pcs_serve_start": (i, [ctypes.POINTER(vp), ctypes.POINTER(pcs_server_config)]),
        "pcs_serve_prepare_size": (i, [vp, i, i, ctypes.POINTER(pcs_tuning)]),
        "pcs_serve_open": (i, [vp, i, i, i, d, vp, ctypes.POINTER(ctypes.c_longlong)]),
        "pcs_serve_push": (i, [vp, ctypes.c_longlong, i, i, vp, vp]),
        "pcs_serve_poll": (i, [vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(d), ctypes.POINTER(i), i,
                               ctypes.POINTER(i)]),
        "pcs_serve_request_bytes": (i, [i, i, i, ctypes.POINTER(ctypes.c_size_t)]),
        "pcs_serve_arena_plan": (i, [ctypes.c_size_t, ctypes.POINTER(ctypes.c_longlong), i,
                                     ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_size_t)]),
        "pcs_serve_fail_next_launch": (i, [vp, ctypes.c_longlong]),
        "pcs_serve_stats": (i, [vp, ctypes.POINTER(pcs_serve_summary)]),
        "pcs_serve_stop": (None, [vp]),
        "pcs_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def declared_functions(header: str = HEADER):
    """Names of the functions include/pcs.h declares."""
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pcs_[a-z_0-9]+)\s*\(", text)))


def last_error() -> str:
    return load_library().pcs_last_error().decode()


def _check(status: int, where: str):
    if status != PCS_OK:
        raise PcsError(status, where, last_error())


def _dev_ptr(t, dtype_name: str, shape, what: str):
    import torch

    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{what} must be a torch tensor")
    if not t.is_cuda:
        raise ValueError(f"{what} must be on a CUDA device")
    if str(t.dtype) != f"torch.{dtype_name}":
        raise TypeError(f"{what} must be {dtype_name}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{what} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _host_ptr(a, dtype, shape, what: str):
    import numpy as np

    if not isinstance(a, np.ndarray) or a.dtype != dtype or tuple(a.shape) != tuple(shape):
        raise TypeError(f"{what} must be a numpy {np.dtype(dtype).name} array of shape {tuple(shape)}")
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError(f"{what} must be C-contiguous")
    return ctypes.c_void_p(a.ctypes.data)


# --------------------------------------------------------------------------- C-named wrappers


def pcs_supported_size(H: int, W: int) -> bool:
    return bool(load_library().pcs_supported_size(H, W))


KERNEL_DEFAULT, KERNEL_STREAMING, KERNEL_RESIDENT = 0, 1, 2


def pcs_create(H: int, W: int, max_slices: int, b0_axis: int = 0, cluster_size: int = 0, max_clusters: int = 0,
               kernel: int = KERNEL_DEFAULT, threads: int = 0, use_graph: bool = False, tv: int = 0,
               stream=None, tile: int = 0):
    """Create a context; returns an opaque handle (c_void_p).  stream: torch.cuda.Stream or None (current)."""
    import torch

    lib = load_library()
    opt = pcs_options()
    lib.pcs_options_default(ctypes.byref(opt))
    opt.b0_axis, opt.cluster_size, opt.max_clusters, opt.kernel = b0_axis, cluster_size, max_clusters, kernel
    opt.threads = threads
    opt.use_graph = 1 if use_graph else 0
    opt.tv = tv
    opt.tile = tile
    s = (stream or torch.cuda.current_stream()).cuda_stream
    h = ctypes.c_void_p()
    _check(lib.pcs_create(ctypes.byref(h), H, W, max_slices, ctypes.byref(opt), ctypes.c_void_p(s)), "pcs_create")
    return h


def pcs_set_stream(ctx, stream):
    _check(load_library().pcs_set_stream(ctx, ctypes.c_void_p(stream.cuda_stream)), "pcs_set_stream")


def pcs_solve_slices(ctx, field, mask, lam: float, tau: float, sigma: float, n_iter: int, chi_out, report=False):
    """Solve every slice of field/mask ([S][H][W] float32 / uint8 CUDA tensors) into chi_out."""
    S, H, W = field.shape
    f = _dev_ptr(field, "float32", (S, H, W), "field")
    m = _dev_ptr(mask, "uint8", (S, H, W), "mask")
    c = _dev_ptr(chi_out, "float32", (S, H, W), "chi_out")
    rep = (pcs_slice_report * S)() if report and S > 0 else None
    _check(load_library().pcs_solve_slices(ctx, f, m, S, lam, tau, sigma, n_iter, c, rep), "pcs_solve_slices")
    return [r.as_dict() for r in rep] if rep is not None else None


def pcs_solve_slices_weighted(ctx, field, mask, weight, lam: float, tau: float, sigma: float, n_iter: int, chi_out,
                              report=False):
    """pcs_solve_slices with data weighting W = weight ([S][H][W] float32 CUDA tensor, values in [0, 1]);
    mask is the TV mask M."""
    S, H, W = field.shape
    f = _dev_ptr(field, "float32", (S, H, W), "field")
    m = _dev_ptr(mask, "uint8", (S, H, W), "mask")
    w = _dev_ptr(weight, "float32", (S, H, W), "weight")
    c = _dev_ptr(chi_out, "float32", (S, H, W), "chi_out")
    rep = (pcs_slice_report * S)() if report and S > 0 else None
    _check(load_library().pcs_solve_slices_weighted(ctx, f, m, w, S, lam, tau, sigma, n_iter, c, rep),
           "pcs_solve_slices_weighted")
    return [r.as_dict() for r in rep] if rep is not None else None


def pcs_solve_volume_3d(field, mask, lam: float, tau: float, sigma: float, n_iter: int, chi_out, tv: int = 0,
                        weight=None, stream=None, report=False, voxel=None):
    """3-D solve of one volume (field/mask/chi_out: [S][H][W] float32/uint8/float32 CUDA tensors;
    weight: optional float32 data weighting W, default W = mask).  report=True returns the
    volume's FP64 diagnostics as a dict (objective, gap, stationarity, data_residual, iters).
    voxel: optional (dz, dy, dx) voxel edge lengths (default isotropic)."""
    import torch

    S, H, W = field.shape
    f = _dev_ptr(field, "float32", (S, H, W), "field")
    m = _dev_ptr(mask, "uint8", (S, H, W), "mask")
    w = None if weight is None else _dev_ptr(weight, "float32", (S, H, W), "weight")
    c = _dev_ptr(chi_out, "float32", (S, H, W), "chi_out")
    st = (stream or torch.cuda.current_stream()).cuda_stream
    rep = pcs_slice_report() if report else None
    vox = None if voxel is None else (ctypes.c_double * 3)(*[float(v) for v in voxel])
    _check(load_library().pcs_solve_volume_3d(f, m, w, S, H, W, lam, tau, sigma, n_iter, tv, vox, c,
                                              ctypes.byref(rep) if rep is not None else None, ctypes.c_void_p(st)),
           "pcs_solve_volume_3d")
    return rep.as_dict() if rep is not None else None


def pcs_solve_slices_generic(field, mask, lam: float, tau: float, sigma: float, n_iter: int, chi_out, tv: int = 0,
                             weight=None, b0_axis: int = 0, stream=None, report=False):
    """Per-slice solve for any even H x W with prime factors <= 61 (field/mask/chi_out: [S][H][W]
    float32/uint8/float32 CUDA tensors; weight: optional float32 data weighting W, default W = mask).
    report=True returns the per-slice FP64 reports as a list of dicts."""
    import torch

    S, H, W = field.shape
    f = _dev_ptr(field, "float32", (S, H, W), "field")
    m = _dev_ptr(mask, "uint8", (S, H, W), "mask")
    w = None if weight is None else _dev_ptr(weight, "float32", (S, H, W), "weight")
    c = _dev_ptr(chi_out, "float32", (S, H, W), "chi_out")
    st = (stream or torch.cuda.current_stream()).cuda_stream
    rep = (pcs_slice_report * S)() if report and S > 0 else None
    _check(load_library().pcs_solve_slices_generic(f, m, w, S, H, W, b0_axis, lam, tau, sigma, n_iter, tv, c, rep,
                                                   ctypes.c_void_p(st)),
           "pcs_solve_slices_generic")
    return [r.as_dict() for r in rep] if rep is not None else None


def pcs_supported_generic(H: int, W: int) -> bool:
    return bool(load_library().pcs_supported_generic(H, W))


def pcs_field_map(s0, s1, t_shift_s: float, b0_tesla: float, threshold: float, field_out, weight_out, mask_out,
                  stream=None):
    """Field map (ppm), weighting and mask from two complex64 CUDA tensors of the same shape."""
    import torch

    shape = tuple(s0.shape)
    a = _dev_ptr(torch.view_as_real(s0), "float32", shape + (2,), "s0")
    b = _dev_ptr(torch.view_as_real(s1), "float32", shape + (2,), "s1")
    f = _dev_ptr(field_out, "float32", shape, "field_out")
    w = _dev_ptr(weight_out, "float32", shape, "weight_out")
    m = _dev_ptr(mask_out, "uint8", shape, "mask_out")
    n = 1
    for x in shape:
        n *= x
    st = (stream or torch.cuda.current_stream()).cuda_stream
    _check(load_library().pcs_field_map(a, b, n, t_shift_s, b0_tesla, threshold, f, w, m, ctypes.c_void_p(st)),
           "pcs_field_map")


def pcs_schedule_plan(S: int, n_iter: int, clusters: int):
    """The balanced schedule: ([(slice, first, end, flags), ...], offsets per cluster)."""
    lib = load_library()
    n = ctypes.c_int(0)
    _check(lib.pcs_schedule_plan(S, n_iter, clusters, None, ctypes.byref(n), None), "pcs_schedule_plan")
    segs = (ctypes.c_int * (4 * n.value))()
    off = (ctypes.c_int * (clusters + 1))()
    _check(lib.pcs_schedule_plan(S, n_iter, clusters, segs, ctypes.byref(n), off), "pcs_schedule_plan")
    return [tuple(segs[4 * k:4 * k + 4]) for k in range(n.value)], list(off)


def pcs_check(ctx):
    """Synchronise the context's stream; raise if an earlier solve gave up a bounded wait."""
    _check(load_library().pcs_check(ctx), "pcs_check")


def pcs_selftest_wait(limit_cycles: int, stream=None) -> bool:
    """Run the schedule's bounded wait on a flag nothing sets; True if it gave up."""
    import torch

    out = ctypes.c_int(0)
    st = (stream or torch.cuda.current_stream()).cuda_stream
    _check(load_library().pcs_selftest_wait(ctypes.c_void_p(st), limit_cycles, ctypes.byref(out)), "pcs_selftest_wait")
    return bool(out.value)


def pcs_supported_volume_3d(S: int, H: int, W: int) -> bool:
    return bool(load_library().pcs_supported_volume_3d(S, H, W))


def pcs_solve_slices_host(ctx, field, mask, lam: float, tau: float, sigma: float, n_iter: int, chi_out, report=False):
    """Host-buffer variant: numpy arrays in (pinned or pageable), chi_out numpy array filled on return."""
    import numpy as np

    S, H, W = field.shape
    f = _host_ptr(field, np.float32, (S, H, W), "field")
    m = _host_ptr(mask, np.uint8, (S, H, W), "mask")
    c = _host_ptr(chi_out, np.float32, (S, H, W), "chi_out")
    rep = (pcs_slice_report * S)() if report and S > 0 else None
    _check(load_library().pcs_solve_slices_host(ctx, f, m, S, lam, tau, sigma, n_iter, c, rep),
           "pcs_solve_slices_host")
    return [r.as_dict() for r in rep] if rep is not None else None


def pcs_solve_slices_monitored(ctx, field, mask, lam: float, tau: float, sigma: float, n_iter: int, check_every: int,
                               rel_gap_tol: float, chi_out):
    """Chunked solve with FP64 diagnostics every check_every iterations and optional per-slice early stop."""
    S, H, W = field.shape
    f = _dev_ptr(field, "float32", (S, H, W), "field")
    m = _dev_ptr(mask, "uint8", (S, H, W), "mask")
    c = _dev_ptr(chi_out, "float32", (S, H, W), "chi_out")
    rep = (pcs_slice_report * max(S, 1))()
    _check(load_library().pcs_solve_slices_monitored(ctx, f, m, S, lam, tau, sigma, n_iter, check_every,
                                                     rel_gap_tol, c, rep), "pcs_solve_slices_monitored")
    return [rep[k].as_dict() for k in range(S)]


def pcs_report(ctx, field, mask, lam: float, chi):
    S, H, W = field.shape
    f = _dev_ptr(field, "float32", (S, H, W), "field")
    m = _dev_ptr(mask, "uint8", (S, H, W), "mask")
    c = _dev_ptr(chi, "float32", (S, H, W), "chi")
    rep = (pcs_slice_report * S)()
    _check(load_library().pcs_report(ctx, f, m, S, lam, c, rep), "pcs_report")
    return [r.as_dict() for r in rep]


def pcs_opnorm(ctx, mask, power_iters: int = 200):
    S, H, W = mask.shape
    m = _dev_ptr(mask, "uint8", (S, H, W), "mask")
    out = (ctypes.c_double * S)()
    _check(load_library().pcs_opnorm(ctx, m, S, power_iters, out), "pcs_opnorm")
    return list(out)


def pcs_solve_slices_noalloc(field, mask, lam: float, tau: float, sigma: float, n_iter: int, chi_out,
                             b0_axis: int = 0, stream=None):
    """Solve without any device allocation by the library (static scratch of
    PCS_NOALLOC_MAX_VOXELS voxels shared by all calls; see include/pcs.h)."""
    import torch

    S, H, W = field.shape
    f = _dev_ptr(field, "float32", (S, H, W), "field")
    m = _dev_ptr(mask, "uint8", (S, H, W), "mask")
    c = _dev_ptr(chi_out, "float32", (S, H, W), "chi_out")
    s = (stream or torch.cuda.current_stream()).cuda_stream
    _check(load_library().pcs_solve_slices_noalloc(f, m, H, W, S, lam, tau, sigma, n_iter, c, b0_axis,
                                                   ctypes.c_void_p(s)), "pcs_solve_slices_noalloc")


def pcs_destroy(ctx):
    if ctx is not None:
        load_library().pcs_destroy(ctx)


def pcs_solve_slices_f64(field, mask, lam: float, tau: float, sigma: float, n_iter: int, chi_out, b0_axis: int = 0,
                         stream=None):
    """All-FP64 solve of field/mask (float64 / uint8 CUDA tensors [S][H][W]) into chi_out (float64)."""
    import torch

    S, H, W = field.shape
    f = _dev_ptr(field, "float64", (S, H, W), "field")
    m = _dev_ptr(mask, "uint8", (S, H, W), "mask")
    c = _dev_ptr(chi_out, "float64", (S, H, W), "chi_out")
    s = (stream or torch.cuda.current_stream()).cuda_stream
    _check(load_library().pcs_solve_slices_f64(f, m, H, W, S, lam, tau, sigma, n_iter, c, b0_axis,
                                               ctypes.c_void_p(s)), "pcs_solve_slices_f64")


def pcs_batch_create(autotune: bool = True, stream=None, **opts):
    """Create an uneven-batch solver (see include/pcs.h); opts as for pcs_create."""
    import torch

    lib = load_library()
    opt = pcs_options()
    lib.pcs_options_default(ctypes.byref(opt))
    for k, v in opts.items():
        setattr(opt, k, int(v))
    s = (stream or torch.cuda.current_stream()).cuda_stream
    h = ctypes.c_void_p()
    _check(lib.pcs_batch_create(ctypes.byref(h), ctypes.byref(opt), 1 if autotune else 0, ctypes.c_void_p(s)),
           "pcs_batch_create")
    return h


def pcs_batch_solve(batch, volumes, n_iter: int):
    """volumes: list of (field, mask, lam, chi_out) with [S][H][W] CUDA tensors."""
    arr = (pcs_volume * max(1, len(volumes)))()
    for k, (field, mask, lam, chi) in enumerate(volumes):
        S, H, W = field.shape
        arr[k].H, arr[k].W, arr[k].S, arr[k].lam = H, W, S, lam
        arr[k].field = _dev_ptr(field, "float32", (S, H, W), "field").value
        arr[k].mask = _dev_ptr(mask, "uint8", (S, H, W), "mask").value
        arr[k].chi_out = _dev_ptr(chi, "float32", (S, H, W), "chi_out").value
    _check(load_library().pcs_batch_solve(batch, arr, len(volumes), n_iter), "pcs_batch_solve")


def pcs_batch_tuning(batch, H: int, W: int):
    t = pcs_tuning()
    _check(load_library().pcs_batch_tuning(batch, H, W, ctypes.byref(t)), "pcs_batch_tuning")
    return t.as_dict()


def pcs_batch_check(batch):
    """Synchronise the batch stream; raise PcsError(PCS_ETIMEOUT) if a launch gave up a bounded wait."""
    _check(load_library().pcs_batch_check(batch), "pcs_batch_check")


def pcs_batch_destroy(batch):
    if batch is not None:
        load_library().pcs_batch_destroy(batch)


def pcs_serve_start(hbm_budget_bytes: int, slots: int = 8, n_iter: int = 400, autotune: bool = True,
                    b0_axis: int = 0):
    """Start a serving loop (scheduler thread in libpcs); returns its handle."""
    cfg = pcs_server_config()
    cfg.hbm_budget_bytes, cfg.slots, cfg.n_iter = int(hbm_budget_bytes), slots, n_iter
    cfg.autotune, cfg.b0_axis = 1 if autotune else 0, b0_axis
    h = ctypes.c_void_p()
    _check(load_library().pcs_serve_start(ctypes.byref(h), ctypes.byref(cfg)), "pcs_serve_start")
    return h


def pcs_serve_prepare_size(server, H: int, W: int):
    t = pcs_tuning()
    _check(load_library().pcs_serve_prepare_size(server, H, W, ctypes.byref(t)), "pcs_serve_prepare_size")
    return t.as_dict()


def pcs_serve_open(server, H: int, W: int, S: int, lam: float, chi_host) -> int:
    """chi_host: numpy float32 [S][H][W] (pinned recommended), filled when the request completes."""
    import numpy as np

    c = _host_ptr(chi_host, np.float32, (S, H, W), "chi_host")
    rid = ctypes.c_longlong()
    _check(load_library().pcs_serve_open(server, H, W, S, lam, c, ctypes.byref(rid)), "pcs_serve_open")
    return rid.value


def pcs_serve_push(server, rid: int, s0: int, field_host, mask_host):
    """Slices s0.. of request rid have arrived: numpy float32 / uint8 [n][H][W] (kept alive by the caller)."""
    import numpy as np

    n, H, W = field_host.shape
    f = _host_ptr(field_host, np.float32, (n, H, W), "field_host")
    m = _host_ptr(mask_host, np.uint8, (n, H, W), "mask_host")
    _check(load_library().pcs_serve_push(server, rid, s0, n, f, m), "pcs_serve_push")


def pcs_serve_poll(server, max_items: int = 256):
    """Finished requests since the last poll: [(id, latency_s, status)], status PCS_OK or an error code."""
    ids = (ctypes.c_longlong * max_items)()
    lat = (ctypes.c_double * max_items)()
    st = (ctypes.c_int * max_items)()
    n = ctypes.c_int()
    _check(load_library().pcs_serve_poll(server, ids, lat, st, max_items, ctypes.byref(n)), "pcs_serve_poll")
    return [(ids[k], lat[k], st[k]) for k in range(n.value)]


def pcs_serve_arena_plan(capacity: int, ops):
    """Replay allocate (> 0 bytes) / release (-(k+1): the range of op k) ops on the serving arena's
    host-side placement; returns (offsets, bytes in use after each op)."""
    n = len(ops)
    arr = (ctypes.c_longlong * max(1, n))(*ops)
    off = (ctypes.c_longlong * max(1, n))()
    used = (ctypes.c_size_t * max(1, n))()
    _check(load_library().pcs_serve_arena_plan(capacity, arr, n, off, used), "pcs_serve_arena_plan")
    return list(off)[:n], list(used)[:n]


def pcs_serve_request_bytes(H: int, W: int, S: int) -> int:
    """Device bytes one request holds while admitted (its share of the server's budget)."""
    out = ctypes.c_size_t()
    _check(load_library().pcs_serve_request_bytes(H, W, S, ctypes.byref(out)), "pcs_serve_request_bytes")
    return out.value


def pcs_serve_fail_next_launch(server, rid: int):
    """Host-side failure injection (tests): the next launch of request rid reports an error."""
    _check(load_library().pcs_serve_fail_next_launch(server, rid), "pcs_serve_fail_next_launch")


def pcs_serve_stats(server):
    out = pcs_serve_summary()
    _check(load_library().pcs_serve_stats(server, ctypes.byref(out)), "pcs_serve_stats")
    return out.as_dict()


def pcs_serve_stop(server):
    if server is not None:
        load_library().pcs_serve_stop(server)


class Solver:
    """Owns one context: ``with Solver(H, W, S) as s: s.solve(field, mask, lam, n_iter)``."""

    def __init__(self, H: int, W: int, max_slices: int, **opts):
        self.H, self.W, self.max_slices = H, W, max_slices
        self.ctx = pcs_create(H, W, max_slices, **opts)
        self._L = None

    def step_sizes(self, power_iters: int = 300):
        """(L, tau, sigma) with tau = sigma = 1/L for the full-mask operator of this slice size
        (device power iteration)."""
        import torch

        if self._L is None:
            ones = torch.ones((1, self.H, self.W), dtype=torch.uint8, device="cuda")
            self._L = pcs_opnorm(self.ctx, ones, power_iters)[0]
        return self._L, 1.0 / self._L, 1.0 / self._L

    def solve(self, field, mask, lam: float, n_iter: int, tau: float | None = None, sigma: float | None = None,
              chi_out=None, report=False):
        import torch

        if tau is None or sigma is None:
            _, tau, sigma = self.step_sizes()
        if chi_out is None:
            chi_out = torch.empty_like(field)
        rep = pcs_solve_slices(self.ctx, field, mask, lam, tau, sigma, n_iter, chi_out, report=report)
        return (chi_out, rep) if report else chi_out

    def close(self):
        pcs_destroy(self.ctx)
        self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
