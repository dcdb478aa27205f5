"""Worker functions for spawn process pools in the GPU tests (oracle solves and phantom
generation on every host core).  Importing this module touches no GPU."""

import numpy as np


def oracle_slice(args):
    """chi_N of one slice by the FP64 oracle: (field, mask, lam, tau, sigma, n_iter) -> array."""
    from oracle import pd_oracle as O

    f, m, lam, tau, sigma, n_iter = args
    return O.pd_solve(np.asarray(f, np.float64), m, lam, tau, sigma, n_iter)


def gen_volume(spec):
    """(field, mask) of one volume of the uneven-batch recipe."""
    import phantoms

    pb = phantoms.volume(spec["size"], spec["size"], spec["slices"], seed=spec["seed"], lam=spec["lam"],
                         n_iter=spec["n_iter"])
    return pb.field, pb.mask


def spawn_pool():
    """A process pool on every host core, started with spawn (safe next to a CUDA context)."""
    import multiprocessing as mp
    import os
    from concurrent.futures import ProcessPoolExecutor

    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(var, "1")
    return ProcessPoolExecutor(max_workers=os.cpu_count() or 1, mp_context=mp.get_context("spawn"))
