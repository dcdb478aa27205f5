"""FP64 CPU oracle for the 3-D variant of the primal-dual iteration.

TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it.  It shares no code with the CUDA path.

Eq. (1) read literally: the gradient G acts "in all three dimensions"
(Sec. II.A) and D is the 3-D dipole convolution of the whole volume, so the
slices of a volume are coupled.  The iteration is the same Sec. II.A
pseudocode as the per-slice oracle (``pd_oracle.pd_solve``) with the volume as
one unknown:

    p  <- (p + sigma (W D chibar - W dB)) / (1 + sigma/lambda)
    q  <- clamp(q + sigma M G chibar)             q = (qx, qy, qz)
    chi+ = chi - tau (D W p + G^T M q)
    chibar = chi+ + theta (chi+ - chi)

Readings (the paper is silent on each):

* Volume layout [S][H][W] = (z, y, x); B0 along z, the slice axis
  (``dipole_kernel_3d(shape, b0_axis=0)``): D(k) = 1/3 - kz^2/|k|^2, D(0) = 0,
  circular on the S x H x W grid.  k is the physical frequency: cycles per
  sample divided by the voxel's edge along that axis (``voxel`` = (dz, dy, dx),
  default isotropic; the paper's acquisitions have 0.72 x 0.72 mm pixels and
  2 mm slices, Sec. III).  G stays the unit forward difference (the paper gives
  no scaling of it).
* G: forward differences along x, y and z with a Neumann boundary (zero
  difference on the last column, row and slice); G^T its exact adjoint.
* The TV dual prox clamps each of the three components (anisotropic);
  ``tv="iso"`` projects (qx, qy, qz) onto the unit ball instead.
* W = M = mask (0/1) unless given.

numpy's n-D FFT is a library primitive; the rest follows the pseudocode.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

from .pd_oracle import Diagnostics, apply_D_3d, clamp_unit, dipole_kernel_3d, prox_dual_data


def grad3(x: np.ndarray):
    """Forward differences with a Neumann boundary: (gx along x, gy along y, gz along z)."""
    gx = np.zeros_like(x)
    gy = np.zeros_like(x)
    gz = np.zeros_like(x)
    gx[:, :, :-1] = x[:, :, 1:] - x[:, :, :-1]
    gy[:, :-1, :] = x[:, 1:, :] - x[:, :-1, :]
    gz[:-1, :, :] = x[1:, :, :] - x[:-1, :, :]
    return gx, gy, gz


def grad3_adjoint(a: np.ndarray, b: np.ndarray, c: np.ndarray) -> np.ndarray:
    """G^T (a, b, c): the exact adjoint of ``grad3``."""
    out = np.zeros_like(a)
    out[:, :, 1:] += a[:, :, :-1]
    out[:, :, :-1] -= a[:, :, :-1]
    out[:, 1:, :] += b[:, :-1, :]
    out[:, :-1, :] -= b[:, :-1, :]
    out[1:, :, :] += c[:-1, :, :]
    out[:-1, :, :] -= c[:-1, :, :]
    return out


def prox_dual_tv3_iso(vx, vy, vz):
    """Isotropic reading: project each (vx, vy, vz) onto the unit ball."""
    n = np.maximum(1.0, np.sqrt(vx * vx + vy * vy + vz * vz))
    return vx / n, vy / n, vz / n


@dataclasses.dataclass
class PDState3:
    chi: np.ndarray
    chi_bar: np.ndarray
    p: np.ndarray
    qx: np.ndarray
    qy: np.ndarray
    qz: np.ndarray
    n: int


def pd_solve_3d(
    field: np.ndarray,
    mask: np.ndarray,
    lam: float,
    tau: float,
    sigma: float,
    n_iter: int,
    weight: np.ndarray | None = None,
    tv_mask: np.ndarray | None = None,
    theta: float = 1.0,
    return_state: bool = False,
    tv: str = "aniso",
    voxel=None,
):
    """N iterations of the Sec. II.A pseudocode on a whole [S][H][W] volume, in FP64."""
    f = np.asarray(field, dtype=np.float64)
    m = np.asarray(mask, dtype=np.float64)
    Wt = m if weight is None else np.asarray(weight, dtype=np.float64)
    Mt = m if tv_mask is None else np.asarray(tv_mask, dtype=np.float64)
    Dk = dipole_kernel_3d(f.shape, b0_axis=0, voxel=voxel)
    b = Wt * f

    # zero start, chi_bar_0 = chi_0
    chi = np.zeros_like(f)
    chi_bar = chi.copy()
    p = np.zeros_like(f)
    qx = np.zeros_like(f)
    qy = np.zeros_like(f)
    qz = np.zeros_like(f)

    for _ in range(n_iter):
        # dual data prox
        p = prox_dual_data(p + sigma * (Wt * apply_D_3d(chi_bar, Dk)), b, sigma, lam)
        # dual TV prox on the three difference components
        gx, gy, gz = grad3(chi_bar)
        vx, vy, vz = qx + sigma * Mt * gx, qy + sigma * Mt * gy, qz + sigma * Mt * gz
        if tv == "iso":
            qx, qy, qz = prox_dual_tv3_iso(vx, vy, vz)
        else:
            qx, qy, qz = clamp_unit(vx), clamp_unit(vy), clamp_unit(vz)
        # primal step (identity prox) and over-relaxation
        chi_new = chi - tau * apply_D_3d(Wt * p, Dk) - tau * grad3_adjoint(Mt * qx, Mt * qy, Mt * qz)
        chi_bar = chi_new + theta * (chi_new - chi)
        chi = chi_new

    if return_state:
        return PDState3(chi=chi, chi_bar=chi_bar, p=p, qx=qx, qy=qy, qz=qz, n=n_iter)
    return chi


def diagnostics_3d(
    state: PDState3,
    field: np.ndarray,
    mask: np.ndarray,
    lam: float,
    weight: np.ndarray | None = None,
    tv_mask: np.ndarray | None = None,
    tv: str = "aniso",
    voxel=None,
) -> Diagnostics:
    """Objective, Fenchel-Young gap, stationarity and residual of the 3-D problem
    at (chi, p, q) (the same terms as ``pd_oracle.diagnostics``)."""
    f = np.asarray(field, dtype=np.float64)
    m = np.asarray(mask, dtype=np.float64)
    Wt = m if weight is None else np.asarray(weight, dtype=np.float64)
    Mt = m if tv_mask is None else np.asarray(tv_mask, dtype=np.float64)
    Dk = dipole_kernel_3d(f.shape, b0_axis=0, voxel=voxel)
    r = Wt * apply_D_3d(state.chi, Dk) - Wt * f
    gx, gy, gz = (Mt * g for g in grad3(state.chi))
    if tv == "iso":
        tvn = float(np.sum(np.sqrt(gx * gx + gy * gy + gz * gz)))
    else:
        tvn = float(np.sum(np.abs(gx)) + np.sum(np.abs(gy)) + np.sum(np.abs(gz)))
    primal = 0.5 * lam * float(np.sum(r * r)) + tvn
    fy1 = float(np.sum((state.p - lam * r) ** 2)) / (2.0 * lam)
    fy2 = tvn - float(np.sum(state.qx * gx) + np.sum(state.qy * gy) + np.sum(state.qz * gz))
    kty = apply_D_3d(Wt * state.p, Dk) + grad3_adjoint(Mt * state.qx, Mt * state.qy, Mt * state.qz)
    return Diagnostics(
        primal=primal,
        gap=fy1 + fy2,
        stationarity=float(np.sqrt(np.sum(kty * kty))),
        data_residual=float(np.sqrt(np.sum(r * r))),
    )


def apply_K3(x, Dk, Wt, Mt):
    """K x = (W D x, M gx, M gy, M gz)."""
    gx, gy, gz = grad3(x)
    return Wt * apply_D_3d(x, Dk), Mt * gx, Mt * gy, Mt * gz


def apply_KT3(y0, y1, y2, y3, Dk, Wt, Mt):
    """K^T y = D W y0 + G^T (M y1, M y2, M y3)."""
    return apply_D_3d(Wt * y0, Dk) + grad3_adjoint(Mt * y1, Mt * y2, Mt * y3)


def opnorm_3d(
    mask: np.ndarray,
    max_iter: int = 5000,
    rtol: float = 1e-12,
    seed: int = 1234,
    weight: np.ndarray | None = None,
    tv_mask: np.ndarray | None = None,
    voxel=None,
) -> float:
    """L = ||K||_2 of the 3-D operator by power iteration on K^T K."""
    m = np.asarray(mask, dtype=np.float64)
    Wt = m if weight is None else np.asarray(weight, dtype=np.float64)
    Mt = m if tv_mask is None else np.asarray(tv_mask, dtype=np.float64)
    Dk = dipole_kernel_3d(m.shape, b0_axis=0, voxel=voxel)
    x = np.random.default_rng(seed).standard_normal(m.shape)
    x /= np.linalg.norm(x)
    est = 0.0
    for _ in range(max_iter):
        y = apply_KT3(*apply_K3(x, Dk, Wt, Mt), Dk, Wt, Mt)
        new = float(np.vdot(x, y))
        nrm = float(np.linalg.norm(y))
        if nrm == 0.0:
            return 0.0
        x = y / nrm
        if est > 0 and abs(new - est) <= rtol * new:
            est = new
            break
        est = new
    return math.sqrt(est)
