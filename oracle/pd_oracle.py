"""FP64 CPU oracle for the per-slice primal-dual (Chambolle-Pock) iteration.

TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it.  It shares no code with the CUDA path.

What it computes (Wang et al., "Positive Contrast Susceptibility MR Imaging
Using GPU-based Primal-Dual Algorithm"):

    chi = argmin_chi  lambda/2 ||W(D chi - dB)||^2 + ||M G chi||_1        Eq. (1)

solved slice by slice with the first-order primal-dual iteration of the
Sec. II.A pseudocode: L = ||K||_2, tau = sigma = 1/L, theta = 1, zero start,
then repeat (dual data prox, dual TV prox, primal step, over-relaxation) until
n >= N, with K = [W D; M G] (the operator of F(K chi), Sec. II.A).

Readings of the paper taken here (the paper is silent or ambiguous on each):

* 2-D per slice: D and G act in the slice plane; slices are independent
  (Sec. II.C.2).  B0 lies in-plane along y, the rows axis (``b0_axis=0``).
* D chi = Re IFFT2( D(k) FFT2(chi) ), D(k) = 1/3 - k_par^2/|k|^2, D(0) = 0,
  circular on the H x W slice, k from ``numpy.fft.fftfreq`` (cycles/pixel,
  isotropic in-plane pixels).
* G: forward differences with a Neumann boundary (zero difference on the last
  column / row); G^T is its exact adjoint (minus a backward divergence).
* W = M = mask (0/1) by default; the data prox uses the weighted field
  b = W * dB, which is the exact prox of the Eq. (1) data term.
* The norm in the TV dual prox is taken componentwise (anisotropic), the
  literal dual of the l1 norm in Eq. (1): the prox is a clamp to [-1, 1].
  ``tv="iso"`` takes the other reading (pointwise Euclidean norm, isotropic
  TV): the prox projects (qx, qy) onto the unit disc.
* The primal function is zero, so prox_tau[G] is the identity: the primal
  step is chi - tau K^T y.
* Fixed iteration count N; the output is chi_N (not chi-bar).

numpy's FFT is used as a library primitive; every other step is written out
in the order the pseudocode gives it.  Parity is pinned by
``tests/test_oracle_*.py`` against closed forms, dense brute force, adjoint
identities, prox optimality, a per-frequency closed form of the linear case,
and KKT certificates.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np


# --------------------------------------------------------------------------- operators


def frequencies(H: int, W: int):
    """(ky, kx) grids in cycles per pixel, ky along rows (axis 0)."""
    ky = np.fft.fftfreq(H)[:, None]
    kx = np.fft.fftfreq(W)[None, :]
    return ky, kx


def dipole_kernel(H: int, W: int, b0_axis: int = 0) -> np.ndarray:
    """D(k) = 1/3 - k_par^2 / |k|^2 with D(0) = 0 on the FFT grid (Eq. (1)'s D).

    ``b0_axis`` = 0: B0 along y (rows); 1: along x (columns).
    """
    ky, kx = frequencies(H, W)
    k2 = kx * kx + ky * ky
    kpar2 = (ky * ky) if b0_axis == 0 else (kx * kx)
    kpar2 = np.broadcast_to(kpar2, k2.shape)
    D = np.zeros((H, W), dtype=np.float64)
    nz = k2 > 0
    D[nz] = 1.0 / 3.0 - kpar2[nz] / k2[nz]
    return D


def dipole_kernel_3d(shape, b0_axis: int = 0, voxel=None) -> np.ndarray:
    """3-D D(k) = 1/3 - k_par^2 / |k|^2, D(0) = 0, B0 along ``b0_axis``.

    ``voxel``: the voxel's edge lengths along the three axes (any unit; None =
    isotropic).  D depends on the physical frequencies k_i = f_i / voxel_i, f_i in
    cycles per sample; only their ratios matter.
    """
    vox = (1.0, 1.0, 1.0) if voxel is None else tuple(float(v) for v in voxel)
    ks = np.meshgrid(*[np.fft.fftfreq(n) / v for n, v in zip(shape, vox)], indexing="ij")
    k2 = sum(k * k for k in ks)
    D = np.zeros(shape, dtype=np.float64)
    nz = k2 > 0
    D[nz] = 1.0 / 3.0 - (ks[b0_axis] ** 2)[nz] / k2[nz]
    return D


def apply_D(x: np.ndarray, Dk: np.ndarray) -> np.ndarray:
    """Dipole convolution F^-1 D(k) F x on the last two axes (real in, real out).

    D(k) is real and even, so the result is real up to rounding; the
    discarded imaginary part is checked to be at rounding level.
    """
    y = np.fft.ifft2(Dk * np.fft.fft2(x, axes=(-2, -1)), axes=(-2, -1))
    scale = max(float(np.max(np.abs(x))), 1e-300)
    assert float(np.max(np.abs(y.imag))) <= 1e-10 * scale, "imaginary leak in D"
    return y.real


def apply_D_3d(x: np.ndarray, Dk: np.ndarray) -> np.ndarray:
    """3-D dipole convolution F^-1 D(k) F x (real part)."""
    return np.fft.ifftn(Dk * np.fft.fftn(x)).real


def grad(x: np.ndarray):
    """Forward differences with Neumann boundary: (gx along columns, gy along rows)."""
    gx = np.zeros_like(x)
    gy = np.zeros_like(x)
    gx[..., :, :-1] = x[..., :, 1:] - x[..., :, :-1]
    gy[..., :-1, :] = x[..., 1:, :] - x[..., :-1, :]
    return gx, gy


def grad_adjoint(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """G^T (a, b): the exact adjoint of ``grad`` (minus a backward divergence)."""
    out = np.zeros_like(a)
    out[..., :, 1:] += a[..., :, :-1]
    out[..., :, :-1] -= a[..., :, :-1]
    out[..., 1:, :] += b[..., :-1, :]
    out[..., :-1, :] -= b[..., :-1, :]
    return out


def soft_threshold(v: np.ndarray, t: float) -> np.ndarray:
    """sign(v) max(|v| - t, 0): the prox of t*||.||_1."""
    return np.sign(v) * np.maximum(np.abs(v) - t, 0.0)


def clamp_unit(v: np.ndarray) -> np.ndarray:
    """Projection onto the l-inf unit ball: v / max(1, |v|) componentwise."""
    return v / np.maximum(1.0, np.abs(v))


def prox_dual_data(v: np.ndarray, b: np.ndarray, sigma: float, lam: float) -> np.ndarray:
    """prox of sigma F1^* for F1(z) = lambda/2 ||z - b||^2: (v - sigma b) / (1 + sigma/lambda)."""
    return (v - sigma * b) / (1.0 + sigma / lam)


def prox_dual_tv(v: np.ndarray) -> np.ndarray:
    """prox of sigma F2^* for F2 = ||.||_1 (indicator of the unit ball): a clamp."""
    return clamp_unit(v)


def prox_dual_tv_iso(vx: np.ndarray, vy: np.ndarray):
    """Isotropic reading: F2 = sum of pointwise Euclidean norms of (gx, gy); its
    conjugate's prox projects each (vx, vy) onto the unit disc:
    v / max(1, |v|_2)."""
    n = np.maximum(1.0, np.sqrt(vx * vx + vy * vy))
    return vx / n, vy / n


# --------------------------------------------------------------------------- solver


@dataclasses.dataclass
class PDState:
    chi: np.ndarray
    chi_bar: np.ndarray
    p: np.ndarray
    qx: np.ndarray
    qy: np.ndarray
    n: int


def pd_solve(
    field: np.ndarray,
    mask: np.ndarray,
    lam: float,
    tau: float,
    sigma: float,
    n_iter: int,
    b0_axis: int = 0,
    weight: np.ndarray | None = None,
    tv_mask: np.ndarray | None = None,
    theta: float = 1.0,
    return_state: bool = False,
    tv: str = "aniso",
):
    """Run N iterations of the Sec. II.A primal-dual pseudocode in FP64.

    ``field`` (dB, ppm) and ``mask`` are [H][W] or [S][H][W]; slices are
    solved independently.  W = ``weight`` (default: mask) and M = ``tv_mask``
    (default: mask).  ``tv``: "aniso" reads the norm of the TV dual prox
    componentwise (clamp), "iso" pointwise Euclidean (projection onto the unit
    disc).  Returns chi_N (float64), or the full state when ``return_state``
    is true.
    """
    f = np.asarray(field, dtype=np.float64)
    m = np.asarray(mask, dtype=np.float64)
    Wt = m if weight is None else np.asarray(weight, dtype=np.float64)
    Mt = m if tv_mask is None else np.asarray(tv_mask, dtype=np.float64)
    H, W = f.shape[-2:]
    Dk = dipole_kernel(H, W, b0_axis)
    b = Wt * f

    # pseudocode steps 1-3: zero start, chi_bar_0 = chi_0
    chi = np.zeros_like(f)
    chi_bar = chi.copy()
    p = np.zeros_like(f)
    qx = np.zeros_like(f)
    qy = np.zeros_like(f)

    for _ in range(n_iter):
        # dual data prox: p <- (p + sigma (W D chi_bar - dB_w)) / (1 + sigma/lambda)
        p = prox_dual_data(p + sigma * (Wt * apply_D(chi_bar, Dk)), b, sigma, lam)
        # dual TV prox: q <- (q + sigma M G chi_bar) / max(1, |.|)
        gx, gy = grad(chi_bar)
        if tv == "iso":
            qx, qy = prox_dual_tv_iso(qx + sigma * Mt * gx, qy + sigma * Mt * gy)
        else:
            qx = prox_dual_tv(qx + sigma * Mt * gx)
            qy = prox_dual_tv(qy + sigma * Mt * gy)
        # primal step: chi+ = chi - tau D^T W^T p - tau G^T M^T q  (prox of 0 = identity)
        chi_new = chi - tau * apply_D(Wt * p, Dk) - tau * grad_adjoint(Mt * qx, Mt * qy)
        # over-relaxation: chi_bar = chi+ + theta (chi+ - chi)
        chi_bar = chi_new + theta * (chi_new - chi)
        chi = chi_new

    if return_state:
        return PDState(chi=chi, chi_bar=chi_bar, p=p, qx=qx, qy=qy, n=n_iter)
    return chi


# --------------------------------------------------------------------------- diagnostics


@dataclasses.dataclass
class Diagnostics:
    primal: float  # lambda/2 ||W(D chi - dB)||^2 + ||M G chi||_1
    gap: float  # Fenchel-Young gap of (chi, p, q); >= 0, = 0 iff optimal with stationarity
    stationarity: float  # ||D W p + G^T M q||_2 = ||K^T y||
    data_residual: float  # ||W (D chi - dB)||_2


def diagnostics(
    state: PDState,
    field: np.ndarray,
    mask: np.ndarray,
    lam: float,
    b0_axis: int = 0,
    weight: np.ndarray | None = None,
    tv_mask: np.ndarray | None = None,
    tv: str = "aniso",
) -> Diagnostics:
    """Objective, Fenchel-Young gap and stationarity of Eq. (1) at (chi, p, q).

    With F1(z) = lambda/2||z - b||^2 and F2 = ||.||_1 the Fenchel-Young terms
    are F1(z) + F1*(p) - <p, z> = ||p - lambda (z - b)||^2 / (2 lambda) for
    z = W D chi, and ||g||_1 - <q, g> for g = M G chi (with |q| <= 1).  Both
    are >= 0, and together with K^T y = 0 they vanish exactly at a saddle
    point.  Sums run over the whole array (all slices).
    """
    f = np.asarray(field, dtype=np.float64)
    m = np.asarray(mask, dtype=np.float64)
    Wt = m if weight is None else np.asarray(weight, dtype=np.float64)
    Mt = m if tv_mask is None else np.asarray(tv_mask, dtype=np.float64)
    H, W = f.shape[-2:]
    Dk = dipole_kernel(H, W, b0_axis)
    b = Wt * f
    z = Wt * apply_D(state.chi, Dk)
    gx, gy = grad(state.chi)
    gx, gy = Mt * gx, Mt * gy
    r = z - b
    if tv == "iso":
        tvn = float(np.sum(np.sqrt(gx * gx + gy * gy)))
    else:
        tvn = float(np.sum(np.abs(gx)) + np.sum(np.abs(gy)))
    primal = 0.5 * lam * float(np.sum(r * r)) + tvn
    fy1 = float(np.sum((state.p - lam * r) ** 2)) / (2.0 * lam)
    fy2 = tvn - float(np.sum(state.qx * gx) + np.sum(state.qy * gy))
    kty = apply_D(Wt * state.p, Dk) + grad_adjoint(Mt * state.qx, Mt * state.qy)
    return Diagnostics(
        primal=primal,
        gap=fy1 + fy2,
        stationarity=float(np.sqrt(np.sum(kty * kty))),
        data_residual=float(np.sqrt(np.sum(r * r))),
    )


# --------------------------------------------------------------------------- step sizes


def apply_K(x, Dk, Wt, Mt):
    """K x = (W D x, M gx, M gy)."""
    gx, gy = grad(x)
    return Wt * apply_D(x, Dk), Mt * gx, Mt * gy


def apply_KT(y0, y1, y2, Dk, Wt, Mt):
    """K^T (y0, y1, y2) = D W y0 + G^T (M y1, M y2)."""
    return apply_D(Wt * y0, Dk) + grad_adjoint(Mt * y1, Mt * y2)


def opnorm(
    mask: np.ndarray,
    b0_axis: int = 0,
    max_iter: int = 5000,
    rtol: float = 1e-12,
    seed: int = 1234,
    weight: np.ndarray | None = None,
    tv_mask: np.ndarray | None = None,
) -> float:
    """L = ||K||_2 by power iteration on K^T K (pseudocode step 1).

    Starts from a seeded Gaussian vector and stops when the Rayleigh
    estimate of ||K||^2 changes by less than ``rtol`` (relative).
    """
    m = np.asarray(mask, dtype=np.float64)
    Wt = m if weight is None else np.asarray(weight, dtype=np.float64)
    Mt = m if tv_mask is None else np.asarray(tv_mask, dtype=np.float64)
    H, W = m.shape[-2:]
    Dk = dipole_kernel(H, W, b0_axis)
    x = np.random.default_rng(seed).standard_normal(m.shape)
    x /= np.linalg.norm(x)
    est = 0.0
    for _ in range(max_iter):
        y = apply_KT(*apply_K(x, Dk, Wt, Mt), Dk, Wt, Mt)
        new = float(np.vdot(x, y))  # Rayleigh quotient of K^T K (x normalised)
        nrm = float(np.linalg.norm(y))
        if nrm == 0.0:
            return 0.0
        x = y / nrm
        if est > 0 and abs(new - est) <= rtol * new:
            est = new
            break
        est = new
    return math.sqrt(est)


def step_sizes(H: int, W: int, b0_axis: int = 0):
    """(L, tau, sigma) with tau = sigma = 1/L for the full-mask operator of an H x W slice.

    A 0/1 mask only shrinks ||K||, so these steps are valid for every mask of
    that size.
    """
    L = opnorm(np.ones((H, W)), b0_axis=b0_axis)
    return L, 1.0 / L, 1.0 / L
