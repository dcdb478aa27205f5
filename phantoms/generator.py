"""Seeded phantoms and simulated field maps (inputs only; no solver arithmetic).

Conventions shared with every consumer of these inputs:

* a slice is H x W, row index i runs along y, column index j along x; stacks
  are ``[S][H][W]`` row-major;
* the main field B0 lies in the slice plane along y (the rows axis);
* susceptibility chi and the normalised field f = dB/B0 are both in ppm;
* the mask is ``uint8`` 0/1 and is used as both the data weighting W and the
  gradient mask M of Eq. (1).

Field model.  Each slice is treated as the cross-section of an object that
is uniform along z (perpendicular to the slice).  The field of such an
object, with B0 along y, is the convolution of chi with the 2-D dipole
Green's function

    g(x, y) = -delta(x, y) / 6 + PV (y^2 - x^2) / (2 pi (x^2 + y^2)^2),

the -1/6 term being the Lorentz-corrected self field of a long cylinder
magnetised across its axis.  ``dipole_green_2d`` integrates g exactly over
each pixel (the principal value over the centre pixel is zero by the x<->y
antisymmetry of the integrand) and ``simulate_field`` applies it as a linear,
non-periodic convolution.  A uniform disc of radius a then has the textbook
field -chi/6 inside and (chi/2)(a/r)^2 cos(2 phi) outside, phi measured from
B0; ``tests/test_phantoms.py`` checks both.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy import fft as sfft
from scipy import ndimage


# --------------------------------------------------------------------------- field model


def dipole_green_2d(H: int, W: int) -> np.ndarray:
    """Pixel-integrated 2-D dipole Green's function for offsets |dy|<H, |dx|<W.

    Returns a float64 array of shape (2H-1, 2W-1); entry [dy+H-1, dx+W-1] is
    the field at offset (dy, dx) from a unit-susceptibility pixel.

    The off-centre integral uses d/dx [x/(x^2+y^2)] = (y^2-x^2)/(x^2+y^2)^2,
    so the integral over [x0,x1]x[y0,y1] equals
    atan(y1/x1) - atan(y0/x1) - atan(y1/x0) + atan(y0/x0); x0, x1 are
    half-integers and never zero.
    """
    dy = np.arange(-(H - 1), H, dtype=np.float64)[:, None]
    dx = np.arange(-(W - 1), W, dtype=np.float64)[None, :]
    x0, x1 = dx - 0.5, dx + 0.5
    y0, y1 = dy - 0.5, dy + 0.5
    g = (np.arctan(y1 / x1) - np.arctan(y0 / x1) - np.arctan(y1 / x0) + np.arctan(y0 / x0)) / (
        2.0 * math.pi
    )
    g[H - 1, W - 1] = -1.0 / 6.0  # Lorentz-corrected self term; PV part is 0
    return g


def simulate_field(chi: np.ndarray, chunk: int = 16) -> np.ndarray:
    """Noise-free field (ppm, float64) of a chi stack [S][H][W] (ppm).

    Linear convolution with ``dipole_green_2d`` (every pixel of the slice
    sees every other pixel; nothing wraps around), done with zero-padded
    FFTs of size 2H x 2W: the full linear result spans indices 0..3H-3, and
    with period 2H >= 2H-1 no alias lands in the kept window H-1..2H-2.
    """
    chi = np.asarray(chi, dtype=np.float64)
    squeeze = chi.ndim == 2
    if squeeze:
        chi = chi[None]
    S, H, W = chi.shape
    shape = (2 * H, 2 * W)
    G = sfft.rfft2(dipole_green_2d(H, W), s=shape, workers=-1)
    out = np.empty((S, H, W), dtype=np.float64)
    for s0 in range(0, S, chunk):
        F = sfft.rfft2(chi[s0 : s0 + chunk], s=shape, axes=(1, 2), workers=-1)
        full = sfft.irfft2(F * G, s=shape, axes=(1, 2), workers=-1)
        out[s0 : s0 + chunk] = full[:, H - 1 : 2 * H - 1, W - 1 : 2 * W - 1]
    return out[0] if squeeze else out


# --------------------------------------------------------------------------- shapes


def ellipse_mask(H: int, W: int, ax: float = 0.45, ay: float = 0.35) -> np.ndarray:
    """Centred elliptical mask (uint8) with semi-axes ax*W along x, ay*H along y."""
    y = np.arange(H, dtype=np.float64)[:, None] - (H - 1) / 2.0
    x = np.arange(W, dtype=np.float64)[None, :] - (W - 1) / 2.0
    return (((x / (ax * W)) ** 2 + (y / (ay * H)) ** 2) <= 1.0).astype(np.uint8)


def disc(H: int, W: int, ci: float, cj: float, r: float) -> np.ndarray:
    """Boolean disc by the pixel-centre rule (i-ci)^2 + (j-cj)^2 <= r^2."""
    i = np.arange(H, dtype=np.float64)[:, None]
    j = np.arange(W, dtype=np.float64)[None, :]
    return (i - ci) ** 2 + (j - cj) ** 2 <= r * r


def rod(H: int, W: int, ci: float, cj: float, length: float, angle: float, half_width: float = 1.0):
    """Boolean in-plane rod: pixel centres within ``half_width`` of a segment.

    The segment is centred at (ci, cj), has the given length and makes
    ``angle`` (radians) with the x axis.
    """
    i = np.arange(H, dtype=np.float64)[:, None]
    j = np.arange(W, dtype=np.float64)[None, :]
    ux, uy = math.cos(angle), math.sin(angle)
    rx, ry = j - cj, i - ci
    t = np.clip(rx * ux + ry * uy, -length / 2.0, length / 2.0)
    dx, dy = rx - t * ux, ry - t * uy
    return dx * dx + dy * dy <= half_width * half_width


# --------------------------------------------------------------------------- problems


@dataclasses.dataclass
class SliceProblem:
    """A stack of independent slice problems sharing (H, W), lambda and N."""

    name: str
    field: np.ndarray  # float32 [S][H][W], ppm
    mask: np.ndarray  # uint8 [S][H][W]
    chi_true: np.ndarray  # float32 [S][H][W], ppm
    lam: float
    n_iter: int

    @property
    def shape(self):
        return self.field.shape

    @property
    def voxels(self) -> int:
        return int(np.prod(self.field.shape))


def config1() -> SliceProblem:
    """One 64x64 slice: two discs (r=2 px, 180 ppm), one 2x20 px rod (150 ppm).

    Full mask, noise 0.01 ppm (seed 0), lambda = 1e-3, 300 iterations.
    """
    H = W = 64
    chi = np.zeros((H, W), dtype=np.float64)
    chi[disc(H, W, 20, 20, 2.0)] = 180.0
    chi[disc(H, W, 44, 24, 2.0)] = 180.0
    chi[40:42, 34:54] = 150.0  # rod across B0 (rows 40-41, cols 34-53)
    rng = np.random.default_rng(0)
    field = simulate_field(chi) + rng.normal(0.0, 0.01, size=(H, W))
    return SliceProblem(
        name="cfg1-64x64x1",
        field=field[None].astype(np.float32),
        mask=np.ones((1, H, W), dtype=np.uint8),
        chi_true=chi[None].astype(np.float32),
        lam=1e-3,
        n_iter=300,
    )


def _inside_ellipse_point(rng, H, W, ax=0.45, ay=0.35, margin=0.85):
    """Uniform point inside a slightly shrunk copy of the mask ellipse."""
    while True:
        u, v = rng.uniform(-1.0, 1.0, size=2)
        if u * u + v * v <= 1.0:
            return (H - 1) / 2.0 + v * margin * ay * H, (W - 1) / 2.0 + u * margin * ax * W


def volume(
    H: int,
    W: int,
    S: int,
    seed: int,
    lam: float = 5e-4,
    n_iter: int = 500,
    n_objects: int = 6,
    noise_std: float = 0.02,
    tissue_std: float = 0.5,
    name: str | None = None,
) -> SliceProblem:
    """A brachytherapy-style volume: seeds and needles in smooth tissue.

    Random draws, all from ``numpy.random.default_rng(seed)`` in this order:
    tissue white noise [S][H][W]; then per object: type (seed or needle,
    probability 1/2 each), chi ~ U[120, 200] ppm, centre uniform inside the
    mask ellipse, and for a seed its first slice (a disc of radius 2 px over
    3 consecutive slices), for a needle its length U[20, 60] px, in-plane
    angle U[0, pi), slice run U{8..64} and first slice; finally the field
    noise N(0, noise_std) [S][H][W].  Tissue = white noise low-passed by a
    Gaussian (sigma 4, 4, 1 px along x, y, slice), rescaled to zero mean and
    ``tissue_std`` inside the elliptical mask, zero outside.
    """
    rng = np.random.default_rng(seed)
    mask2 = ellipse_mask(H, W)
    m = mask2.astype(bool)
    tissue = ndimage.gaussian_filter(rng.standard_normal((S, H, W)), sigma=(1.0, 4.0, 4.0))
    inside = tissue[:, m]
    tissue = (tissue - inside.mean()) * (tissue_std / max(inside.std(), 1e-30))
    chi = tissue * mask2[None]
    for _ in range(n_objects):
        is_seed = rng.random() < 0.5
        value = rng.uniform(120.0, 200.0)
        ci, cj = _inside_ellipse_point(rng, H, W)
        if is_seed:
            run = min(3, S)
            s0 = int(rng.integers(0, S - run + 1))
            shape = disc(H, W, ci, cj, 2.0)
        else:
            length = rng.uniform(20.0, 60.0)
            angle = rng.uniform(0.0, math.pi)
            run = min(int(rng.integers(8, 65)), S)
            s0 = int(rng.integers(0, S - run + 1))
            shape = rod(H, W, ci, cj, length, angle)
        chi[s0 : s0 + run][:, shape] = value
    field = simulate_field(chi) + rng.normal(0.0, noise_std, size=(S, H, W))
    return SliceProblem(
        name=name or f"vol-{H}x{W}x{S}-seed{seed}",
        field=field.astype(np.float32),
        mask=np.ascontiguousarray(np.broadcast_to(mask2, (S, H, W)), dtype=np.uint8),
        chi_true=chi.astype(np.float32),
        lam=lam,
        n_iter=n_iter,
    )


def magnitude_weight(mask: np.ndarray, seed: int, floor: float = 0.2) -> np.ndarray:
    """A magnitude-like data weighting W in [floor, 1] inside the mask, 0 outside.

    Smooth image intensity stand-in (the paper's W comes from the scanner
    magnitude, which is not available): white noise from
    ``default_rng(seed)`` low-passed by a Gaussian (sigma 6 px in-plane, 1
    slice), mapped linearly onto [floor, 1] over the mask, times the mask.
    float32 [S][H][W].
    """
    rng = np.random.default_rng(seed)
    m = np.asarray(mask) != 0
    sm = ndimage.gaussian_filter(rng.standard_normal(m.shape), sigma=(1.0, 6.0, 6.0))
    lo, hi = sm[m].min(), sm[m].max()
    w = floor + (1.0 - floor) * (sm - lo) / max(hi - lo, 1e-30)
    return np.ascontiguousarray(np.where(m, w, 0.0), dtype=np.float32)


def echo_pair(field_ppm: np.ndarray, mask: np.ndarray, seed: int, b0_tesla: float = 3.0,
              t_shift_s: float = 0.6e-3, noise: float = 0.002):
    """Two complex acquisitions (without and with the readout shift) of a local field.

    Forward model of the acquisition only: magnitude = a smooth image in
    [0.2, 1] inside the mask and 0.02 outside (``magnitude_weight`` recipe),
    a smooth receiver phase phi0 common to both, and the shifted one accrues
    2 pi gamma_bar B0 T_shift dB (gamma_bar = 42.577478518 MHz/T, dB in ppm);
    complex Gaussian noise of standard deviation ``noise`` on each.  Draws
    from ``default_rng(seed)``.  Returns (s0, s1) complex64 [S][H][W].
    """
    rng = np.random.default_rng(seed)
    mag = magnitude_weight(mask, seed + 1).astype(np.float64)
    mag = np.where(np.asarray(mask) != 0, mag, 0.02)
    phi0 = ndimage.gaussian_filter(rng.standard_normal(mag.shape), sigma=(1.0, 8.0, 8.0))
    phi0 *= math.pi / max(float(np.abs(phi0).max()), 1e-30)
    rad_per_ppm = 2.0 * math.pi * 42.577478518e6 * b0_tesla * t_shift_s * 1e-6
    s0 = mag * np.exp(1j * phi0)
    s1 = s0 * np.exp(1j * rad_per_ppm * np.asarray(field_ppm, dtype=np.float64))
    shape = mag.shape
    s0 = s0 + noise * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))
    s1 = s1 + noise * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))
    return s0.astype(np.complex64), s1.astype(np.complex64)


def config2(S: int = 64) -> SliceProblem:
    """256x256x64 volume, six seeds/needles, lambda = 5e-4, 500 iterations, seed 0."""
    return volume(256, 256, S, seed=0, lam=5e-4, n_iter=500, name=f"cfg2-256x256x{S}")


CONFIG4_SIZES = (128, 192, 256, 384, 512)
CONFIG4_LAMBDAS = (2e-4, 5e-4, 1e-3)


def config4_volumes(n_volumes: int = 48):
    """Specs of the uneven batch: (idx, size, slices, lambda, seed), 400 iterations.

    Volume idx draws size, slice count U{16..96} and lambda from
    ``default_rng(1000 + idx)``; its content is ``volume(..., seed=1000+idx)``.
    """
    specs = []
    for idx in range(n_volumes):
        rng = np.random.default_rng(1000 + idx)
        size = int(rng.choice(CONFIG4_SIZES))
        S = int(rng.integers(16, 97))
        lam = float(rng.choice(CONFIG4_LAMBDAS))
        specs.append(dict(idx=idx, size=size, slices=S, lam=lam, seed=1000 + idx, n_iter=400))
    return specs


def config5_arrivals(n_requests: int = 400, rate_hz: float = 40.0, seed: int = 0):
    """Poisson arrival times (s) and uneven-batch-style volume specs for serving.

    Exponential inter-arrival gaps of mean 1/rate_hz from ``default_rng(seed)``;
    request k carries the spec of ``config4_volumes`` drawn with seed 5000+k.
    """
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, size=n_requests))
    reqs = []
    for k in range(n_requests):
        r = np.random.default_rng(5000 + k)
        size = int(r.choice(CONFIG4_SIZES))
        S = int(r.integers(16, 97))
        lam = float(r.choice(CONFIG4_LAMBDAS))
        reqs.append(dict(idx=k, t=float(t[k]), size=size, slices=S, lam=lam, seed=5000 + k, n_iter=400))
    return reqs
