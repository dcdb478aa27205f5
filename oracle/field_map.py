"""FP64 CPU oracle for the field-map preprocessing (Sec. II.B step (1)).

TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it.  It shares no code with the CUDA path.

Sec. II (acquisition) and Sec. II.B step (1): two 3-D acquisitions, one with
its readouts shifted by a small time T_shift (0.2-0.7 ms; 0.6 ms in the
experiments, at 3 T), and the preprocessing turns them into the local field
dB, the weighting W and the mask that Eq. (1) takes.  The paper names these
outputs but gives no formula; the readings taken here:

* the phase accrued over T_shift is the angle of S1 conj(S0) (the wrapped
  phase difference, in (-pi, pi]; no unwrapping -- the short shift is what
  keeps the phase small), and dB in ppm = that angle / (2 pi gamma_bar B0
  T_shift) * 1e6 with gamma_bar = 42.577478518 MHz/T;
* W = |S0| / max |S0| over the volume (magnitude weighting, values in [0, 1]);
* Mask: |S0|^2 >= t^2 max |S0|^2 for a relative threshold t, decided in
  FP64 from the acquisitions' values (exact squares of float32 inputs up to
  one FP64 rounding).  A float32 implementation can decide the other way only
  for voxels whose |S0|^2 lies within float32 rounding of t^2 max |S0|^2;
  ``mask_boundary_band`` marks those voxels.

The field is set to zero outside the mask.
"""

from __future__ import annotations

import math

import numpy as np

GAMMA_BAR_HZ_PER_T = 42.577478518e6


def ppm_per_radian(b0_tesla: float, t_shift_s: float) -> float:
    """Field (ppm) per radian of phase accrued over t_shift."""
    return 1e6 / (2.0 * math.pi * GAMMA_BAR_HZ_PER_T * b0_tesla * t_shift_s)


def mag2(s: np.ndarray) -> np.ndarray:
    """|s|^2 = re^2 + im^2 in FP64."""
    z = np.asarray(s).astype(np.complex128)
    return z.real * z.real + z.imag * z.imag


def mask_boundary_band(s0: np.ndarray, threshold: float, rel: float = 8 * 2.0**-24) -> np.ndarray:
    """Voxels whose mask decision is within ``rel`` (relative) of the threshold: |S0|^2 and
    t^2 max |S0|^2 closer than rel * (|S0|^2 + t^2 max |S0|^2).  Outside this band a float32
    evaluation (a few roundings of relative size 2^-24 each) decides as the FP64 one does."""
    m2 = mag2(s0)
    lim = threshold * threshold * (float(m2.max()) if m2.size else 0.0)
    return np.abs(m2 - lim) <= rel * (m2 + lim)


def field_map(s0: np.ndarray, s1: np.ndarray, t_shift_s: float, b0_tesla: float, threshold: float):
    """(field ppm float64, weight float64, mask uint8) from the two complex acquisitions."""
    s0 = np.asarray(s0)
    s1 = np.asarray(s1)
    m2 = mag2(s0)
    max2 = float(m2.max()) if m2.size else 0.0
    mask = (m2 >= threshold * threshold * max2).astype(np.uint8)
    z = s1.astype(np.complex128) * np.conj(s0.astype(np.complex128))
    field = np.angle(z) * ppm_per_radian(b0_tesla, t_shift_s)
    field = np.where(mask != 0, field, 0.0)
    mag = np.abs(s0.astype(np.complex128))
    mmax = float(mag.max()) if mag.size else 0.0
    weight = mag / mmax if mmax > 0 else np.zeros_like(mag)
    return field, weight, mask
