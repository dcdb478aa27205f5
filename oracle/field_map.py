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
* Mask: |S0|^2 >= t^2 max |S0|^2 for a relative threshold t.  This decision
  sets a 0/1 value, so it is taken in float32 with a fixed operation order
  (re*re + im*im, each product and the sum rounded to float32; the threshold
  t^2 rounded to float32 once; their product rounded to float32), the same
  arithmetic the GPU kernel uses.

The field is set to zero outside the mask.
"""

from __future__ import annotations

import math

import numpy as np

GAMMA_BAR_HZ_PER_T = 42.577478518e6


def ppm_per_radian(b0_tesla: float, t_shift_s: float) -> float:
    """Field (ppm) per radian of phase accrued over t_shift."""
    return 1e6 / (2.0 * math.pi * GAMMA_BAR_HZ_PER_T * b0_tesla * t_shift_s)


def mag2_f32(s: np.ndarray) -> np.ndarray:
    """|s|^2 in float32: re*re + im*im, every operation rounded to float32."""
    re = np.ascontiguousarray(s.real, dtype=np.float32)
    im = np.ascontiguousarray(s.imag, dtype=np.float32)
    return (re * re) + (im * im)


def field_map(s0: np.ndarray, s1: np.ndarray, t_shift_s: float, b0_tesla: float, threshold: float):
    """(field ppm float64, weight float64, mask uint8) from the two complex acquisitions."""
    s0 = np.asarray(s0)
    s1 = np.asarray(s1)
    m2 = mag2_f32(s0)
    max2 = np.float32(m2.max()) if m2.size else np.float32(0)
    thr2 = np.float32(threshold * threshold)
    mask = (m2 >= np.float32(thr2 * max2)).astype(np.uint8)
    z = s1.astype(np.complex128) * np.conj(s0.astype(np.complex128))
    field = np.angle(z) * ppm_per_radian(b0_tesla, t_shift_s)
    field = np.where(mask != 0, field, 0.0)
    mag = np.abs(s0.astype(np.complex128))
    mmax = float(mag.max()) if mag.size else 0.0
    weight = mag / mmax if mmax > 0 else np.zeros_like(mag)
    return field, weight, mask
