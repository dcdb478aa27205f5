"""Pins of the field-map oracle (``oracle/field_map.py``) to things other than itself."""

import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import field_map as FM


def test_ppm_per_radian_constant_by_hand():
    # 1 ppm at 3 T is 42.577478518 MHz/T * 3 T * 1e-6 = 127.732435554 Hz; over 0.6 ms that is
    # 2 pi * 127.732435554 * 0.0006 = 0.481540 rad, so one radian is 2.07667 ppm
    rad_per_ppm = 2.0 * math.pi * 127.732435554 * 0.0006
    assert rad_per_ppm == pytest.approx(0.4815399, abs=1e-7)
    assert FM.ppm_per_radian(3.0, 0.6e-3) == pytest.approx(1.0 / rad_per_ppm, rel=1e-12)


def _echoes(f_ppm, mag, phi0, b0=3.0, t=0.6e-3):
    kappa = 1.0 / FM.ppm_per_radian(b0, t)  # rad per ppm (pinned above)
    s0 = mag * np.exp(1j * phi0)
    s1 = s0 * np.exp(1j * kappa * f_ppm)
    return s0, s1


def test_noise_free_field_is_recovered_exactly_inside_the_wrap():
    rng = np.random.default_rng(0)
    shape = (3, 8, 10)
    f = rng.uniform(-6.0, 6.0, shape)  # |phase| <= 6 * 0.4815 < pi
    mag = rng.uniform(0.5, 2.0, shape)
    phi0 = rng.uniform(-np.pi, np.pi, shape)
    s0, s1 = _echoes(f, mag, phi0)
    field, weight, mask = FM.field_map(s0, s1, 0.6e-3, 3.0, 0.1)
    assert mask.all()
    assert np.allclose(field, f, rtol=0, atol=1e-12)


def test_wrap_beyond_pi():
    kappa = 1.0 / FM.ppm_per_radian(3.0, 0.6e-3)
    f = np.array([[[(np.pi + 0.2) / kappa, (-np.pi - 0.3) / kappa]]])
    s0, s1 = _echoes(f, np.ones_like(f), np.zeros_like(f))
    field, _, _ = FM.field_map(s0, s1, 0.6e-3, 3.0, 0.0)
    assert field[0, 0, 0] == pytest.approx((-np.pi + 0.2) / kappa, abs=1e-12)
    assert field[0, 0, 1] == pytest.approx((np.pi - 0.3) / kappa, abs=1e-12)


def test_weight_and_mask_invariants():
    rng = np.random.default_rng(1)
    shape = (2, 6, 7)
    s0 = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)
    s1 = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)
    _, w, m0 = FM.field_map(s0, s1, 0.6e-3, 3.0, 0.0)
    assert m0.all()  # threshold 0 keeps every voxel
    assert w.max() == pytest.approx(1.0, abs=0) and w.min() >= 0.0
    k = np.unravel_index(np.argmax(np.abs(s0)), shape)
    assert w[k] == 1.0
    assert np.allclose(w, np.abs(s0.astype(np.complex128)) / np.abs(s0.astype(np.complex128)).max(), atol=1e-15)
    prev = m0.sum()
    for t in (0.2, 0.4, 0.6, 0.8):
        field, _, m = FM.field_map(s0, s1, 0.6e-3, 3.0, t)
        assert m.sum() <= prev and np.all(m <= m0)
        assert np.all(field[m == 0] == 0.0)
        prev = m.sum()
    _, _, m_none = FM.field_map(s0, s1, 0.6e-3, 3.0, 1.5)
    assert not m_none.any()


def test_mask_decision_at_the_boundary_by_exact_arithmetic():
    # max |s|^2 = 1 and threshold 0.5: a voxel is kept iff |s|^2 >= 1/4, decided here by exact
    # rational arithmetic on the float32 inputs.  The last voxel lies 3.7e-9 below 1/4, which a
    # float32 evaluation rounds up to 1/4 (and keeps): the oracle must decide exactly.
    re_last = np.float32(0.5 - 2.0**-25)
    im_last = np.float32(1.653e-4)
    s0 = np.array([[[1.0 + 0j, 0.3 + 0.4j, 0.5 + 0j, 0.49 + 0j, complex(re_last, im_last)]]], dtype=np.complex64)
    want = []
    for z in s0.ravel():
        m2 = Fraction(float(z.real)) ** 2 + Fraction(float(z.imag)) ** 2
        want.append(1 if m2 >= Fraction(1, 4) else 0)
    assert want == [1, 1, 1, 0, 0]
    f32 = np.float32(re_last) * np.float32(re_last) + np.float32(im_last) * np.float32(im_last)
    assert f32 == np.float32(0.25)  # the float32 evaluation sits on the threshold
    _, _, m = FM.field_map(s0, s0, 0.6e-3, 3.0, 0.5)
    assert m.ravel().tolist() == want
    band = FM.mask_boundary_band(s0, 0.5)
    assert band.ravel().tolist() == [False, True, True, False, True]  # 0.3+0.4i: 4.8e-8 above 1/4


def test_scaling_both_acquisitions_changes_nothing():
    rng = np.random.default_rng(2)
    shape = (2, 5, 6)
    s0 = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)
    s1 = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)
    a = FM.field_map(s0, s1, 0.6e-3, 3.0, 0.3)
    b = FM.field_map(s0 * 4, s1 * 4, 0.6e-3, 3.0, 0.3)  # power of two: float32 products stay exact
    for x, y in zip(a, b):
        assert np.array_equal(x, y) or np.allclose(x, y, rtol=1e-15, atol=0)
