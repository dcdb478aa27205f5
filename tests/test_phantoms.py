"""The seeded input generator: determinism, shapes, and its physical field model.

The field model (pixel-integrated 2-D dipole Green's function, linear
convolution) is pinned against the long-cylinder closed form and against a
direct double sum on a tiny slice.
"""

import math

import numpy as np
import pytest

import phantoms as P


def test_green_function_direct_sum_tiny():
    rng = np.random.default_rng(0)
    H, W = 5, 7
    chi = rng.standard_normal((H, W))
    g = P.dipole_green_2d(H, W)
    ref = np.zeros((H, W))
    for i in range(H):
        for j in range(W):
            for a in range(H):
                for b in range(W):
                    ref[i, j] += chi[a, b] * g[i - a + H - 1, j - b + W - 1]
    assert np.allclose(P.simulate_field(chi), ref, atol=1e-12)


def test_green_function_far_field_and_symmetry():
    g = P.dipole_green_2d(40, 40)
    c = 39
    # far from the source the pixel integral tends to cos(2 phi) / (2 pi r^2)
    assert g[c + 30, c] == pytest.approx(1.0 / (2 * math.pi * 900), rel=1e-3)
    assert g[c, c + 30] == pytest.approx(-1.0 / (2 * math.pi * 900), rel=1e-3)
    assert abs(g[c + 10, c + 10]) < 1e-15  # 45 degrees: cos(2 phi) = 0
    assert np.allclose(g, g[::-1, :]) and np.allclose(g, g[:, ::-1])
    assert g[c, c] == -1.0 / 6.0


def test_disc_field_matches_cylinder_closed_form():
    N, a = 256, 10
    chi = np.zeros((N, N))
    c = N // 2
    chi[P.disc(N, N, c, c, a)] = 1.0
    f = P.simulate_field(chi)
    a_eff = math.sqrt(chi.sum() / math.pi)
    assert f[c, c] == pytest.approx(-1.0 / 6.0, abs=2e-3)
    for r in (30, 50, 80):
        expect = 0.5 * (a_eff / r) ** 2
        assert f[c + r, c] == pytest.approx(expect, rel=1e-2)  # along B0 (rows)
        assert f[c, c + r] == pytest.approx(-expect, rel=1e-2)


def test_config1_recipe():
    pb = P.config1()
    assert pb.field.shape == (1, 64, 64) and pb.field.dtype == np.float32
    assert pb.mask.dtype == np.uint8 and pb.mask.min() == 1
    assert pb.chi_true.max() == 180.0 and (pb.chi_true == 150.0).sum() == 40
    assert pb.lam == 1e-3 and pb.n_iter == 300
    again = P.config1()
    assert np.array_equal(pb.field, again.field)


def test_volume_recipe_deterministic_and_masked():
    v1 = P.volume(64, 64, 8, seed=3, n_iter=10)
    v2 = P.volume(64, 64, 8, seed=3, n_iter=10)
    assert np.array_equal(v1.field, v2.field) and np.array_equal(v1.chi_true, v2.chi_true)
    v3 = P.volume(64, 64, 8, seed=4, n_iter=10)
    assert not np.array_equal(v1.field, v3.field)
    m = v1.mask[0].astype(bool)
    tissue = np.where(v1.chi_true < 100, v1.chi_true, 0)
    assert np.all(tissue[:, ~m] == 0)
    assert 0.3 < tissue[:, m].std() < 0.7
    assert v1.chi_true.max() >= 120.0


def test_ellipse_mask_axes():
    m = P.ellipse_mask(256, 256)
    rows = np.nonzero(m[:, 128])[0]
    cols = np.nonzero(m[128, :])[0]
    assert abs(len(rows) - 2 * 0.35 * 256) <= 2
    assert abs(len(cols) - 2 * 0.45 * 256) <= 2


def test_config4_and_config5_specs():
    specs = P.config4_volumes()
    assert len(specs) == 48
    assert {s["size"] for s in specs} <= set(P.generator.CONFIG4_SIZES)
    assert all(16 <= s["slices"] <= 96 and s["n_iter"] == 400 for s in specs)
    reqs = P.config5_arrivals(50)
    t = [r["t"] for r in reqs]
    assert all(b > a for a, b in zip(t, t[1:]))
    assert 0.5 < t[-1] / (50 / 40.0) < 2.0
