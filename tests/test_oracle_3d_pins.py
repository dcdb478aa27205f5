"""Pins of the 3-D oracle (``oracle/pd_oracle_3d.py``) to things other than itself.

* G (3-D) and G^T against explicit difference matrices built by hand;
* D (3-D) against an explicit-DFT dense matrix, and on a z-invariant field
  against its closed form (only kz = 0 survives, where D = 1/3 off DC);
* the whole iteration on tiny volumes against an independent dense-matrix
  implementation of the pseudocode (both TV readings, binary and weighted W);
* ||K|| against the dense spectral norm;
* a KKT certificate: gap and stationarity vanish as the iteration converges;
* planted mistakes in the oracle's building blocks fail the dense pin.
"""

import itertools

import numpy as np
import pytest

from oracle import pd_oracle as O
from oracle import pd_oracle_3d as O3


def freq(k, n):
    """Signed frequency in cycles per sample of DFT index k of length n."""
    return k / n if k < (n + 1) // 2 else (k - n) / n


def dense_D3(S, H, W, voxel=(1.0, 1.0, 1.0)):
    """F^-1 diag(D) F for the 3-D dipole kernel with B0 along z, built with exp() and the
    formula 1/3 - kz^2/|k|^2 written out here (no numpy.fft, no oracle kernel); k_i is the
    frequency in cycles per sample over the voxel edge along axis i."""
    N = S * H * W
    idx = list(itertools.product(range(S), range(H), range(W)))
    F = np.empty((N, N), complex)
    d = np.empty(N)
    for r, (kz, ky, kx) in enumerate(idx):
        fz, fy, fx = freq(kz, S) / voxel[0], freq(ky, H) / voxel[1], freq(kx, W) / voxel[2]
        k2 = fz * fz + fy * fy + fx * fx
        d[r] = 0.0 if k2 == 0 else 1.0 / 3.0 - fz * fz / k2
        for c, (z, y, x) in enumerate(idx):
            F[r, c] = np.exp(-2j * np.pi * (kz * z / S + ky * y / H + kx * x / W))
    return (F.conj().T @ np.diag(d) @ F).real / N


def dense_grad3(S, H, W):
    """Forward differences with a Neumann boundary as explicit matrices (row-major z, y, x)."""
    def d1(n):
        M = np.zeros((n, n))
        for i in range(n - 1):
            M[i, i], M[i, i + 1] = -1.0, 1.0
        return M

    I = np.eye
    Gx = np.kron(np.kron(I(S), I(H)), d1(W))
    Gy = np.kron(np.kron(I(S), d1(H)), I(W))
    Gz = np.kron(np.kron(d1(S), I(H)), I(W))
    return Gx, Gy, Gz


def dense_pd(f, m, w, lam, tau, sigma, n_iter, tv, voxel=(1.0, 1.0, 1.0)):
    """The Sec. II.A pseudocode with explicit matrices on the flattened volume."""
    S, H, W = f.shape
    D = dense_D3(S, H, W, voxel)
    Gx, Gy, Gz = dense_grad3(S, H, W)
    fv, mv, wv = f.ravel(), m.ravel().astype(float), w.ravel()
    n = fv.size
    chi = np.zeros(n)
    cb = np.zeros(n)
    p = np.zeros(n)
    q = [np.zeros(n) for _ in range(3)]
    for _ in range(n_iter):
        p = (p + sigma * (wv * (D @ cb) - wv * fv)) / (1.0 + sigma / lam)
        v = [q[a] + sigma * mv * (G @ cb) for a, G in enumerate((Gx, Gy, Gz))]
        if tv == "iso":
            nrm = np.maximum(1.0, np.sqrt(v[0] ** 2 + v[1] ** 2 + v[2] ** 2))
            q = [va / nrm for va in v]
        else:
            q = [np.minimum(1.0, np.maximum(-1.0, va)) for va in v]
        new = chi - tau * (D @ (wv * p)) - tau * (Gx.T @ (mv * q[0]) + Gy.T @ (mv * q[1]) + Gz.T @ (mv * q[2]))
        cb = 2.0 * new - chi
        chi = new
    return chi.reshape(f.shape)


def test_grad3_and_adjoint_match_dense():
    rng = np.random.default_rng(0)
    S, H, W = 3, 4, 5
    x = rng.standard_normal((S, H, W))
    Gx, Gy, Gz = dense_grad3(S, H, W)
    gx, gy, gz = O3.grad3(x)
    for g, G in ((gx, Gx), (gy, Gy), (gz, Gz)):
        assert np.allclose(g.ravel(), G @ x.ravel(), atol=1e-14)
    a, b, c = (rng.standard_normal((S, H, W)) for _ in range(3))
    ref = Gx.T @ a.ravel() + Gy.T @ b.ravel() + Gz.T @ c.ravel()
    assert np.allclose(O3.grad3_adjoint(a, b, c).ravel(), ref, atol=1e-14)


@pytest.mark.parametrize("shape", [(2, 3, 4), (4, 3, 2), (3, 4, 4)])
def test_D3_matches_dense_dft(shape):
    x = np.random.default_rng(1).standard_normal(shape)
    D = dense_D3(*shape)
    got = O.apply_D_3d(x, O.dipole_kernel_3d(shape, b0_axis=0))
    assert np.allclose(got.ravel(), D @ x.ravel(), atol=1e-13)


def test_anisotropic_voxel_kernel_hand_fractions():
    # (4, 6, 8) grid, voxel 2 x 1 x 1: kz = fz / 2.  Index (1, 0, 1): kz = kx = 1/8 -> 1/3 - 1/2;
    # (1, 1, 0): kz = 1/8, ky = 1/6 -> 1/3 - (1/64) / (1/64 + 1/36) = 1/3 - 9/25 = -2/75;
    # (2, 0, 2): kz = -1/4, kx = 1/4 -> -1/6; single axes as in the isotropic kernel
    D = O.dipole_kernel_3d((4, 6, 8), b0_axis=0, voxel=(2.0, 1.0, 1.0))
    assert D[1, 0, 1] == pytest.approx(-1.0 / 6.0, abs=1e-15)
    assert D[1, 1, 0] == pytest.approx(-2.0 / 75.0, abs=1e-15)
    assert D[2, 0, 2] == pytest.approx(-1.0 / 6.0, abs=1e-15)
    assert D[1, 0, 0] == pytest.approx(-2.0 / 3.0, abs=1e-15)
    assert D[0, 1, 0] == pytest.approx(1.0 / 3.0, abs=1e-15) and D[0, 0, 0] == 0.0
    # the isotropic kernel at the same index differs: kz = kx = 1/4 and 1/8 -> 1/3 - 0.8
    assert O.dipole_kernel_3d((4, 6, 8))[1, 0, 1] == pytest.approx(1.0 / 3.0 - 0.8, abs=1e-15)


def test_voxel_scale_invariance():
    # only the ratios of the voxel edges matter; unit voxels are the isotropic kernel
    iso = O.dipole_kernel_3d((5, 6, 4))
    assert np.array_equal(O.dipole_kernel_3d((5, 6, 4), voxel=(1.0, 1.0, 1.0)), iso)
    assert np.array_equal(O.dipole_kernel_3d((5, 6, 4), voxel=(2.0, 2.0, 2.0)), iso)
    a = O.dipole_kernel_3d((5, 6, 4), voxel=(2.0, 0.72, 0.72))
    b = O.dipole_kernel_3d((5, 6, 4), voxel=(4.0, 1.44, 1.44))
    assert np.allclose(a, b, rtol=0, atol=1e-15)


@pytest.mark.parametrize("voxel", [(2.0, 0.72, 0.72), (1.0, 3.0, 0.5)])
def test_D3_anisotropic_matches_dense_dft(voxel):
    shape = (3, 4, 4)
    x = np.random.default_rng(4).standard_normal(shape)
    got = O.apply_D_3d(x, O.dipole_kernel_3d(shape, b0_axis=0, voxel=voxel))
    assert np.allclose(got.ravel(), dense_D3(*shape, voxel) @ x.ravel(), atol=1e-13)


def test_D3_of_z_invariant_field_is_a_third_of_the_deviation():
    # only kz = 0 is present, where D = 1/3 - 0 = 1/3 except at DC (D = 0)
    g = np.random.default_rng(2).standard_normal((8, 6))
    x = np.broadcast_to(g, (5, 8, 6)).copy()
    got = O.apply_D_3d(x, O.dipole_kernel_3d(x.shape, b0_axis=0))
    assert np.allclose(got, (x - g.mean()) / 3.0, atol=1e-14)


@pytest.mark.parametrize("tv", ["aniso", "iso"])
@pytest.mark.parametrize("weighted", [False, True])
def test_whole_iteration_matches_dense_pseudocode(tv, weighted):
    rng = np.random.default_rng(3)
    S, H, W = 3, 4, 4
    f = rng.standard_normal((S, H, W))
    m = (rng.random((S, H, W)) > 0.25).astype(np.uint8)
    w = m * rng.uniform(0.2, 1.0, (S, H, W)) if weighted else m.astype(float)
    lam, tau, sigma, n = 5.0, 0.28, 0.28, 25
    got = O3.pd_solve_3d(f, m, lam, tau, sigma, n, weight=w if weighted else None, tv=tv)
    ref = dense_pd(f, m, w, lam, tau, sigma, n, tv)
    assert np.allclose(got, ref, rtol=0, atol=1e-12 * max(1.0, np.abs(ref).max()))
    assert np.abs(ref).max() > 1e-3  # the iteration moved


def test_whole_iteration_anisotropic_voxel_matches_dense_pseudocode():
    rng = np.random.default_rng(5)
    S, H, W = 3, 4, 4
    f = rng.standard_normal((S, H, W))
    m = (rng.random((S, H, W)) > 0.25).astype(np.uint8)
    vox = (2.0, 0.72, 0.72)
    got = O3.pd_solve_3d(f, m, 5.0, 0.28, 0.28, 25, voxel=vox)
    ref = dense_pd(f, m, m.astype(float), 5.0, 0.28, 0.28, 25, "aniso", vox)
    assert np.allclose(got, ref, rtol=0, atol=1e-12 * max(1.0, np.abs(ref).max()))
    iso = O3.pd_solve_3d(f, m, 5.0, 0.28, 0.28, 25)
    assert np.abs(got - iso).max() > 1e-3  # the voxel shape changes the result


def test_opnorm3_matches_dense_spectral_norm():
    rng = np.random.default_rng(4)
    S, H, W = 2, 4, 4
    m = (rng.random((S, H, W)) > 0.3).astype(np.uint8)
    D = dense_D3(S, H, W)
    Gx, Gy, Gz = dense_grad3(S, H, W)
    M = np.diag(m.ravel().astype(float))
    K = np.vstack([M @ D, M @ Gx, M @ Gy, M @ Gz])
    assert O3.opnorm_3d(m) == pytest.approx(np.linalg.norm(K, 2), rel=1e-9)
    # full mask: bounded by sqrt(max D^2 + max eig G^T G) = sqrt(4/9 + 12)
    assert O3.opnorm_3d(np.ones((S, H, W))) <= np.sqrt(4.0 / 9.0 + 12.0)


@pytest.mark.parametrize("tv", ["aniso", "iso"])
def test_gap_and_stationarity_vanish(tv):
    rng = np.random.default_rng(5)
    S, H, W = 3, 6, 6
    f = rng.standard_normal((S, H, W))
    m = np.ones((S, H, W), np.uint8)
    m[:, 0, 0] = 0
    lam = 2.0
    L = O3.opnorm_3d(np.ones((S, H, W)))
    seen = []
    for n in (50, 400, 3000):
        st = O3.pd_solve_3d(f, m, lam, 1 / L, 1 / L, n, return_state=True, tv=tv)
        d = O3.diagnostics_3d(st, f, m, lam, tv=tv)
        assert d.gap >= -1e-12
        if seen:
            assert d.gap < seen[-1].gap and d.stationarity < seen[-1].stationarity
        seen.append(d)
    assert seen[-1].gap < 1e-6 * seen[-1].primal
    assert seen[-1].stationarity < 1e-2 * seen[0].stationarity


# --------------------------------------------------------------------------- planted mistakes


def _mistake_grad3_drops_z(x):
    gx, gy, _ = np.asarray(x) * 0, np.asarray(x) * 0, None
    gx[:, :, :-1] = x[:, :, 1:] - x[:, :, :-1]
    gy[:, :-1, :] = x[:, 1:, :] - x[:, :-1, :]
    return gx, gy, np.zeros_like(x)


def _mistake_adjoint_z_sign(a, b, c):
    out = np.zeros_like(a)
    out[:, :, 1:] += a[:, :, :-1]
    out[:, :, :-1] -= a[:, :, :-1]
    out[:, 1:, :] += b[:, :-1, :]
    out[:, :-1, :] -= b[:, :-1, :]
    out[1:, :, :] -= c[:-1, :, :]
    out[:-1, :, :] += c[:-1, :, :]
    return out


def _mistake_b0_along_x(shape, b0_axis=0, voxel=None):
    return O.dipole_kernel_3d(shape, b0_axis=2, voxel=voxel)


@pytest.mark.parametrize(
    "name,target,fake",
    [("grad3", O3, _mistake_grad3_drops_z), ("grad3_adjoint", O3, _mistake_adjoint_z_sign),
     ("dipole_kernel_3d", O3, _mistake_b0_along_x)],
)
def test_planted_mistakes_fail_the_dense_pin(monkeypatch, name, target, fake):
    rng = np.random.default_rng(6)
    S, H, W = 3, 4, 4
    f = rng.standard_normal((S, H, W))
    m = np.ones((S, H, W), np.uint8)
    ref = dense_pd(f, m, m.astype(float), 5.0, 0.28, 0.28, 25, "aniso")
    monkeypatch.setattr(target, name, fake)
    got = O3.pd_solve_3d(f, m, 5.0, 0.28, 0.28, 25)
    assert not np.allclose(got, ref, rtol=0, atol=1e-6)
