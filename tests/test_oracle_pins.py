"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test names what it pins.  A plausible slip in the oracle (a dropped term,
a swapped axis, a wrong sign, a wrong index, a transposed operand, the wrong
iterate fed to a step) fails at least one of them:

* kernel table       -> hand-computed fractions (tests/golden/dipole_kernel_points.txt)
* forward operator   -> cylinder and sphere closed forms; dense explicit-DFT brute force
* gradient / adjoint -> dense difference matrices; adjoint identities
* proxes             -> numerical minimisation; Moreau identity; library clip
* iteration order    -> first-iterate closed form; per-frequency matrix power of
                        the linear case (TV switched off, W = 1)
* convergence        -> Fenchel-Young gap and stationarity -> 0; KKT certificate
                        by bounded least squares; convexity probe
* step size          -> dense spectral norm; analytic upper bound
"""

import math
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy import optimize

from oracle import pd_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------- helpers (dense, independent of numpy.fft)


def dft_matrix(n):
    k = np.arange(n)
    return np.exp(-2j * np.pi * np.outer(k, k) / n)


def dense_D(H, W, Dk):
    """F^-1 diag(D) F as an explicit (HW x HW) matrix built from exp(), not numpy.fft."""
    F = np.kron(dft_matrix(H), dft_matrix(W))  # row-major flattening: idx = i*W + j
    Finv = F.conj().T / (H * W)
    return (Finv @ np.diag(Dk.ravel()) @ F).real


def dense_grad(H, W):
    """Forward differences (Neumann) as explicit matrices acting on row-major vectors."""
    n = H * W
    Gx = np.zeros((n, n))
    Gy = np.zeros((n, n))
    for i in range(H):
        for j in range(W):
            r = i * W + j
            if j < W - 1:
                Gx[r, r] = -1.0
                Gx[r, r + 1] = 1.0
            if i < H - 1:
                Gy[r, r] = -1.0
                Gy[r, r + W] = 1.0
    return Gx, Gy


def frac(s):
    """Parse '1/3-9/13' style sums of fractions."""
    total = Fraction(0)
    s = s.replace("-", "+-")
    for term in s.split("+"):
        if term:
            total += Fraction(term)
    return float(total)


# --------------------------------------------------------------------------- kernel table


def test_dipole_kernel_matches_hand_fractions():
    path = os.path.join(GOLDEN, "dipole_kernel_points.txt")
    n = 0
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        H, W, ax, i, j, expect = line.split()
        D = O.dipole_kernel(int(H), int(W), b0_axis=int(ax))
        assert D[int(i), int(j)] == pytest.approx(frac(expect), abs=1e-15), line
        n += 1
    assert n >= 15


def test_dipole_kernel_range_and_symmetry():
    D = O.dipole_kernel(12, 18)
    assert D.max() <= 1.0 / 3.0 + 1e-15 and D.min() >= -2.0 / 3.0 - 1e-15
    # even in each axis separately (depends on kx^2 and ky^2 only)
    assert np.array_equal(D, np.roll(D[::-1, :], 1, axis=0))
    assert np.array_equal(D, np.roll(D[:, ::-1], 1, axis=1))


def test_kernel_3d_restricts_to_2d_kernel():
    # the 2-D slice model is the 3-D kernel on the k_z = 0 plane (B0 in-plane along y)
    D3 = O.dipole_kernel_3d((10, 12, 6), b0_axis=0)
    assert np.allclose(D3[:, :, 0], O.dipole_kernel(10, 12, b0_axis=0), atol=1e-15)


# --------------------------------------------------------------------------- forward operator closed forms


def _golden_fields():
    vals = {}
    for line in open(os.path.join(GOLDEN, "dipole_field_closed_forms.txt")):
        if line.strip() and not line.startswith("#"):
            body, q, v = line.split()
            vals[(body, q)] = float(v)
    return vals


def test_cylinder_field_closed_form():
    g = _golden_fields()
    N, a = 1024, 24
    i = np.arange(N)[:, None]
    j = np.arange(N)[None, :]
    c = N // 2
    chi = ((i - c) ** 2 + (j - c) ** 2 <= a * a).astype(float)
    f = O.apply_D(chi, O.dipole_kernel(N, N))
    # D(0) = 0 removes the field's mean; the continuous field's mean over the
    # box is -(1/6) * area/N^2, so the periodic field is shifted by +that.
    offset = chi.sum() / (N * N) / 6.0
    a_eff = math.sqrt(chi.sum() / math.pi)
    assert f[c, c] - offset == pytest.approx(g[("cylinder", "inside_over_chi")], rel=2e-3)
    for r in (64, 96, 128):
        expect = g[("cylinder", "outside_coeff_over_chi")] * (a_eff / r) ** 2
        assert f[c + r, c] - offset == pytest.approx(expect, rel=1e-2)  # along B0 (y)
        assert f[c, c + r] - offset == pytest.approx(-expect, rel=1e-2)  # across B0


def test_sphere_field_closed_form():
    g = _golden_fields()
    N, a = 128, 8
    ax = np.arange(N) - N // 2
    Z, Y, X = np.meshgrid(ax, ax, ax, indexing="ij")
    s = (X**2 + Y**2 + Z**2 <= a * a).astype(float)
    f = O.apply_D_3d(s, O.dipole_kernel_3d((N, N, N), b0_axis=0))
    c = N // 2
    a_eff = (s.sum() * 3.0 / (4.0 * math.pi)) ** (1.0 / 3.0)
    assert abs(f[c, c, c] - g[("sphere", "inside_over_chi")]) < 1e-12
    for r in (16, 24, 32):
        coeff = g[("sphere", "outside_coeff_over_chi")] * (a_eff / r) ** 3
        assert f[c + r, c, c] == pytest.approx(2.0 * coeff, rel=2e-2)  # theta = 0
        assert f[c, c + r, c] == pytest.approx(-coeff, rel=2e-2)  # theta = 90 deg


# --------------------------------------------------------------------------- dense brute force of the operators


@pytest.mark.parametrize("H,W", [(4, 4), (5, 6), (6, 8), (3, 7), (4, 22), (2, 86)])
def test_apply_D_matches_dense_dft(H, W):
    rng = np.random.default_rng(H * 100 + W)
    Dk = O.dipole_kernel(H, W)
    x = rng.standard_normal((H, W))
    ref = dense_D(H, W, Dk) @ x.ravel()
    assert np.allclose(O.apply_D(x, Dk).ravel(), ref, atol=1e-13)


@pytest.mark.parametrize("H,W", [(4, 4), (5, 6), (1, 7), (7, 1)])
def test_grad_and_adjoint_match_dense(H, W):
    rng = np.random.default_rng(7)
    Gx, Gy = dense_grad(H, W)
    x = rng.standard_normal((H, W))
    gx, gy = O.grad(x)
    assert np.allclose(gx.ravel(), Gx @ x.ravel(), atol=1e-14)
    assert np.allclose(gy.ravel(), Gy @ x.ravel(), atol=1e-14)
    a = rng.standard_normal((H, W))
    b = rng.standard_normal((H, W))
    assert np.allclose(O.grad_adjoint(a, b).ravel(), Gx.T @ a.ravel() + Gy.T @ b.ravel(), atol=1e-14)


def test_adjoint_identities_random():
    rng = np.random.default_rng(11)
    H, W = 24, 20
    Dk = O.dipole_kernel(H, W)
    m = (rng.random((H, W)) > 0.3).astype(float)
    x, y = rng.standard_normal((2, H, W))
    lhs, rhs = np.vdot(O.apply_D(x, Dk), y), np.vdot(x, O.apply_D(y, Dk))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)
    a, b = rng.standard_normal((2, H, W))
    gx, gy = O.grad(x)
    lhs, rhs = np.vdot(gx, a) + np.vdot(gy, b), np.vdot(x, O.grad_adjoint(a, b))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)
    y0, y1, y2 = rng.standard_normal((3, H, W))
    k0, k1, k2 = O.apply_K(x, Dk, m, m)
    lhs = np.vdot(k0, y0) + np.vdot(k1, y1) + np.vdot(k2, y2)
    rhs = np.vdot(x, O.apply_KT(y0, y1, y2, Dk, m, m))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_D_output_is_real():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((32, 48))
    Dk = O.dipole_kernel(32, 48)
    y = np.fft.ifft2(Dk * np.fft.fft2(x))
    assert np.max(np.abs(y.imag)) < 1e-15 * np.max(np.abs(x)) * 32


# --------------------------------------------------------------------------- proxes


def test_prox_dual_data_is_moreau_of_numerical_primal_prox():
    rng = np.random.default_rng(5)
    lam, sigma = 0.7, 0.35
    v, b = rng.standard_normal((2, 6))

    # prox of (F1/sigma) at v/sigma, F1(z) = lam/2 ||z - b||^2, by numerical minimisation
    def obj(z):
        return 0.5 * lam * np.sum((z - b) ** 2) + 0.5 * sigma * np.sum((z - v / sigma) ** 2)

    z = optimize.minimize(obj, np.zeros(6), method="BFGS", options={"gtol": 1e-12}).x
    assert np.allclose(O.prox_dual_data(v, b, sigma, lam), v - sigma * z, atol=1e-7)


def test_clamp_soft_threshold_moreau_and_library():
    v = np.linspace(-3, 3, 601)
    assert np.array_equal(O.clamp_unit(v) + O.soft_threshold(v, 1.0), v)  # Moreau, exact
    assert np.array_equal(O.prox_dual_tv(v), np.clip(v, -1.0, 1.0))
    # soft-threshold minimises |z| + (z - v)^2 / 2 (brute force on a fine grid)
    grid = np.linspace(-4, 4, 80001)
    for vi in (-2.5, -0.3, 0.0, 0.8, 1.7):
        zbest = grid[np.argmin(np.abs(grid) + 0.5 * (grid - vi) ** 2)]
        assert abs(O.soft_threshold(np.array(vi), 1.0) - zbest) <= 1e-4


# --------------------------------------------------------------------------- iteration order


def test_first_iterate_closed_form():
    # chi_bar_0 = 0 => p_1 = -sigma b / (1 + sigma/lam), q_1 = 0,
    # chi_1 = -tau D W p_1 = tau sigma / (1 + sigma/lam) D (W b)
    rng = np.random.default_rng(21)
    H, W = 6, 5
    f = rng.standard_normal((H, W))
    m = (rng.random((H, W)) > 0.25).astype(float)
    w = m * rng.uniform(0.5, 1.5, (H, W))  # non-binary weight: W enters twice
    lam, tau, sigma = 0.3, 0.31, 0.33
    Dd = dense_D(H, W, O.dipole_kernel(H, W))
    for weight in (None, w):
        wt = m if weight is None else w
        chi1 = O.pd_solve(f, m, lam, tau, sigma, 1, weight=weight)
        ref = tau * sigma / (1 + sigma / lam) * (Dd @ (wt * wt * f).ravel())
        assert np.allclose(chi1.ravel(), ref, atol=1e-15)


@pytest.mark.parametrize("n_iter", [1, 2, 3, 17, 200])
def test_linear_case_per_frequency_matrix_power(n_iter):
    """W = 1 and M = 0: every frequency follows its own affine 3-state recurrence.

    State (p, chi, chi_bar) per frequency with d = D(k), c = 1/(1 + sigma/lam):
      p'   = c p + c sigma d chi_bar - c sigma f
      chi' = chi - tau d p'
      cb'  = 2 chi' - chi
    chi_N = [A^N]_{chi, 1} from the zero start, evaluated with matrix_power.
    """
    rng = np.random.default_rng(100 + n_iter)
    H, W = 8, 6
    f = rng.standard_normal((H, W))
    lam, L = 0.8, 2.9
    tau = sigma = 1.0 / L
    out = O.pd_solve(f, np.ones((H, W)), lam, tau, sigma, n_iter, weight=np.ones((H, W)), tv_mask=np.zeros((H, W)))
    Dk = O.dipole_kernel(H, W)
    fh = np.fft.fft2(f)
    c = 1.0 / (1.0 + sigma / lam)
    chih = np.zeros((H, W), dtype=complex)
    for i in range(H):
        for j in range(W):
            d, fk = Dk[i, j], fh[i, j]
            A = np.array(
                [
                    [c, 0, c * sigma * d, -c * sigma * fk],
                    [-tau * d * c, 1, -tau * c * sigma * d * d, tau * d * c * sigma * fk],
                    [-2 * tau * d * c, 1, -2 * tau * c * sigma * d * d, 2 * tau * d * c * sigma * fk],
                    [0, 0, 0, 1],
                ],
                dtype=complex,
            )
            chih[i, j] = np.linalg.matrix_power(A, n_iter)[1, 3]
    ref = np.fft.ifft2(chih).real
    assert np.allclose(out, ref, atol=1e-12 * max(1.0, np.abs(ref).max()))


def test_fixed_points_zero_field_and_empty_mask():
    rng = np.random.default_rng(2)
    H, W = 16, 12
    L, tau, sigma = 2.9, 1 / 2.9, 1 / 2.9
    assert np.all(O.pd_solve(np.zeros((H, W)), np.ones((H, W)), 0.1, tau, sigma, 50) == 0)
    assert np.all(O.pd_solve(rng.standard_normal((H, W)), np.zeros((H, W)), 0.1, tau, sigma, 50) == 0)
    assert np.all(O.pd_solve(rng.standard_normal((H, W)), np.ones((H, W)), 0.1, tau, sigma, 0) == 0)


def test_slices_are_independent():
    rng = np.random.default_rng(9)
    f = rng.standard_normal((3, 10, 8))
    m = (rng.random((3, 10, 8)) > 0.2).astype(float)
    tau = sigma = 1 / 2.9
    stack = O.pd_solve(f, m, 0.5, tau, sigma, 40)
    for s in range(3):
        alone = O.pd_solve(f[s], m[s], 0.5, tau, sigma, 40)
        assert np.allclose(stack[s], alone, rtol=0, atol=1e-14)


# --------------------------------------------------------------------------- step size


@pytest.mark.parametrize("H,W,seed", [(6, 6, 0), (8, 8, 1), (5, 7, 2)])
def test_opnorm_matches_dense_spectral_norm(H, W, seed):
    rng = np.random.default_rng(seed)
    m = (rng.random((H, W)) > 0.3).astype(float)
    Dd = dense_D(H, W, O.dipole_kernel(H, W))
    Gx, Gy = dense_grad(H, W)
    Mm = np.diag(m.ravel())
    K = np.vstack([Mm @ Dd, Mm @ Gx, Mm @ Gy])
    assert O.opnorm(m, rtol=1e-14) == pytest.approx(np.linalg.norm(K, 2), rel=1e-7)


def test_golden_step_size_table_is_the_oracles():
    import os

    path = os.path.join(GOLDEN, "opnorm_full_mask.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    for H, W, ax, L in rows:
        if int(H) <= 64:  # recompute the cheap ones
            assert O.opnorm(np.ones((int(H), int(W))), b0_axis=int(ax)) == pytest.approx(float(L), rel=1e-12)
        assert 2.7 < float(L) <= math.sqrt(4.0 / 9.0 + 8.0)


def test_opnorm_bounds_full_mask():
    # ||D|| <= 2/3 and ||G||^2 <= 8 give ||K|| <= sqrt(4/9 + 8)
    for n in (8, 32, 64):
        L = O.opnorm(np.ones((n, n)))
        assert 2.7 < L <= math.sqrt(4.0 / 9.0 + 8.0)


# --------------------------------------------------------------------------- convergence and optimality


def _kkt_residual(chi, f, m, lam, w=None):
    """Smallest ||G^T(M q) + lam D W (W D chi - b)|| over admissible subgradients q.

    q must lie in [-1, 1]^2 and equal sign(g) where |g| = |M G chi| > 1e-7;
    solved by bounded least squares (independent of the iterates' q).
    """
    H, W = chi.shape
    Dd = dense_D(H, W, O.dipole_kernel(H, W))
    Gx, Gy = dense_grad(H, W)
    mv = m.ravel()
    wv = mv if w is None else w.ravel()
    g = np.concatenate([mv * (Gx @ chi.ravel()), mv * (Gy @ chi.ravel())])
    A = np.hstack([Gx.T @ np.diag(mv), Gy.T @ np.diag(mv)])
    rhs = -lam * (Dd @ (wv * (wv * (Dd @ chi.ravel()) - wv * f.ravel())))
    lo = -np.ones(g.size)
    hi = np.ones(g.size)
    act = np.abs(g) > 1e-7
    lo[act] = np.sign(g[act]) - 1e-12
    hi[act] = np.sign(g[act]) + 1e-12
    res = optimize.lsq_linear(A, rhs, bounds=(lo, hi), method="bvls", tol=1e-15, lsmr_tol=None)
    return float(np.linalg.norm(A @ res.x - rhs)), float(np.linalg.norm(rhs))


@pytest.mark.parametrize(
    "seed,lam,mask_kind",
    [(0, 50.0, "one_hole"), (1, 1.0, "full"), (2, 50.0, "random"), (3, 20.0, "weighted")],
)
def test_gap_stationarity_and_kkt_8x8(seed, lam, mask_kind):
    rng = np.random.default_rng(seed)
    H = W = 8
    f = rng.standard_normal((H, W))
    m = np.ones((H, W))
    if mask_kind == "one_hole":
        m[3, 4] = 0.0
    elif mask_kind == "random":
        m = (rng.random((H, W)) > 0.25).astype(float)
    w = None
    if mask_kind == "weighted":  # non-binary W (pins where W enters), M = 1
        w = rng.uniform(0.3, 1.0, (H, W))
    L = O.opnorm(np.ones((H, W)))
    st = O.pd_solve(f, m, lam, 1 / L, 1 / L, 10000, weight=w, return_state=True)
    dg = O.diagnostics(st, f, m, lam, weight=w)
    assert dg.gap >= -1e-12
    assert dg.gap < 1e-9
    assert dg.stationarity < 1e-8
    res, scale = _kkt_residual(st.chi, f, m, lam, w)
    assert res < 1e-7 * max(1.0, scale)
    # convexity probe: random perturbations never lower the objective
    base = dg.primal
    for _ in range(20):
        d = rng.standard_normal((H, W)) * 1e-3
        pert = O.PDState(st.chi + d, st.chi_bar, st.p, st.qx, st.qy, st.n)
        assert O.diagnostics(pert, f, m, lam, weight=w).primal >= base - 1e-12


def test_gap_decreases_on_phantom():
    from phantoms import config1

    pb = config1()
    f, m = pb.field[0].astype(float), pb.mask[0].astype(float)
    L = O.opnorm(np.ones(f.shape))
    gaps = []
    for n in (50, 400, 3000):
        st = O.pd_solve(f, m, 10.0, 1 / L, 1 / L, n, return_state=True)
        gaps.append(O.diagnostics(st, f, m, 10.0).gap)
    assert gaps[0] > gaps[1] > gaps[2] >= 0


# --------------------------------------------------------------------------- isotropic TV reading


def test_iso_prox_is_disc_projection():
    rng = np.random.default_rng(31)
    vx, vy = rng.standard_normal((2, 200)) * 1.5
    px, py = O.prox_dual_tv_iso(vx, vy)
    assert np.all(px * px + py * py <= 1 + 1e-12)
    inside = vx * vx + vy * vy <= 1
    assert np.array_equal(px[inside], vx[inside]) and np.array_equal(py[inside], vy[inside])
    # outside: the nearest point of the disc is on the same ray (brute force on a fine circle)
    th = np.linspace(0, 2 * np.pi, 200001)
    for k in np.nonzero(~inside)[0][:10]:
        d = (np.cos(th) - vx[k]) ** 2 + (np.sin(th) - vy[k]) ** 2
        t = th[np.argmin(d)]
        assert abs(px[k] - np.cos(t)) < 1e-4 and abs(py[k] - np.sin(t)) < 1e-4


def test_iso_equals_aniso_on_single_row_slices():
    # with one row G_y = 0, so the pointwise Euclidean norm is the absolute value
    rng = np.random.default_rng(32)
    f = rng.standard_normal((3, 1, 24))
    m = np.ones((3, 1, 24))
    a = O.pd_solve(f, m, 2.0, 0.3, 0.3, 80, tv="aniso")
    b = O.pd_solve(f, m, 2.0, 0.3, 0.3, 80, tv="iso")
    assert np.allclose(a, b, rtol=0, atol=1e-15)


def test_iso_gap_and_stationarity_vanish_8x8():
    rng = np.random.default_rng(33)
    f = rng.standard_normal((8, 8))
    m = np.ones((8, 8))
    m[2, 5] = 0
    L = O.opnorm(np.ones((8, 8)))
    st = O.pd_solve(f, m, 30.0, 1 / L, 1 / L, 10000, return_state=True, tv="iso")
    dg = O.diagnostics(st, f, m, 30.0, tv="iso")
    assert 0 <= dg.gap < 1e-9 and dg.stationarity < 1e-8
    assert np.all(st.qx ** 2 + st.qy ** 2 <= 1 + 1e-12)
    # the iso solution differs from the aniso one (the readings are not equivalent)
    st2 = O.pd_solve(f, m, 30.0, 1 / L, 1 / L, 10000, return_state=True)
    assert np.linalg.norm(st.chi - st2.chi) > 1e-6 * np.linalg.norm(st2.chi)
