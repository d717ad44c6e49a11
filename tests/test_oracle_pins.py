"""Pins for the FP64 CPU oracle (no GPU).

Each test checks the oracle against something other than itself: a closed
form, an independent (Hessian-matrix) statement of the discrete operator, a
brute-force dense Newton solve, an FFT Poisson solve, or the spherical
closed form of Eq. (eomvarphi_sph2).  Every one is chosen so that a dropped
term, a wrong sign, a wrong index or a transposed operand fails it.
"""
import os

import numpy as np
import pytest

import oracle
import workload
from tests import _pins

HERE = os.path.dirname(os.path.abspath(__file__))


# ---------------------------------------------------------------- coefficients

def _golden(name):
    rows = {}
    with open(os.path.join(HERE, "golden", name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split("=")
                rows[k.strip()] = float(v)
    return rows


def test_coefficients_golden_a1():
    """Eq. (beta) at a = 1 for the LCDM-matched background: beta = 3 - Omega_m0 when H0 r_c = 1."""
    g = _golden("coefficients_a1.txt")
    beta, alpha, s = oracle.ndgp_coefficients(1.0, g["omega_m0"], g["h0rc"])
    assert beta == pytest.approx(g["beta"], rel=1e-15)
    assert alpha * s == pytest.approx(g["eps"], rel=1e-13)


@pytest.mark.parametrize("a,om,h0rc", [(0.5, 0.3, 1.0), (0.8, 0.269, 1.0), (0.33, 0.3, 2.0)])
def test_coefficients_vs_numerical_derivative(a, om, h0rc):
    """beta(a) of Eq. (beta) with Hdot taken by a numerical time derivative of H(a)."""
    H0 = 100.0 / 299792.458

    def H(x):
        return H0 * np.sqrt(om / x ** 3 + 1.0 - om)

    da = 1e-6 * a
    dHda = (H(a + da) - H(a - da)) / (2 * da)
    Hdot = dHda * a * H(a)          # da/dt = a H
    rc = h0rc / H0
    beta_ref = 1.0 + 2.0 * H(a) * rc * (1.0 + Hdot / (3.0 * H(a) ** 2))
    beta, alpha, s = oracle.ndgp_coefficients(a, om, h0rc)
    assert beta == pytest.approx(beta_ref, rel=1e-9)
    assert alpha == pytest.approx(rc ** 2 / (3 * beta_ref * a * a), rel=1e-9)
    # 8 pi G rho_bar(a) a^2 / (3 beta) with 8 pi G rho_bar0 = 3 H0^2 Omega_m0
    assert s == pytest.approx(3 * H0 ** 2 * om / a ** 3 * a ** 2 / (3 * beta_ref), rel=1e-9)


# ---------------------------------------------------------------- operator

@pytest.mark.parametrize("n,h,alpha", [(8, 0.7, 0.37), (12, 1.3, 2.0), (6, 0.25, 0.0)])
def test_operator_matches_hessian_matrix_form(n, h, alpha):
    phi = workload.smooth_periodic_field(n, 1.0, 3) + 0.1 * workload.lognormal_delta(n, 1.0, 5)
    a = oracle.operator(phi, h, alpha)
    b = _pins.op_matrix(phi, h, alpha)
    assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()


@pytest.mark.parametrize("nvec", [(1, 2, 3), (0, 1, 0), (2, -1, 1), (3, 3, 0)])
def test_operator_fourier_symbol(nvec):
    n, h, alpha, amp = 16, 0.9, 0.4, 0.8
    phi = amp * np.cos(_pins.cos_mode(n, nvec, h))
    a = oracle.operator(phi, h, alpha)
    b = _pins.op_symbol_cos(n, nvec, h, alpha, amp)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


def test_operator_continuum_limit():
    """Discrete operator -> analytic L + alpha[(lap)^2 - (dd)^2] with O(h^2) error."""
    errs = []
    for n in (32, 64):
        h = 2 * np.pi / n
        x = (np.arange(n) + 0.5) * h
        X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
        phi = np.sin(X) * np.cos(2 * Y) + 0.5 * np.sin(Y + Z)
        # analytic second derivatives
        pxx = -np.sin(X) * np.cos(2 * Y)
        pyy = -4 * np.sin(X) * np.cos(2 * Y) - 0.5 * np.sin(Y + Z)
        pzz = -0.5 * np.sin(Y + Z)
        pxy = -2 * np.cos(X) * np.sin(2 * Y)
        pxz = np.zeros_like(X)
        pyz = -0.5 * np.sin(Y + Z)
        lap = pxx + pyy + pzz
        dd = pxx ** 2 + pyy ** 2 + pzz ** 2 + 2 * (pxy ** 2 + pxz ** 2 + pyz ** 2)
        exact = lap + 0.3 * (lap ** 2 - dd)
        errs.append(np.abs(oracle.operator(phi, h, 0.3) - exact).max())
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.1)


# ---------------------------------------------------------------- cell update

def _rand_state(n, seed, amp=1.0):
    return workload.smooth_periodic_field(n, amp, seed) + 0.05 * workload.lognormal_delta(n, 1.0, seed + 1)


@pytest.mark.parametrize("alpha", [0.0, 0.05, 0.3])
def test_cell_update_solves_its_equation(alpha):
    """Back-substitution: after the update, the cell's own equation holds."""
    n, h = 8, 1.0
    phi = _rand_state(n, 2)
    rng = np.random.default_rng(0)
    for _ in range(20):
        i, j, k = rng.integers(0, n, 3)
        rhs = float(rng.uniform(-0.4, 2))      # 1 + 8 alpha b / 3 > 0: a real root exists
        new = oracle.cell_update(phi, (i, j, k), h, alpha, rhs)
        p2 = phi.copy()
        p2[i, j, k] = new
        lhs = _pins.op_matrix(p2, h, alpha)[i, j, k]
        assert lhs == pytest.approx(rhs, abs=1e-12 * max(1.0, abs(rhs)))


def test_cell_update_clamps_negative_discriminant():
    """No real root: the discriminant is clamped to zero and the clamp is counted."""
    n, h, alpha = 8, 1.0, 0.3
    phi = np.zeros((n, n, n))
    before = oracle.clamped()
    v = oracle.cell_update(phi, (1, 1, 1), h, alpha, -5.0)   # 1 + 8 (0.3)(-5)/3 < 0
    assert oracle.clamped() == before + 1
    # clamped root L = 2b, phi = -h^2 L / 6
    assert v == pytest.approx(-(2 * -5.0) / 6.0, rel=1e-15)


def test_cell_update_is_newton_fixed_point():
    """Iterating Eq. (newton) on one cell with frozen neighbours reaches the same value."""
    n, h, alpha = 8, 1.0, 0.2
    phi = _rand_state(n, 4)
    idx = (3, 5, 1)
    rhs = 0.7
    target = oracle.cell_update(phi, idx, h, alpha, rhs)
    p = phi.copy()

    def T(v):
        p[idx] = v
        return _pins.op_matrix(p, h, alpha)[idx] - rhs

    v = phi[idx]
    for _ in range(50):
        d = 1e-3
        dT = (T(v + d) - T(v - d)) / (2 * d)      # exact: T is quadratic in v
        step = T(v) / dT
        v = v - step
        if abs(step) < 1e-16:
            break
    assert v == pytest.approx(target, abs=1e-13)


def test_cell_update_physical_branch_is_linear_limit():
    """For alpha -> 0 the update tends to the Poisson (Gauss-Seidel) value."""
    n, h = 8, 1.0
    phi = _rand_state(n, 6)
    lin = oracle.cell_update(phi, (1, 2, 3), h, 0.0, 0.4)
    for alpha in (1e-3, 1e-5, 1e-7):
        v = oracle.cell_update(phi, (1, 2, 3), h, alpha, 0.4)
        assert abs(v - lin) < 50 * alpha


# ---------------------------------------------------------------- sweep

@pytest.mark.parametrize("alpha", [0.0, 0.25])
def test_sweep_snapshot_semantics(alpha):
    """Every red cell solves its equation against the start-of-sweep state, every
    black cell against (new red, start-of-sweep black); red is (i+j+k) even."""
    n, h = 8, 0.8
    phi0 = _rand_state(n, 8)
    f = workload.lognormal_delta(n, 1.0, 9)
    c = 0.013
    phi1 = oracle.sweep(phi0, f, c, h, alpha)
    i = np.arange(n)
    I, J, K = np.meshgrid(i, i, i, indexing="ij")
    red = (I + J + K) % 2 == 0
    mid = np.where(red, phi1, phi0)
    rng = np.random.default_rng(1)
    for _ in range(40):
        p = tuple(rng.integers(0, n, 3))
        base = phi0.copy() if red[p] else mid.copy()
        base[p] = phi1[p]
        lhs = _pins.op_matrix(base, h, alpha)[p]
        assert lhs == pytest.approx(f[p] + c, abs=1e-12)
    # ordering: sweeping black first would give a different state
    assert not np.allclose(phi1, phi0)


# ---------------------------------------------------------------- transfers

def test_restrict_prolong_fourier_closed_forms():
    nf, kx = 16, 3
    hf = 1.0
    i = np.arange(nf)
    xf = (i + 0.5) * hf
    th = 2 * np.pi * kx / (nf * hf)
    fine = np.broadcast_to(np.cos(th * xf)[:, None, None], (nf,) * 3).copy()
    c = oracle.restrict(fine)
    Xc = (np.arange(nf // 2) + 0.5) * 2 * hf
    ref = np.cos(th * Xc) * np.cos(th * hf / 2)      # mean of the two children
    assert np.abs(c[:, 0, 0] - ref).max() < 1e-14
    # prolongation of a coarse mode: 3/4 parent + 1/4 neighbour on the fine centre's side
    coarse = np.broadcast_to(np.cos(th * Xc)[:, None, None], (nf // 2,) * 3).copy()
    pf = oracle.prolong_add(coarse, np.zeros((nf,) * 3))[:, 3, 5]
    # fine centre sits hf/2 from the parent centre; neighbour is 3hf/2 away on that side
    expect = np.real(np.exp(1j * th * xf) * (0.75 * np.exp(-1j * th * hf / 2 * np.where(i % 2, 1, -1))
                                           + 0.25 * np.exp(1j * th * 3 * hf / 2 * np.where(i % 2, 1, -1))))
    assert np.abs(pf - expect).max() < 1e-14


def test_transfers_constants_and_mean():
    fine = workload.lognormal_delta(8, 1.0, 3)
    assert oracle.restrict(fine).mean() == pytest.approx(fine.mean(), abs=1e-15)
    ones = np.ones((4, 4, 4))
    assert np.allclose(oracle.prolong_add(ones * 2.5, np.zeros((8, 8, 8))), 2.5, atol=1e-15)
    assert np.allclose(oracle.restrict(np.full((8, 8, 8), -1.25)), -1.25, atol=1e-15)


# ---------------------------------------------------------------- force

@pytest.mark.parametrize("nvec", [(1, 0, 0), (2, 3, 1)])
def test_force_fourier_closed_form(nvec):
    n, h = 16, 0.6
    th = _pins.cos_mode(n, nvec, h)
    phi = np.cos(th)
    g = oracle.force(phi, h)
    for a in range(3):
        kh = 2 * np.pi * nvec[a] / n
        ref = -np.sin(th) * np.sin(kh) / h
        assert np.abs(g[a] - ref).max() < 1e-13


def test_force_box_interior_matches_periodic():
    n, h, gh = 12, 0.5, 2
    phi = _rand_state(n, 10)
    box = np.pad(phi, gh, mode="wrap")
    gp = oracle.force(phi, h)
    gb = oracle.force(box, h, ghost=gh, periodic=False)
    assert np.abs(gp - gb).max() < 1e-15


# ---------------------------------------------------------------- solve

@pytest.mark.parametrize("n", [16, 32])
def test_solve_linear_limit_matches_fft_poisson(n):
    d = workload.lognormal_delta(n, 1.0, 7)
    phi, info = oracle.solve(d, 0.0, 1.3, 0.9, tol=1e-13)
    ref = _pins.fft_poisson(1.3 * d, 0.9)
    assert info.status == 0
    assert np.linalg.norm(phi - ref) / np.linalg.norm(ref) < 1e-12
    assert abs(info.compat_c) < 1e-14


@pytest.mark.parametrize("n,alpha", [(4, 0.2), (8, 0.2), (8, 0.05)])
def test_solve_matches_dense_newton(n, alpha):
    d = workload.lognormal_delta(n, 1.0, 11)
    pn, cn = _pins.dense_newton(d, 1.0, alpha)
    phi, info = oracle.solve(d, alpha, 1.0, 1.0, tol=1e-14, max_cycles=200)
    assert info.status == 0
    assert np.linalg.norm(phi - pn) / np.linalg.norm(pn) < 1e-12
    assert info.compat_c == pytest.approx(cn, rel=1e-11)


@pytest.mark.parametrize("n", [16, 24])
def test_solve_manufactured_solution(n):
    h, alpha, s = 0.5, 0.1, 2.0
    phim = workload.smooth_periodic_field(n, 0.02, 13)
    f = _pins.op_matrix(phim, h, alpha)
    cstar = f.mean()
    delta = (f - cstar) / s
    phi, info = oracle.solve(delta, alpha, s, h, tol=1e-12)
    ref = phim - phim.mean()
    assert info.status == 0
    assert np.linalg.norm(phi - ref) / np.linalg.norm(ref) < 1e-10
    assert info.compat_c == pytest.approx(cstar, rel=1e-8)


def test_solve_final_residual_below_tol_and_mean_zero():
    n, h = 16, 250.0 / 512
    beta, alpha, s = oracle.ndgp_coefficients(1.0, 0.3, 1.0)
    d = workload.lognormal_delta(n, 1.0, 1)
    phi, info = oracle.solve(d, alpha, s, h, tol=1e-10)
    r = _pins.op_matrix(phi, h, alpha) - s * d - info.compat_c
    assert np.linalg.norm(r) / np.linalg.norm(s * d) <= 1e-10
    assert abs(phi.mean()) < 1e-12 * np.abs(phi).max()


def test_compat_constant_vanishes_as_h_squared():
    """The periodic compatibility constant is a discretisation artefact: c ~ h^2."""
    cs = []
    L, R, A, alpha = 32.0, 3.0, 50.0, 0.2
    for n in (16, 32):
        h = L / n
        d = workload.gaussian_blob(n, A, R / h)
        _, info = oracle.solve(d, alpha, 1.0, h, tol=1e-10)
        cs.append(info.compat_c)
    assert cs[0] / cs[1] == pytest.approx(4.0, rel=0.15)


def _radial_error(n, L, R, A, alpha, s=1.0):
    h = L / n
    d = workload.gaussian_blob(n, A, R / h)
    phi, info = oracle.solve(d, alpha, s, h, tol=1e-10)
    g = oracle.force(phi, h)
    x = (np.arange(n) - (n / 2 - 0.5)) * h
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    r = np.sqrt(X ** 2 + Y ** 2 + Z ** 2)
    gr = (g[0] * X + g[1] * Y + g[2] * Z) / np.maximum(r, 1e-30)
    sel = (r > 1.5 * R) & (r < 4 * R)
    bg = (A * np.exp(-r ** 2 / (2 * R ** 2))).mean()
    m = _pins.gaussian_enclosed(r[sel], A, R, bg)
    ref = _pins.spherical_dphi_dr(r[sel], m, alpha, s)
    lin = _pins.spherical_dphi_dr(r[sel], m, 0.0, s)
    err = np.sqrt(np.mean((gr[sel] - ref) ** 2)) / np.sqrt(np.mean(ref ** 2))
    return err, float(np.mean(lin) / np.mean(ref)), info


def test_spherical_vainshtein_profile():
    """Eq. (eomvarphi_sph2): radial phi_r of a Gaussian overdensity (delta_max = 250,
    3x the nominal eps = alpha s, so the force is screened by ~40%) matches the
    closed form to the periodic-image floor, and the discretisation error falls
    ~4x from N = 32 to 64."""
    L, R, A, alpha = 64.0, 4.0, 250.0, 3 * 0.0137174
    e32, screen, _ = _radial_error(32, L, R, A, alpha)
    e64, _, info = _radial_error(64, L, R, A, alpha)
    assert screen > 1.5                      # the nonlinear term matters here
    assert e64 < 6e-3
    assert e32 / e64 > 2.5
    assert info.clamped == 0


@pytest.mark.slow
def test_spherical_vainshtein_profile_128():
    L, R, A, alpha = 64.0, 4.0, 250.0, 3 * 0.0137174
    e128, _, _ = _radial_error(128, L, R, A, alpha)
    assert e128 < 6e-3


def test_spherical_linear_limit():
    """Eq. (forcelarge): alpha = 0 gives the unscreened force (here: Poisson)."""
    L, R, A = 64.0, 4.0, 10.0
    e32, screen, _ = _radial_error(32, L, R, A, 0.0)
    e64, _, _ = _radial_error(64, L, R, A, 0.0)
    assert screen == pytest.approx(1.0)
    assert e64 < 4e-3 and e32 / e64 > 3.0


def test_tophat_screening_grows_inward():
    """Eq. (forcesmall): outside a top-hat the ratio F5 / F5_linear falls as r / r_V falls.

    The closed form is met to a few per cent: the staircase edge of a top-hat
    6 cells in radius costs O(h) in the nonlinear term (2.5% here, 4.6% at
    4 cells), while the linear case agrees to 1e-4 at either radius.
    """
    n, h, A, Rth, alpha = 48, 1.0, 60.0, 6.0, 3 * 0.0137174
    x = np.arange(n) - (n / 2 - 0.5)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    r = np.sqrt(X ** 2 + Y ** 2 + Z ** 2)
    raw = np.where(r < Rth, A, 0.0)
    d = raw - raw.mean()
    phi, _ = oracle.solve(d, alpha, 1.0, h, tol=1e-10)
    philin, _ = oracle.solve(d, 0.0, 1.0, h, tol=1e-10)
    g, gl = oracle.force(phi, h), oracle.force(philin, h)
    gr = (g[0] * X + g[1] * Y + g[2] * Z) / r
    glr = (gl[0] * X + gl[1] * Y + gl[2] * Z) / r
    shells = [(1.2 * Rth, 1.5 * Rth), (1.7 * Rth, 2.1 * Rth), (2.5 * Rth, 3.0 * Rth)]
    ratios = []
    for lo, hi in shells:
        sel = (r > lo) & (r < hi)
        ratios.append(np.mean(gr[sel]) / np.mean(glr[sel]))
    assert ratios[0] < ratios[1] < ratios[2] < 1.0
    # closed form (top-hat mass, background included) in the middle shell
    M = raw.sum() / (4 * np.pi)
    sel = (r > 1.7 * Rth) & (r < 2.1 * Rth)
    m = M - raw.mean() * r[sel] ** 3 / 3
    ref = _pins.spherical_dphi_dr(r[sel], m, alpha, 1.0)
    lin = _pins.spherical_dphi_dr(r[sel], m, 0.0, 1.0)
    assert np.mean(gr[sel]) == pytest.approx(np.mean(ref), rel=0.04)
    assert np.mean(glr[sel]) == pytest.approx(np.mean(lin), rel=1e-3)


# ---------------------------------------------------------------- refine_interpolate

def test_refine_interpolate_constant_and_linear():
    nc = 16
    c = np.full((nc,) * 3, 3.25)
    f = oracle.refine_interpolate(c, (2, 3, 4), (4, 5, 6), 1)
    assert f.shape == (10, 12, 14)
    assert np.allclose(f, 3.25, atol=1e-14)
    # linear field: exact where the stencil does not wrap
    i = np.arange(nc) + 0.5
    I, J, K = np.meshgrid(i, i, i, indexing="ij")
    lin = 0.3 * I - 1.1 * J + 2.0 * K
    o, pn, g = (3, 4, 5), (4, 4, 4), 1
    f = oracle.refine_interpolate(lin, o, pn, g)
    loc = [o[a] + (np.arange(2 * pn[a] + 2 * g) - g + 0.5) / 2 for a in range(3)]
    X, Y, Z = np.meshgrid(*loc, indexing="ij")
    assert np.abs(f - (0.3 * X - 1.1 * Y + 2.0 * Z)).max() < 1e-13


def test_refine_interpolate_child_average_closed_form():
    """1-D: the mean of the two fine children of coarse cell i is 3/4 phi_i + 1/8 (phi_{i-1} + phi_{i+1})."""
    nc = 16
    rng = np.random.default_rng(3)
    line = rng.standard_normal(nc)
    c = np.broadcast_to(line[:, None, None], (nc,) * 3).copy()
    f = oracle.refine_interpolate(c, (0, 0, 0), (nc, 2, 2), 0)
    avg = 0.5 * (f[0::2, 1, 1] + f[1::2, 1, 1])
    ref = 0.75 * line + 0.125 * (np.roll(line, 1) + np.roll(line, -1))
    assert np.abs(avg - ref).max() < 1e-14


def test_refine_interpolate_translation_invariance():
    """Periodic wrap: interpolating a rolled field at a shifted origin gives the same patch."""
    nc = 12
    phi = _rand_state(nc, 21)
    a = oracle.refine_interpolate(phi, (10, 11, 0), (4, 3, 5), 2)
    b = oracle.refine_interpolate(np.roll(phi, (-5, -7, 3), axis=(0, 1, 2)), (5, 4, 3), (4, 3, 5), 2)
    assert np.abs(a - b).max() < 1e-14


def test_refine_cubic_reproduces_cubics_and_constants():
    """The tricubic variant (4-point Lagrange per axis, an extension) is exact for any cubic
    polynomial where its stencil does not wrap, and keeps constants."""
    nc = 20
    c = np.full((nc,) * 3, -1.75)
    assert np.allclose(oracle.refine_cubic(c, (3, 7, 11), (4, 5, 3), 1), -1.75, atol=1e-14)
    i = np.arange(nc) + 0.5
    I, J, K = np.meshgrid(i, i, i, indexing="ij")
    cub = lambda x, y, z: 0.02 * x ** 3 - 0.1 * x * y * z + 0.5 * y ** 2 - 0.03 * z ** 3 + x * z + 1.0
    o, pn, g = (4, 5, 6), (5, 4, 6), 1
    f = oracle.refine_cubic(cub(I, J, K), o, pn, g)
    loc = [o[a] + (np.arange(2 * pn[a] + 2 * g) - g + 0.5) / 2 for a in range(3)]
    X, Y, Z = np.meshgrid(*loc, indexing="ij")
    assert np.abs(f - cub(X, Y, Z)).max() < 1e-11
    # trilinear is not exact on the same cubic (the pin discriminates the two)
    assert np.abs(oracle.refine_interpolate(cub(I, J, K), o, pn, g) - cub(X, Y, Z)).max() > 1e-3


def test_refine_cubic_one_dimensional_weights():
    """1-D closed form: the fine child a quarter cell right of coarse centre i (w = 1/4 from i)
    gets (-7 phi_{i-1} + 105 phi_i + 35 phi_{i+1} - 5 phi_{i+2}) / 128."""
    nc = 16
    rng = np.random.default_rng(8)
    line = rng.standard_normal(nc)
    c = np.broadcast_to(line[:, None, None], (nc,) * 3).copy()
    f = oracle.refine_cubic(c, (0, 0, 0), (nc, 1, 1), 0)
    right = f[1::2, 0, 0]                       # fine cells at coarse coordinate i + 3/4
    ref = (-7 * np.roll(line, 1) + 105 * line + 35 * np.roll(line, -1) - 5 * np.roll(line, -2)) / 128
    assert np.abs(right - ref).max() < 1e-14


# ---------------------------------------------------------------- patch relaxation

def test_relax_patch_manufactured_dirichlet():
    pf, h, alpha, s, c = (10, 12, 8), 0.5, 0.08, 1.5, 0.02
    dims = tuple(x + 2 for x in pf)
    x = [(np.arange(dims[a]) - 0.5) * h for a in range(3)]
    X, Y, Z = np.meshgrid(*x, indexing="ij")
    phim = 0.05 * (np.sin(0.7 * X + 0.2) * np.cos(0.4 * Y) + 0.5 * np.cos(0.9 * Z - 0.3 * X))
    f = _pins.op_matrix_box(phim, h, alpha)
    delta = (f - c) / s
    start = phim.copy()
    rng = np.random.default_rng(5)
    start[1:-1, 1:-1, 1:-1] += 0.01 * rng.standard_normal(pf)
    out, nsw, rel = oracle.relax_patch(delta, start, alpha, s, h, c, tol=1e-12)
    assert rel <= 1e-12
    assert np.abs(out - phim).max() < 1e-10 * np.abs(phim).max() * 100
    # ghosts are untouched
    inner = np.zeros(dims, bool)
    inner[1:-1, 1:-1, 1:-1] = True
    assert np.array_equal(out[~inner], phim[~inner])


def test_patch_sweep_snapshot_semantics():
    pf, h, alpha, c = (6, 6, 6), 1.0, 0.2, 0.01
    dims = tuple(x + 2 for x in pf)
    rng = np.random.default_rng(7)
    phi0 = 0.1 * rng.standard_normal(dims)
    f = 0.05 * rng.standard_normal(pf)
    phi1 = oracle.patch_sweep(phi0, f, c, h, alpha)
    i = [np.arange(d) for d in dims]
    I, J, K = np.meshgrid(*i, indexing="ij")
    red = (I + J + K - 3) % 2 == 0
    mid = np.where(red, phi1, phi0)
    for _ in range(30):
        p = tuple(int(rng.integers(1, d - 1)) for d in dims)
        base = phi0.copy() if red[p] else mid.copy()
        base[p] = phi1[p]
        lhs = _pins.op_matrix_box(base, h, alpha)[tuple(q - 1 for q in p)]
        assert lhs == pytest.approx(f[tuple(q - 1 for q in p)] + c, abs=1e-12)


# --------------------------------------------------------------------------
# position-dependent truncation (Sec. 3.3): masked patch relaxation, parent mask
# --------------------------------------------------------------------------

def _masked_case(pf, seed, h=0.5, alpha=0.08, s=1.5, c=0.02):
    rng = np.random.default_rng(seed)
    dims = tuple(x + 2 for x in pf)
    box = 0.05 * rng.standard_normal(dims)
    delta = 0.2 * rng.standard_normal(pf)
    return box, delta, h, alpha, s, c


def test_relax_patch_masked_all_ones_is_relax_patch():
    box, delta, h, alpha, s, c = _masked_case((8, 10, 6), 11)
    ones = np.ones(delta.shape, np.uint8)
    a, na, ra = oracle.relax_patch(delta, box, alpha, s, h, c, tol=1e-9)
    b, nb, rb = oracle.relax_patch_masked(delta, box, ones, alpha, s, h, c, tol=1e-9)
    assert na == nb and ra == rb
    assert np.array_equal(a, b)


def test_relax_patch_masked_empty_mask_is_identity():
    box, delta, h, alpha, s, c = _masked_case((6, 6, 8), 12)
    out, nsw, rel = oracle.relax_patch_masked(delta, box, np.zeros(delta.shape, np.uint8),
                                              alpha, s, h, c, tol=1e-9)
    assert nsw == 0 and rel == 0.0
    assert np.array_equal(out, box)


def test_relax_patch_masked_box_is_sub_patch():
    """A mask that is one sub-box [a, b) of the interior relaxes exactly as that sub-box
    solved as its own patch, its ghost shell the surrounding (fixed) cells; the offset a has
    an even sum so the red-black colours agree."""
    pf = (12, 10, 14)
    box, delta, h, alpha, s, c = _masked_case(pf, 13)
    a, b = (1, 3, 2), (9, 9, 12)
    mask = np.zeros(pf, np.uint8)
    mask[a[0]:b[0], a[1]:b[1], a[2]:b[2]] = 1
    out, nsw, rel = oracle.relax_patch_masked(delta, box, mask, alpha, s, h, c, tol=1e-10)
    sub_box = box[a[0]:b[0] + 2, a[1]:b[1] + 2, a[2]:b[2] + 2]
    sub_delta = delta[a[0]:b[0], a[1]:b[1], a[2]:b[2]]
    ref, nref, rref = oracle.relax_patch(sub_delta, sub_box, alpha, s, h, c, tol=1e-10)
    assert nsw == nref and rel == rref and nsw > 0
    assert np.array_equal(out[a[0]:b[0] + 2, a[1]:b[1] + 2, a[2]:b[2] + 2], ref)
    keep = np.ones(box.shape, bool)
    keep[a[0] + 1:b[0] + 1, a[1] + 1:b[1] + 1, a[2] + 1:b[2] + 1] = False
    assert np.array_equal(out[keep], box[keep])


def test_relax_patch_masked_linear_matches_sparse_direct_solve():
    """alpha = 0: the masked problem is the 7-point Poisson equation on the masked cells
    with every other cell a known value; scipy's sparse direct solve gives it exactly."""
    sp = pytest.importorskip("scipy.sparse")
    spla = pytest.importorskip("scipy.sparse.linalg")
    pf = (8, 8, 10)
    box, delta, h, _, s, c = _masked_case(pf, 14)
    rng = np.random.default_rng(15)
    mask = (rng.random(pf) < 0.55).astype(np.uint8)
    out, nsw, rel = oracle.relax_patch_masked(delta, box, mask, 0.0, s, h, c, tol=1e-13)
    assert rel <= 1e-13
    act = np.argwhere(mask != 0)
    idx = -np.ones(pf, int)
    idx[tuple(act.T)] = np.arange(len(act))
    rows, cols, vals = [], [], []
    rhs = (s * delta[tuple(act.T)] + c) * h * h
    for r, p in enumerate(act):
        rows.append(r); cols.append(r); vals.append(-6.0)
        for d in range(3):
            for sg in (-1, 1):
                q = p.copy(); q[d] += sg
                inside = all(0 <= q[e] < pf[e] for e in range(3))
                if inside and mask[tuple(q)]:
                    rows.append(r); cols.append(int(idx[tuple(q)])); vals.append(1.0)
                else:
                    rhs[r] -= box[tuple(q + 1)]
    A = sp.csr_matrix((vals, (rows, cols)), shape=(len(act), len(act)))
    x = spla.spsolve(A, rhs)
    got = out[1:-1, 1:-1, 1:-1][tuple(act.T)]
    assert np.abs(got - x).max() < 1e-10 * max(1.0, np.abs(x).max())
    unmasked = np.ones(box.shape, bool)
    unmasked[1:-1, 1:-1, 1:-1] = mask != 0
    assert np.array_equal(out[~unmasked], box[~unmasked])


def test_relax_patch_masked_nonlinear_converges_on_mask():
    pf = (10, 8, 8)
    box, delta, h, alpha, s, c = _masked_case(pf, 16)
    rng = np.random.default_rng(17)
    mask = (rng.random(pf) < 0.4).astype(np.uint8)
    out, nsw, rel = oracle.relax_patch_masked(delta, box, mask, alpha, s, h, c, tol=1e-11)
    assert rel <= 1e-11 and nsw > 0
    r = s * delta + c - _pins.op_matrix_box(out, h, alpha)
    fm = np.where(mask != 0, s * delta, 0.0)
    assert np.linalg.norm(np.where(mask != 0, r, 0.0)) <= 1.5e-11 * np.linalg.norm(fm)
    # the masked-out cells still carry their (nonzero) residual: they were not iterated
    assert np.linalg.norm(np.where(mask == 0, r, 0.0)) > 1e3 * 1e-11 * np.linalg.norm(fm)


def test_parent_force_mask_places_children():
    """One parent cell with F5/F_GR above theta: exactly its 2x2x2 children are marked,
    at the fine indices the patch origin puts them (the patch wraps the periodic grid)."""
    nc, o, pn = 6, (4, 1, 5), (3, 2, 3)
    gphi = np.zeros((3, nc, nc, nc))
    ggr = np.ones((3, nc, nc, nc))
    # |F5| = |grad phi|/2; everywhere ratio 0.1, at coarse cell (0, 2, 0) ratio 0.5
    gphi[:] = 2 * 0.1
    gphi[:, 0, 2, 0] = 2 * 0.5
    m = oracle.parent_force_mask(gphi, ggr, o, pn, 0.3)
    assert m.shape == (6, 4, 6) and m.dtype == np.uint8
    # coarse (0, 2, 0) = patch-local (2, 1, 1): 0 = (4 + 2) mod 6, 2 = 1 + 1, 0 = (5 + 1) mod 6
    want = np.zeros((6, 4, 6), np.uint8)
    want[4:6, 2:4, 2:4] = 1
    assert np.array_equal(m, want)


def test_parent_force_mask_constant_ratio_and_zero_gravity():
    nc = 4
    rng = np.random.default_rng(18)
    ggr = rng.standard_normal((3, nc, nc, nc))
    gphi = 2 * 0.25 * ggr[[1, 2, 0]]           # |F5| = 0.25 |F_GR| (components permuted)
    o, pn = (0, 0, 0), (4, 4, 4)
    assert oracle.parent_force_mask(gphi, ggr, o, pn, 0.2).all()
    assert not oracle.parent_force_mask(gphi, ggr, o, pn, 0.3).any()
    # a refinement's interior as the parent (no wrap): the window of the periodic case
    m_per = oracle.parent_force_mask(gphi, ggr, (1, 0, 1), (2, 3, 3), 0.2 * 1.0)
    m_box = oracle.parent_force_mask(gphi, ggr, (1, 0, 1), (2, 3, 3), 0.2, periodic=False)
    assert np.array_equal(m_per, m_box)
    # F_GR = 0: iterated exactly where F5 != 0
    gphi2 = np.zeros_like(gphi)
    gphi2[0, 1, 1, 1] = 1e-30
    m = oracle.parent_force_mask(gphi2, np.zeros_like(ggr), o, pn, 0.5)
    assert m.sum() == 8 and m[2:4, 2:4, 2:4].all()


def test_parent_force_mask_box_parent_places_children():
    """A non-cubic refinement interior (5 x 6 x 7) as the parent: the children of a hand-placed
    parent (3, 1, 4) of the window starting at (2, 0, 3) sit at fine (2:4, 2:4, 2:4)."""
    pd = (5, 6, 7)
    gphi = np.full((3,) + pd, 2 * 0.1)
    ggr = np.ones((3,) + pd)
    gphi[:, 3, 1, 4] = 2 * 0.5
    gphi[:, 4, 5, 6] = 2 * 0.5          # outside the window: must not appear
    m = oracle.parent_force_mask(gphi, ggr, (2, 0, 3), (3, 2, 4), 0.3, periodic=False)
    want = np.zeros((6, 4, 8), np.uint8)
    want[2:4, 2:4, 2:4] = 1
    assert np.array_equal(m, want)


def test_vcycle_reduction_factor_poisson():
    """Sec. 3.1's point about multigrid (coarse grids remove the long-wavelength error that
    plain relaxation leaves behind) turned into a bound: for the Poisson limit (alpha = 0) each FAS
    V(2,2) cycle of the oracle reduces the residual by a factor <= 0.2, from the first cycle on
    (the smoothing-plus-coarse-correction rate, not a slow tail)."""
    delta = workload.lognormal_delta(32, 1.0, 9)
    phi, info = oracle.solve(delta, 0.0, 1.0, 1.0, tol=1e-12)
    h = [x for x in info.history if x > 0]
    assert info.status == 0 and len(h) >= 5
    ratios = [b / a for a, b in zip(h, h[1:])]
    assert max(ratios) <= 0.2, ratios
