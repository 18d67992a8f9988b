"""Pins of the oracle's shallow-water operators (Sections 2, 4, 5.4).

Analytic steady states, conservation, closed-form velocity recovery, and a
brute-force evaluation of the nonlinear operator from grid derivatives
computed with an independent Legendre derivative identity.
"""
import math

import numpy as np
import pytest
from scipy.special import lpmv

from oracle.sht import SHT, unpack, gauss_legendre
from oracle.swe import (SWEParams, rhs, velocity_coefficients, div_curl, implicit_solve,
                        linear_part, nonlinear_part, kappa, coriolis_linear)
import synthetic as syn

A = syn.EARTH_RADIUS


def params(nu=0.0, omega=syn.OMEGA, phibar=syn.GRAVITY * syn.MEAN_DEPTH):
    return SWEParams(a=A, omega=omega, g=syn.GRAVITY, nu=nu, phibar=phibar)


def level(T):
    nlat, nlon = syn.gaussian_grid_size(T)
    return SHT(T, nlat, nlon)


@pytest.mark.parametrize("T", [15, 63])
def test_balanced_zonal_jet_is_steady(T):
    s = level(T)
    st = unpack(syn.zonal_jet(T), T)
    FE, FI = rhs(st, s, params())
    assert np.max(np.abs(FE + FI)) < 1e-11 * np.max(np.abs(FI))
    assert np.max(np.abs(FI)) > 1e-12


def test_tilted_solid_body_rotation_is_steady_without_coriolis():
    T = 15
    s = level(T)
    e = syn.solid_body_axis(seed=21)
    u0, phi0 = 30.0, 5.0e4
    mu = s.mu[:, None]
    cphi = np.sqrt(1 - mu * mu)
    lam = s.lam[None, :]
    er = e[0] * cphi * np.cos(lam) + e[1] * cphi * np.sin(lam) + e[2] * mu   # e . r
    zeta_g = 2.0 * u0 * er / A
    phi_g = phi0 - 0.5 * u0 * u0 * er * er
    st = np.zeros((3, T + 1, T + 1), dtype=complex)
    st[0] = s.analysis(phi_g, T + 1)
    st[1] = s.analysis(zeta_g, T + 1)
    p = params(omega=0.0, phibar=phi0)
    FE, FI = rhs(st, s, p)
    # scale of each tendency's individual terms: Phi' V / a, zeta V / a, lap Phi
    scales = [0.5 * u0 ** 3 / A, 2 * u0 * u0 / A ** 2, np.max(np.abs(FI[2]))]
    for f in range(3):
        assert np.max(np.abs(FE[f] + FI[f])) < 1e-11 * scales[f], f
    # exercises m = 0, 1, 2
    assert np.abs(st[0, 2, 2]) > 1e-3 * np.abs(st[0, 0, 2])


def test_mass_and_circulation_tendencies_vanish():
    T = 21
    s = level(T)
    st = unpack(syn.zonal_jet(T), T) + unpack(
        syn.random_spectrum(T, (3,), seed=5, rms=1e-5), T) * np.array([1e4, 1, 1])[:, None, None]
    FE = nonlinear_part(st, s, params())
    assert FE[0, 0, 0] == 0.0 and FE[1, 0, 0] == 0.0
    assert np.max(np.abs(FE[0])) > 0.0


def test_velocity_of_solid_body_vorticity_and_potential():
    T = 10
    s = level(T)
    u0 = 20.0
    zeta = np.zeros((T + 1, T + 1), complex)
    delta = np.zeros_like(zeta)
    zeta[0, 1] = 2.0 * u0 / (A * math.sqrt(1.5))          # zeta = 2 u0 mu / a
    U, V = velocity_coefficients(zeta, delta, A)
    one_m = (1 - s.mu ** 2)[:, None]
    assert np.max(np.abs(s.synthesis(U) - u0 * one_m)) < 1e-13 * u0
    assert np.max(np.abs(s.synthesis(V))) < 1e-13 * u0
    # chi = a u0 mu  =>  delta = -2 u0 mu / a, V = u0 (1 - mu^2), U = 0
    zeta[:] = 0
    delta[0, 1] = -2.0 * u0 / (A * math.sqrt(1.5))
    U, V = velocity_coefficients(zeta, delta, A)
    assert np.max(np.abs(s.synthesis(V) - u0 * one_m)) < 1e-13 * u0
    assert np.max(np.abs(s.synthesis(U))) < 1e-13 * u0


def test_div_curl_of_recovered_velocity_gives_back_delta_zeta():
    T = 31
    s = level(T)
    zd = unpack(syn.random_spectrum(T, (2,), seed=9, rms=1e-5), T)
    U, V = velocity_coefficients(zd[0], zd[1], A)
    one_m = (1 - s.mu ** 2)[:, None]
    Ah = s.analysis(s.synthesis(U) / one_m, T + 2)
    Bh = s.analysis(s.synthesis(V) / one_m, T + 2)
    div, curl = div_curl(Ah, Bh, A, T)
    assert np.max(np.abs(curl - zd[0])) < 1e-12 * np.max(np.abs(zd[0]))
    assert np.max(np.abs(div - zd[1])) < 1e-12 * np.max(np.abs(zd[1]))


# ---------------------------------------------------------------------------
# Brute force: N(U) from grid derivatives (independent derivative identity)
# ---------------------------------------------------------------------------

def _pbar(m, n, x):
    norm = math.sqrt((2 * n + 1) / 2.0 * math.exp(math.lgamma(n - m + 1) - math.lgamma(n + m + 1)))
    return (-1) ** m * norm * lpmv(m, n, x)


def _dpbar(m, n, x):
    """d/dmu of P_n^m from the classical identity
    (x^2 - 1) dP_n^m/dx = n x P_n^m - (n + m) P_{n-1}^m (unnormalised)."""
    norm = math.sqrt((2 * n + 1) / 2.0 * math.exp(math.lgamma(n - m + 1) - math.lgamma(n + m + 1)))
    prev = lpmv(m, n - 1, x) if n - 1 >= m else 0.0 * x
    d = (n * x * lpmv(m, n, x) - (n + m) * prev) / (x * x - 1.0)
    return (-1) ** m * norm * d


def _field(c, mu, lam, deriv=None):
    """Field (or d/dlam, d/dmu) from dense coefficients by direct sums."""
    out = np.zeros((mu.size, lam.size))
    Lm, Ln = c.shape
    for m in range(Lm):
        for n in range(m, Ln):
            if c[m, n] == 0:
                continue
            P = (_dpbar(m, n, mu) if deriv == "mu" else _pbar(m, n, mu))[:, None]
            e = np.exp(1j * m * lam)[None, :]
            term = c[m, n] * P * (1j * m * e if deriv == "lam" else e)
            out += (1.0 if m == 0 else 2.0) * term.real
    return out


def _project(g, mu, w, lam, L):
    """Galerkin coefficients of a grid field by direct quadrature sums."""
    nlon = lam.size
    c = np.zeros((L, L), complex)
    for m in range(L):
        Fm = (g * np.exp(-1j * m * lam)[None, :]).sum(axis=1) / nlon
        for n in range(m, L):
            c[m, n] = np.sum(w * _pbar(m, n, mu) * Fm)
    return c


def test_nonlinear_operator_matches_brute_force_grid_derivatives():
    T = 6
    p = params(omega=syn.OMEGA)
    s = level(T)
    st = unpack(syn.zonal_jet(T), T) + unpack(
        syn.random_spectrum(T, (3,), seed=17, rms=1e-5), T) * np.array([3e3, 1, 1])[:, None, None]
    got = nonlinear_part(st, s, p)
    # high-order reference grid: exact for all products involved
    nlat, nlon = 40, 80
    mu, w = gauss_legendre(nlat)
    lam = 2 * math.pi * np.arange(nlon) / nlon
    one_m = (1 - mu * mu)[:, None]
    U, V = velocity_coefficients(st[1], st[2], A)
    Ug, Vg = _field(U, mu, lam), _field(V, mu, lam)
    Ug_l, Vg_l = _field(U, mu, lam, "lam"), _field(V, mu, lam, "lam")
    Ug_m, Vg_m = _field(U, mu, lam, "mu"), _field(V, mu, lam, "mu")
    eta = _field(st[1], mu, lam) + 2 * p.omega * mu[:, None]
    eta_l, eta_m = _field(st[1], mu, lam, "lam"), _field(st[1], mu, lam, "mu") + 2 * p.omega
    php = _field(st[0], mu, lam) - p.phibar
    php_l, php_m = _field(st[0], mu, lam, "lam"), _field(st[0], mu, lam, "mu")

    def div(Ag, Ag_l, Bg, Bg_m):
        return (Ag_l + one_m * Bg_m) / (A * one_m)

    def curl(Ag, Ag_m, Bg, Bg_l):
        return (Bg_l - one_m * Ag_m) / (A * one_m)

    # products and their derivatives (product rule)
    A1, A1_l, A1_m = eta * Ug, eta_l * Ug + eta * Ug_l, eta_m * Ug + eta * Ug_m
    B1, B1_l, B1_m = eta * Vg, eta_l * Vg + eta * Vg_l, eta_m * Vg + eta * Vg_m
    A2, A2_l = php * Ug, php_l * Ug + php * Ug_l
    B2, B2_m = php * Vg, php_m * Vg + php * Vg_m
    E = (Ug * Ug + Vg * Vg) / (2 * one_m)
    L = T + 1
    k = kappa(L, A)
    ref = np.zeros((3, L, L), complex)
    ref[0] = -_project(div(A2, A2_l, B2, B2_m), mu, w, lam, L)
    ref[1] = -_project(div(A1, A1_l, B1, B1_m), mu, w, lam, L)
    ref[2] = _project(curl(A1, A1_m, B1, B1_l), mu, w, lam, L) + k * _project(E, mu, w, lam, L)
    for f in range(3):
        scale = np.max(np.abs(ref[f]))
        assert np.max(np.abs(got[f] - ref[f])) < 1e-10 * scale, f


def test_implicit_solve_against_dense_linear_algebra():
    T = 12
    p = params(nu=1e5)
    h = 37.5
    b = unpack(syn.random_spectrum(T, (3,), seed=4, nmin=0), T)
    x = implicit_solve(b, h, p)
    # residual of the system of Section 5.4, relative to the size of its terms
    hLx = h * linear_part(x, p)
    scale = np.max(np.abs(x)) + np.max(np.abs(hLx)) + np.max(np.abs(b))
    assert np.max(np.abs(x - hLx - b)) < 1e-14 * scale
    # per-coefficient 3x3 matrix assembled from the linear operator, solved by LAPACK
    for (m, n) in [(0, 0), (0, 1), (3, 7), (12, 12)]:
        Mx = np.zeros((3, 3))
        for f in range(3):
            e = np.zeros((3, T + 1, T + 1), complex)
            e[f, m, n] = 1.0
            Mx[:, f] = (e - h * linear_part(e, p))[:, m, n].real
        ref = np.linalg.solve(Mx, b[:, m, n])
        assert np.max(np.abs(ref - x[:, m, n])) <= 1e-13 * np.max(np.abs(ref))


# ---------------------------------------------------------------------------
# Coriolis term in the implicit part (F_I = L + C, F_E = N with eta = zeta)
# ---------------------------------------------------------------------------
def cparams(nu=0.0, omega=syn.OMEGA):
    return SWEParams(a=A, omega=omega, g=syn.GRAVITY, nu=nu, phibar=syn.GRAVITY * syn.MEAN_DEPTH,
                     coriolis_implicit=True)


def _state(T, seed, nmin=0):
    return unpack(syn.random_spectrum(T, (3,), seed=seed, rms=1e-5, nmin=nmin), T) * np.array(
        [1e4, 1, 1])[:, None, None]


@pytest.mark.parametrize("T", [10, 21])
def test_coriolis_operator_is_the_transform_difference_of_f(T):
    """C from mu-multiplication and the recovered U, V against the
    transform-method route: N with eta = zeta + f minus N with eta = zeta
    (grid products f U, f V, analysed and differentiated).  Random states
    include the n = 0 coefficients, which must not enter."""
    s = level(T)
    st = _state(T, 31 + T)
    C = coriolis_linear(st, params())
    diff = nonlinear_part(st, s, params()) - nonlinear_part(st, s, params(omega=0.0))
    assert np.max(np.abs(C[0])) == 0.0
    for f in (1, 2):
        assert np.max(np.abs(C[f] - diff[f])) < 1e-11 * np.max(np.abs(diff[f])), f


def test_coriolis_operator_conserves_kinetic_energy():
    """The Coriolis force does no work: with KE = sum a^2 (|zeta_n|^2 +
    |delta_n|^2) / (n(n+1)) per order, Re sum (conj(zeta) C_zeta +
    conj(delta) C_delta) / (n(n+1)) = 0 for every order m separately."""
    T = 21
    st = _state(T, 5)
    C = coriolis_linear(st, params())
    n = np.arange(T + 1, dtype=float)
    w = np.zeros(T + 1)
    w[1:] = 1.0 / (n[1:] * (n[1:] + 1.0))
    terms = w * (np.conj(st[1]) * C[1] + np.conj(st[2]) * C[2])
    per_m = terms.sum(axis=-1).real
    scale = (w * (np.abs(st[1]) * np.abs(C[1]) + np.abs(st[2]) * np.abs(C[2]))).sum(axis=-1)
    assert np.all(np.abs(per_m) <= 1e-13 * scale.max())
    assert scale.max() > 0.0


@pytest.mark.parametrize("m,n", [(1, 1), (3, 5), (7, 12)])
def test_coriolis_operator_gives_the_rossby_haurwitz_frequency(m, n):
    """A single vorticity harmonic zeta_n^m: the vorticity tendency of C is
    i 2 Omega m / (n(n+1)) zeta_n^m and nothing else (the beta term; the
    classical Rossby-Haurwitz dispersion relation), while the divergence
    tendency lives on degrees n - 1 and n + 1 only."""
    T = 15
    st = np.zeros((3, T + 1, T + 1), complex)
    st[1, m, n] = 0.3 - 0.7j
    C = coriolis_linear(st, params())
    expect = np.zeros((T + 1, T + 1), complex)
    expect[m, n] = 1j * 2.0 * syn.OMEGA * m / (n * (n + 1.0)) * st[1, m, n]
    assert np.max(np.abs(C[1] - expect)) <= 1e-15 * np.abs(expect[m, n])
    mask = np.zeros((T + 1, T + 1), bool)
    mask[m, [d for d in (n - 1, n + 1) if m <= d <= T]] = True
    assert np.max(np.abs(C[2][~mask])) == 0.0
    assert np.max(np.abs(C[2][mask])) > 0.0


@pytest.mark.parametrize("T", [15, 63])
def test_balanced_jet_is_steady_with_implicit_coriolis(T):
    """The sum F_E + F_I does not depend on the split.  F_I = L + C nearly
    cancels itself for this geostrophically balanced flow, so the scale is
    the gravity-wave term L alone."""
    s = level(T)
    st = unpack(syn.zonal_jet(T), T)
    FE, FI = rhs(st, s, cparams())
    scale = np.max(np.abs(linear_part(st, params())))
    assert np.max(np.abs(FE + FI)) < 1e-11 * scale
    assert np.max(np.abs(FI)) < 0.1 * scale     # the gradient-wind remainder (Rossby number ~ 0.03)


def test_implicit_solve_with_coriolis():
    """x - h (L + C)(x) = b by the per-order dense solve: residual through the
    operator, and Omega = 0 reduces to the per-coefficient solve."""
    T = 12
    h = 37.5
    b = _state(T, 6)
    p = cparams(nu=1e5)
    x = implicit_solve(b, h, p)
    hFx = h * linear_part(x, p)
    scale = np.max(np.abs(x)) + np.max(np.abs(hFx)) + np.max(np.abs(b))
    assert np.max(np.abs(x - hFx - b)) < 1e-14 * scale
    # the Coriolis coupling is felt at this step size
    assert np.max(np.abs(x - implicit_solve(b, h, params(nu=1e5)))) > 1e-6 * np.max(np.abs(x))
    x0 = implicit_solve(b, h, cparams(nu=1e5, omega=0.0))
    assert np.max(np.abs(x0 - implicit_solve(b, h, params(nu=1e5, omega=0.0)))) <= 1e-14 * np.max(np.abs(x0))


def test_sdc_collocation_solution_does_not_depend_on_the_split():
    """Iterated to convergence, IMEX-SDC solves the collocation problem of
    dU/dt = F_E + F_I, which is the same for both splits: one step of 600 s,
    5 Lobatto nodes, 30 sweeps."""
    from oracle.sdc import SDCLevel, sdc_step
    T = 10
    nlat, nlon = syn.gaussian_grid_size(T)
    st = unpack(syn.zonal_jet(T), T) + _state(T, 9, nmin=1)
    a = sdc_step(SDCLevel(T, nlat, nlon, 5, 600.0, params(nu=1e5)), st, 30)
    b = sdc_step(SDCLevel(T, nlat, nlon, 5, 600.0, cparams(nu=1e5)), st, 30)
    change = np.linalg.norm(a - st)
    assert np.linalg.norm(a - b) < 1e-11 * change
