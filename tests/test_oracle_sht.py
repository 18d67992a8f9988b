"""Pins of the oracle's spherical-harmonic transform against things other than itself.

Section 3: Gaussian latitudes, normalised associated Legendre functions,
two-step transform.  Each test checks the oracle against an independent
library, a closed form or a brute-force sum.
"""
import math

import mpmath
import numpy as np
import pytest
from scipy.special import lpmv

from oracle.sht import synthesis_rows, SHT, gauss_legendre, legendre_table, pack, unpack, area_mean_square
import synthetic as syn


def pbar_lpmv(m, n, x):
    """Orthonormal P_n^m from scipy (removes scipy's Condon-Shortley phase)."""
    norm = math.sqrt((2 * n + 1) / 2.0 * math.exp(math.lgamma(n - m + 1) - math.lgamma(n + m + 1)))
    return (-1) ** m * norm * lpmv(m, n, x)


@pytest.mark.parametrize("nlat", [2, 7, 48, 96, 384])
def test_gauss_nodes_match_numpy_leggauss(nlat):
    mu, w = gauss_legendre(nlat)
    x, wx = np.polynomial.legendre.leggauss(nlat)
    assert np.all(np.diff(mu) < 0), "north to south ordering"
    assert np.max(np.abs(mu - x[::-1])) < 1e-15
    # numpy's own polar weights are only good to ~4e-10 relative at nlat=384
    assert np.max(np.abs(w - wx[::-1]) / wx[::-1]) < 1e-9


@pytest.mark.parametrize("nlat", [384, 1920])
def test_gauss_nodes_and_weights_match_50_digit_newton(nlat):
    mpmath.mp.dps = 50
    mu, w = gauss_legendre(nlat)

    def P(t):
        p0, p1 = mpmath.mpf(1), t
        for k in range(1, nlat):
            p0, p1 = p1, ((2 * k + 1) * t * p1 - k * p0) / (k + 1)
        return p1, p0

    for j in [0, nlat // 3, nlat // 2 - 1]:
        r = mpmath.mpf(mu[j])
        for _ in range(4):
            p, pm = P(r)
            r = r - p / (nlat * (r * p - pm) / (r * r - 1))
        p, pm = P(r)
        dp = nlat * (r * p - pm) / (r * r - 1)
        wr = float(2 / ((1 - r * r) * dp * dp))
        assert abs(float(r) - mu[j]) < 1e-16
        assert abs(w[j] - wr) < 1e-10 * wr


def test_gauss_moments_and_symmetry():
    nlat = 96
    mu, w = gauss_legendre(nlat)
    for k in range(2 * nlat):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.sum(w * mu ** k) - exact) < 1e-14
    assert np.max(np.abs(mu + mu[::-1])) < 1e-15
    assert np.max(np.abs(w - w[::-1])) < 1e-15


def test_legendre_matches_scipy_lpmv():
    mu, _ = gauss_legendre(64)
    P = legendre_table(41, mu)
    err = 0.0
    for m in range(41):
        for n in range(m, 41):
            err = max(err, np.max(np.abs(P[m, n] - pbar_lpmv(m, n, mu))))
    assert err < 1e-12


_HIGH_MU = np.array([0.7, 0.5, 0.1, -0.37])


@pytest.fixture(scope="module")
def high_degree_table():
    return legendre_table(1280, _HIGH_MU)


@pytest.mark.parametrize("n,m", [(1279, 1000), (700, 3), (255, 255), (256, 128), (511, 300)])
def test_legendre_matches_mpmath_high_degree(high_degree_table, n, m):
    """40-digit hypergeometric evaluation (mpmath), far beyond scipy's range."""
    mpmath.mp.dps = 40
    P = high_degree_table[m, n]
    for x, got in zip(_HIGH_MU, P):
        norm = mpmath.sqrt(mpmath.mpf(2 * n + 1) / 2 * mpmath.factorial(n - m) / mpmath.factorial(n + m))
        ref = (-1) ** m * norm * mpmath.legenp(n, m, mpmath.mpf(x), type=2,
                                               maxprec=200000, maxterms=10**6)
        ref = float(ref)
        if abs(ref) > 1e-250:
            assert abs(got - ref) <= 1e-11 * max(1.0, abs(ref)), (x, got, ref)
        else:
            assert abs(got) < 1e-240


def test_legendre_orthonormal_under_gauss_quadrature():
    T = 63
    nlat, _ = syn.gaussian_grid_size(T)
    mu, w = gauss_legendre(nlat)
    L = T + 3
    P = legendre_table(L, mu)
    G = np.einsum("mnj,mkj,j->mnk", P, P, w)
    for m in range(L):
        I = np.eye(L)
        I[:m, :m] = 0.0
        assert np.max(np.abs(G[m] - I)) < 1e-13


def test_legendre_large_m_polar_underflow_is_clean():
    mu, w = gauss_legendre(1920)
    P = legendre_table(1281, mu[:3])
    assert np.all(np.isfinite(P))
    assert np.all(P[1279, 1279] == 0.0)


def brute_force_synthesis(c, T, mu, lam):
    g = np.zeros((mu.size, lam.size))
    for m in range(T + 1):
        for n in range(m, T + 1):
            Pm = pbar_lpmv(m, n, mu)[:, None]
            if m == 0:
                g += c[m, n].real * Pm
            else:
                g += 2.0 * Pm * (c[m, n].real * np.cos(m * lam)[None] - c[m, n].imag * np.sin(m * lam)[None])
    return g


@pytest.mark.parametrize("T", [5, 10, 15])
def test_synthesis_matches_brute_force_sum(T):
    nlat, nlon = syn.gaussian_grid_size(T)
    s = SHT(T, nlat, nlon, L=T + 1)
    c = unpack(syn.random_spectrum(T, (1,), seed=11, nmin=0)[0], T)
    g = s.synthesis(c)
    ref = brute_force_synthesis(c, T, s.mu, s.lam)
    assert np.max(np.abs(g - ref)) < 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("T", [7, 15])
def test_synthesis_rows_match_brute_force_sum_at_arbitrary_latitudes(T):
    """Rows at points that are not Gaussian latitudes (the table is built for
    the requested mu alone) against the brute-force double sum."""
    nlon = 4 * (T + 1)
    mu = np.array([0.93, -0.41, 0.05, -0.999])
    lam = 2.0 * np.pi * np.arange(nlon) / nlon
    c = unpack(syn.random_spectrum(T, (1,), seed=12, nmin=0)[0], T)
    g = synthesis_rows(c, mu, nlon)
    ref = brute_force_synthesis(c, T, mu, lam)
    assert g.shape == (mu.size, nlon)
    assert np.max(np.abs(g - ref)) < 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("T", [15, 63])
def test_analysis_inverts_synthesis(T):
    nlat, nlon = syn.gaussian_grid_size(T)
    s = SHT(T, nlat, nlon)
    c = unpack(syn.random_spectrum(T, (2,), seed=3, nmin=0), T, L=T + 2)
    c2 = s.analysis(s.synthesis(c))
    assert np.max(np.abs(c2 - c)) < 1e-13 * np.max(np.abs(c))


def test_analysis_of_brute_force_grid():
    """Analysis of an independently synthesised grid recovers the coefficients."""
    T = 10
    nlat, nlon = syn.gaussian_grid_size(T)
    s = SHT(T, nlat, nlon, L=T + 1)
    c = unpack(syn.random_spectrum(T, (1,), seed=5, nmin=0)[0], T)
    g = brute_force_synthesis(c, T, s.mu, s.lam)
    assert np.max(np.abs(s.analysis(g) - c)) < 1e-13 * np.max(np.abs(c))


def test_area_mean_square_matches_quadrature():
    T = 21
    nlat, nlon = syn.gaussian_grid_size(T)
    s = SHT(T, nlat, nlon, L=T + 1)
    c = unpack(syn.random_spectrum(T, (1,), seed=8, rms=3.0)[0], T)
    g = s.synthesis(c)
    quad = 0.5 * np.sum(s.w[:, None] * g * g) / nlon
    assert abs(quad - area_mean_square(c)) < 1e-13 * quad
    assert abs(math.sqrt(quad) - 3.0) < 1e-12


def test_pack_unpack_layout():
    T = 7
    v = np.arange(syn.ncoef(T)) + 0j
    d = unpack(v, T)
    for m in range(T + 1):
        for n in range(m, T + 1):
            assert d[m, n] == syn.packed_index(m, n, T)
    assert np.array_equal(pack(d, T), v)
