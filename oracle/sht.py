"""Spherical-harmonic transform, written out from its definition (Section 3).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Definitions followed (Section 3, Eq. "spectral_to_physical_space" and the
two-step transform described right after it):

* Gaussian latitudes: mu_j are the nlat roots of the Legendre polynomial
  P_nlat, ordered north to south (mu descending), with Gauss weights
  w_j = 2 / ((1 - mu_j^2) P'_nlat(mu_j)^2).
* P_n^m is the associated Legendre function normalised so that its square
  integrates to 1 over mu in [-1, 1], without the Condon-Shortley phase
  (the paper only says "normalized"; this is the reading taken).
* Synthesis: xi(lambda, mu) = sum_m sum_n c_n^m P_n^m(mu) e^{i m lambda} over
  m = -T..T, with c^{-m} = conj(c^m); i.e. F_0 + 2 Re sum_{m>0} F_m e^{i m lambda}
  where F_m(mu) = sum_n c_n^m P_n^m(mu).
* Analysis: first a discrete Fourier transform in lambda,
  F_m(mu_j) = (1/nlon) sum_k xi(lambda_k, mu_j) e^{-i m lambda_k}, then the
  discrete Legendre transform c_n^m = sum_j w_j P_n^m(mu_j) F_m(mu_j).

Spectral arrays here are dense ``[..., m, n]`` complex128 with zeros for n < m;
``pack``/``unpack`` convert to the m-major triangular layout of the library
boundary.

Pins (tests/test_oracle_sht.py): nodes/weights against
``numpy.polynomial.legendre.leggauss`` and moment identities; P_n^m against
``scipy.special.lpmv`` and ``mpmath.legenp`` and quadrature orthonormality;
synthesis against brute-force double sums; analysis o synthesis = identity.
"""
from __future__ import annotations

import math

import numpy as np


# --------------------------------------------------------------------------
# Gaussian grid
# --------------------------------------------------------------------------

def _legendre_p_and_prev(N: int, x: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """P_N(x) and P_{N-1}(x) by the three-term (Bonnet) recurrence."""
    p_prev = np.ones_like(x)
    p = x.copy()
    if N == 0:
        return p_prev, np.zeros_like(x)
    for k in range(1, N):
        p_prev, p = p, ((2 * k + 1) * x * p - k * p_prev) / (k + 1)
    return p, p_prev


def gauss_legendre(nlat: int) -> tuple[np.ndarray, np.ndarray]:
    """Gaussian latitudes mu_j (descending) and weights w_j, by Newton iteration."""
    j = np.arange(nlat, dtype=np.float64)
    x = np.cos(math.pi * (j + 0.75) / (nlat + 0.5))
    for _ in range(100):
        p, pm1 = _legendre_p_and_prev(nlat, x)
        dp = nlat * (x * p - pm1) / (x * x - 1.0)
        dx = p / dp
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    p, pm1 = _legendre_p_and_prev(nlat, x)
    dp = nlat * (x * p - pm1) / (x * x - 1.0)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    return x, w


# --------------------------------------------------------------------------
# Normalised associated Legendre functions
# --------------------------------------------------------------------------

def epsilon(L: int) -> np.ndarray:
    """eps[m, n] = sqrt((n^2 - m^2) / (4 n^2 - 1)) for 0 <= m <= n < L, else 0."""
    eps = np.zeros((L, L))
    for m in range(L):
        for n in range(m, L):
            if n > 0:
                eps[m, n] = math.sqrt((n * n - m * m) / (4.0 * n * n - 1.0))
    return eps


def legendre_table(L: int, mu: np.ndarray) -> np.ndarray:
    """P[m, n, j] = normalised P_n^m(mu_j) for 0 <= m <= n < L (zero for n < m).

    Recurrences: P_0^0 = 1/sqrt(2); P_m^m = sqrt((2m+1)/(2m)) sqrt(1-mu^2)
    P_{m-1}^{m-1}; P_{m+1}^m = sqrt(2m+3) mu P_m^m; and for n >= m+2
    P_n^m = (mu P_{n-1}^m - eps_{n-1}^m P_{n-2}^m) / eps_n^m.  Every value
    is carried as a mantissa times an integer power of two (exact rescaling
    with frexp/ldexp), so that values below the double range (large m near
    the poles) come out as zeros instead of underflow noise.
    """
    mu = np.asarray(mu, dtype=np.float64)
    eps = epsilon(L)
    P = np.zeros((L, L, mu.size))
    sin_theta = np.sqrt((1.0 - mu) * (1.0 + mu))
    pmm, emm = np.frexp(np.full(mu.shape, 1.0 / math.sqrt(2.0)))
    emm = emm.astype(np.int64)
    for m in range(L):
        if m > 0:
            pmm = pmm * (math.sqrt((2 * m + 1) / (2.0 * m)) * sin_theta)
            pmm, e = np.frexp(pmm)
            emm = emm + e
        e_cur = emm.copy()
        p2 = np.zeros_like(mu)
        p1 = pmm.copy()
        for n in range(m, L):
            if n == m + 1:
                p2, p1 = p1, math.sqrt(2 * m + 3) * mu * p1
            elif n > m + 1:
                p2, p1 = p1, (mu * p1 - eps[m, n - 1] * p2) / eps[m, n]
            big = np.abs(p1) > 2.0 ** 400
            if np.any(big):
                p1 = np.where(big, np.ldexp(p1, -400), p1)
                p2 = np.where(big, np.ldexp(p2, -400), p2)
                e_cur = np.where(big, e_cur + 400, e_cur)
            P[m, n] = np.ldexp(p1, np.clip(e_cur, -2000, 2000))
    return P


# --------------------------------------------------------------------------
# Transform
# --------------------------------------------------------------------------

class SHT:
    """Spectral transform at truncation T on an nlat x nlon Gaussian grid.

    ``L`` is the number of orders/degrees kept in the tables (default T+2, so
    that the velocity fields U, V of degree T+1 can be synthesised).
    """

    def __init__(self, T: int, nlat: int, nlon: int, L: int | None = None):
        self.T, self.nlat, self.nlon = T, nlat, nlon
        self.L = T + 2 if L is None else L
        if not (2 * (self.L - 1) < nlon):
            raise ValueError("nlon too small for the truncation")
        self.mu, self.w = gauss_legendre(nlat)
        self.lam = 2.0 * math.pi * np.arange(nlon) / nlon
        self.P = legendre_table(self.L, self.mu)
        self.eps = epsilon(self.L + 1)

    def synthesis(self, c: np.ndarray) -> np.ndarray:
        """Dense [..., m, n] (m, n < L) -> real grid [..., nlat, nlon]."""
        L = c.shape[-1]
        F = np.einsum("...mn,mnj->...jm", c, self.P[:L, :L])
        X = np.zeros(F.shape[:-1] + (self.nlon // 2 + 1,), dtype=np.complex128)
        X[..., :L] = F
        X[..., 0] = X[..., 0].real
        return self.nlon * np.fft.irfft(X, n=self.nlon, axis=-1)

    def analysis(self, g: np.ndarray, L: int | None = None) -> np.ndarray:
        """Real grid [..., nlat, nlon] -> dense [..., m, n] with m, n < L."""
        L = self.L if L is None else L
        F = np.fft.rfft(g, axis=-1)[..., :L] / self.nlon           # [..., j, m]
        return np.einsum("...jm,mnj,j->...mn", F, self.P[:L, :L], self.w)


# --------------------------------------------------------------------------
# Layout helpers (library boundary convention)
# --------------------------------------------------------------------------

def synthesis_rows(c: np.ndarray, mu: np.ndarray, nlon: int) -> np.ndarray:
    """The synthesis of Section 3 evaluated on chosen latitudes only.

    Dense coefficients c [..., m, n] -> real grid rows [..., len(mu), nlon]
    at the points (lambda_k = 2 pi k / nlon, mu): the same definition as
    SHT.synthesis, with the Legendre table built for the requested mu alone,
    so that sample rows of a high truncation cost a single table column.
    """
    L = c.shape[-1]
    P = legendre_table(L, np.atleast_1d(np.asarray(mu, dtype=np.float64)))
    F = np.einsum("...mn,mnj->...jm", c, P)
    X = np.zeros(F.shape[:-1] + (nlon // 2 + 1,), dtype=np.complex128)
    X[..., :L] = F
    X[..., 0] = X[..., 0].real
    return nlon * np.fft.irfft(X, n=nlon, axis=-1)


def pack(c: np.ndarray, T: int) -> np.ndarray:
    """Dense [..., m, n] -> packed m-major triangle [..., (T+1)(T+2)/2]."""
    parts = [c[..., m, m:T + 1] for m in range(T + 1)]
    return np.concatenate(parts, axis=-1)


def unpack(v: np.ndarray, T: int, L: int | None = None) -> np.ndarray:
    """Packed triangle [..., ncoef] -> dense [..., L, L] (L >= T+1)."""
    L = T + 1 if L is None else L
    out = np.zeros(v.shape[:-1] + (L, L), dtype=np.complex128)
    off = 0
    for m in range(T + 1):
        k = T + 1 - m
        out[..., m, m:T + 1] = v[..., off:off + k]
        off += k
    return out


def area_mean_square(c: np.ndarray) -> np.ndarray:
    """Area-mean of the square of a real field given dense coefficients."""
    wt = np.ones(c.shape[-2])
    wt[1:] = 2.0
    return 0.5 * np.einsum("m,...mn->...", wt, np.abs(c) ** 2)
