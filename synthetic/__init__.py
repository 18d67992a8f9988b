"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds no arithmetic of the method itself: it only draws random
spectra, writes down closed-form spectral coefficients of analytic initial
states, and evaluates an analytic height bump at caller-supplied points.
Everything that transforms, differentiates or integrates lives on either side
of the parity boundary, never here.

Conventions (shared by both sides as an interface, not as code):

* A scalar field truncated at degree ``T`` is stored as ``ncoef(T) =
  (T+1)(T+2)/2`` complex coefficients in m-major triangular order: the
  coefficient of order ``m`` and degree ``n`` (``m <= n <= T``) sits at
  ``m*(2T+3-m)//2 + (n-m)``.  Coefficients with ``m = 0`` are real.
* The basis is the orthonormal associated Legendre function (integral of its
  square over mu in [-1, 1] is 1, no Condon-Shortley phase) times
  ``exp(i m lambda)``; a real field is ``sum_n c_n^0 P_n^0 + 2 Re sum_{m>0}
  c_n^m P_n^m e^{i m lambda}`` (Section 3, Eq. "spectral_to_physical_space").
  Its area-mean square is therefore ``(sum_n |c_n^0|^2 + 2 sum_{m>0}
  |c_n^m|^2) / 2``.
* A shallow-water state is ``[Phi, zeta, delta]`` (Section 2), shape
  ``[..., 3, ncoef]`` complex128.
"""
from __future__ import annotations

import math

import numpy as np

# Physical constants of the workloads (Earth values; the paper cites
# Swarztrauber 2004 for them without printing them).
EARTH_RADIUS = 6.37122e6      # a  [m]
OMEGA = 7.292e-5              # Omega [1/s]
GRAVITY = 9.80616             # g  [m/s^2]
NU = 1.0e5                    # second-order diffusion [m^2/s] (Section 6)
MEAN_DEPTH = 1.0e4            # h-bar of the balanced-jet workloads [m]


def ncoef(T: int) -> int:
    """Number of complex coefficients of one field truncated at degree T."""
    return (T + 1) * (T + 2) // 2


def packed_index(m: int, n: int, T: int) -> int:
    """Offset of coefficient (m, n) in the m-major triangular layout."""
    return m * (2 * T + 3 - m) // 2 + (n - m)


def gaussian_grid_size(T: int) -> tuple[int, int]:
    """Grid used by the workloads: nlat = 3(T+1)/2 rounded up to even, nlon = 2 nlat."""
    nlat = -(-3 * (T + 1) // 2)
    nlat += nlat % 2
    return nlat, 2 * nlat


def _degree_of_each_coefficient(T: int) -> tuple[np.ndarray, np.ndarray]:
    ms, ns = [], []
    for m in range(T + 1):
        for n in range(m, T + 1):
            ms.append(m)
            ns.append(n)
    return np.array(ms), np.array(ns)


def area_rms(spec: np.ndarray, T: int) -> np.ndarray:
    """Area-rms of packed real fields (last axis = coefficients)."""
    ms, _ = _degree_of_each_coefficient(T)
    wt = np.where(ms == 0, 1.0, 2.0)
    return np.sqrt(0.5 * np.sum(wt * np.abs(spec) ** 2, axis=-1))


def random_spectrum(T: int, shape: tuple, seed: int, *, slope: float = -3.0,
                    rms: float = 1.0, nmin: int = 1, nmax: int | None = None
                    ) -> np.ndarray:
    """Random real fields with per-degree power proportional to n**slope.

    Draw order (PCG64 ``default_rng(seed)``): for every field in C order of
    ``shape``, for m = 0..T, for n = m..T, one (re, im) pair of standard
    normals.  Per-coefficient standard deviation sqrt(n**slope / (2n+1)) makes
    the power summed over the 2n+1 orders of degree n go as n**slope.  Degrees
    outside [nmin, nmax] are zero, m = 0 coefficients are made real, and each
    field is rescaled to the requested area-rms.
    """
    nmax = T if nmax is None else nmax
    rng = np.random.default_rng(seed)
    nf = int(np.prod(shape)) if shape else 1
    ms, ns = _degree_of_each_coefficient(T)
    draws = rng.standard_normal((nf, ncoef(T), 2))
    z = draws[..., 0] + 1j * draws[..., 1]
    nn = ns.astype(np.float64)
    keep = (ns >= nmin) & (ns <= nmax) & (ns >= 1)
    std = np.zeros_like(nn)
    std[keep] = np.sqrt(nn[keep] ** slope / (2.0 * nn[keep] + 1.0))
    z = z * std
    z[:, ms == 0] = z[:, ms == 0].real
    cur = area_rms(z, T)
    z = z * (rms / np.where(cur > 0, cur, 1.0))[:, None]
    return z.reshape(tuple(shape) + (ncoef(T),))


def zonal_jet(T: int, *, u0: float = 20.0, a: float = EARTH_RADIUS,
              omega: float = OMEGA, g: float = GRAVITY,
              hbar: float = MEAN_DEPTH) -> np.ndarray:
    """Spectral [Phi, zeta, delta] of the balanced zonal flow u = u0 cos(phi).

    Closed form: zeta = 2 u0 mu / a and, from the meridional balance
    (f + u tan(phi)/a) u = -(1/a) dPhi/dphi, Phi = g hbar + C/3 - C mu^2 with
    C = a Omega u0 + u0^2/2 (area mean g hbar).  In the orthonormal basis
    1 = sqrt(2) P_0^0, mu = P_1^0 / sqrt(3/2), mu^2 - 1/3 = (2/3) P_2^0 / sqrt(5/2).
    """
    s = np.zeros((3, ncoef(T)), dtype=np.complex128)
    C = a * omega * u0 + 0.5 * u0 * u0
    s[0, packed_index(0, 0, T)] = math.sqrt(2.0) * g * hbar
    if T >= 2:
        s[0, packed_index(0, 2, T)] = -(2.0 * C / 3.0) / math.sqrt(2.5)
    if T >= 1:
        s[1, packed_index(0, 1, T)] = 2.0 * u0 / (a * math.sqrt(1.5))
    return s


def bump_center(seed: int) -> tuple[float, float]:
    """Seeded bump centre: lambda_c ~ U[0, 2pi), phi_c ~ U[-pi/3, pi/3]."""
    rng = np.random.default_rng(seed)
    lam_c = rng.uniform(0.0, 2.0 * math.pi)
    phi_c = rng.uniform(-math.pi / 3.0, math.pi / 3.0)
    return lam_c, phi_c


def gaussian_bump(mu: np.ndarray, lam: np.ndarray, *, amplitude: float,
                  width: float, lam_c: float, phi_c: float) -> np.ndarray:
    """Height bump amplitude*exp(-(d/a)^2 / width^2) on the grid mu x lam.

    d is the chordal distance to the centre (Section 6.1), so (d/a)^2 =
    (x^2 + y^2 + z^2)/a^2 with the paper's x, y, z; ``width`` is in radians
    (the paper's dome factor alpha equals 1/width^2).  Returns [len(mu), len(lam)].
    """
    mu = np.asarray(mu, dtype=np.float64)[:, None]
    lam = np.asarray(lam, dtype=np.float64)[None, :]
    cphi = np.sqrt(np.maximum(0.0, 1.0 - mu * mu))
    x = np.cos(lam) * cphi - math.cos(lam_c) * math.cos(phi_c)
    y = np.sin(lam) * cphi - math.sin(lam_c) * math.cos(phi_c)
    z = mu - math.sin(phi_c)
    d2 = x * x + y * y + z * z
    return amplitude * np.exp(-d2 / (width * width))


def solid_body_axis(seed: int) -> np.ndarray:
    """Seeded unit vector (axis of a tilted solid-body rotation test state)."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(3)
    return v / np.linalg.norm(v)
