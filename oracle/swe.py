"""Spectral shallow-water operators on the rotating sphere (Sections 2, 3, 4, 5.4).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

State: dense ``[..., 3, L, L]`` complex128 holding [Phi, zeta, delta]
(Section 2, prognostic vector U), degree <= T (L = T+1).

* Linear stiff part (Section 2, Eq. "linear_wave_motion_induced_by_
  gravitational_forces"): L(U) = [-Phibar delta + nu lap Phi',
  nu lap zeta, -lap Phi + nu lap delta], with lap Y_n^m = -n(n+1)/a^2 Y_n^m.
* Nonlinear part (Section 2, Eq. "nonlinear_operators"):
  N(U) = [-div(Phi' V), -div((zeta+f) V), curl((zeta+f) V) - lap(V.V/2)],
  f = 2 Omega mu.
* Velocity from the Helmholtz decomposition (Section 2, Eqs.
  "helmholtz_theorem" .. "identity_defining_delta"): V = k x grad psi +
  grad chi with zeta = lap psi, delta = lap chi; the Laplacian is inverted
  spectrally (n = 0 mode of psi, chi set to 0).
* IMEX split (Section 4): F_I = L, F_E = N.
* Implicit system of Section 5.4: x - h F_I(x) = b, solved per (n, m).
* Alternative split with the Coriolis force implicit (the paper keeps it
  explicit, Section 4; ``SWEParams.coriolis_implicit``): the linear Coriolis
  tendency C(U) = [0, -div(f V), curl(f V)] moves from N to the implicit
  part, F_I = L + C and F_E = N evaluated with eta = zeta.  From
  V = k x grad psi + grad chi and grad f = (2 Omega cos(phi)/a) e_north:
      -div(f V) = -f delta - (2 Omega/a) V,   curl(f V) = f zeta - (2 Omega/a) U
  (U = u cos(phi), V = v cos(phi)), where zeta, delta are the Laplacians of
  psi, chi (their n = 0 coefficients do not enter).  Multiplication by
  mu = sin(phi) couples degree n to n +- 1 within an order:
      (mu X)_n = eps_n X_{n-1} + eps_{n+1} X_{n+1},
  so the implicit system of one order m is banded in n; it is solved here by
  dense linear algebra per order.

Spectral-transform evaluation of N (the standard vorticity-divergence
formulation the paper adopts from Bourke 1972 / Hack 1992): with U = u cos(phi),
V = v cos(phi) and d/dphi = cos(phi) d/dmu,
    U = -(1/a)(1-mu^2) d psi/dmu + (1/a) d chi/dlambda,
    V =  (1/a) d psi/dlambda + (1/a)(1-mu^2) d chi/dmu,
and for a flux (A, B) = (a_u cos(phi), a_v cos(phi))
    div  = [dA/dlambda + (1-mu^2) dB/dmu] / (a (1-mu^2)),
    curl = [dB/dlambda - (1-mu^2) dA/dmu] / (a (1-mu^2)).
The mu-derivatives act on the basis through
    (1-mu^2) dP_n^m/dmu = -n eps_{n+1}^m P_{n+1}^m + (n+1) eps_n^m P_{n-1}^m,
and for div/curl they are moved onto the test function by the Gaussian
quadrature of the analysis (A/(1-mu^2), B/(1-mu^2) are analysed).

Pins (tests/test_oracle_swe.py): the balanced zonal jet is a steady state
(F_E + F_I = 0); a tilted solid-body rotation without Coriolis is steady;
mass and circulation are conserved exactly; velocity recovery reproduces
solid-body U, V in closed form; div/curl of recovered (U, V) give back
delta, zeta; brute-force evaluation of N from grid derivatives at tiny T;
the implicit solve against numpy.linalg.solve.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .sht import SHT


@dataclass
class SWEParams:
    a: float           # sphere radius [m]
    omega: float       # rotation rate [1/s]
    g: float           # gravity (only used to define Phibar by callers)
    nu: float          # diffusion coefficient [m^2/s]
    phibar: float      # mean geopotential Phibar = g hbar
    coriolis_implicit: bool = False   # Coriolis tendency in F_I instead of F_E
    implicit_split: bool = False      # SDC node solve in two substeps (see sdc.py)


def kappa(L: int, a: float) -> np.ndarray:
    """-eigenvalue of the Laplacian on degree n: n(n+1)/a^2, n = 0..L-1."""
    n = np.arange(L, dtype=np.float64)
    return n * (n + 1.0) / (a * a)


def _pad(c: np.ndarray, L: int) -> np.ndarray:
    """Zero-pad dense [..., l, l] coefficients to [..., L, L]."""
    out = np.zeros(c.shape[:-2] + (L, L), dtype=np.complex128)
    l = c.shape[-1]
    out[..., :l, :l] = c
    return out


def inverse_laplacian(c: np.ndarray, a: float) -> np.ndarray:
    """psi with lap psi = c; the n = 0 coefficient is set to 0."""
    k = kappa(c.shape[-1], a)
    inv = np.zeros_like(k)
    inv[1:] = -1.0 / k[1:]
    return c * inv


def velocity_coefficients(zeta: np.ndarray, delta: np.ndarray, a: float
                          ) -> tuple[np.ndarray, np.ndarray]:
    """Coefficients of U = u cos(phi), V = v cos(phi) up to degree T+1.

    Input dense [..., T+1, T+1]; output dense [..., T+2, T+2].
    U_n = [(n-1) eps_n psi_{n-1} - (n+2) eps_{n+1} psi_{n+1} + i m chi_n] / a
    V_n = [i m psi_n - (n-1) eps_n chi_{n-1} + (n+2) eps_{n+1} chi_{n+1}] / a
    """
    T = zeta.shape[-1] - 1
    Lo = T + 2
    Lp = T + 4
    psi = _pad(inverse_laplacian(zeta, a), Lp)
    chi = _pad(inverse_laplacian(delta, a), Lp)
    from .sht import epsilon
    eps = epsilon(Lp)
    m = np.arange(Lp, dtype=np.float64)[:, None]
    n = np.arange(Lp, dtype=np.float64)[None, :]

    def shift_down(x):      # x_{n-1}
        y = np.zeros_like(x)
        y[..., 1:] = x[..., :-1]
        return y

    def shift_up(x):        # x_{n+1}
        y = np.zeros_like(x)
        y[..., :-1] = x[..., 1:]
        return y

    eps_n = eps
    eps_n1 = shift_up(eps)
    U = ((n - 1) * eps_n * shift_down(psi) - (n + 2) * eps_n1 * shift_up(psi)
         + 1j * m * chi) / a
    V = (1j * m * psi - (n - 1) * eps_n * shift_down(chi)
         + (n + 2) * eps_n1 * shift_up(chi)) / a
    valid = (n >= m)
    U = np.where(valid, U, 0.0)[..., :Lo, :Lo]
    V = np.where(valid, V, 0.0)[..., :Lo, :Lo]
    return U, V


def div_curl(Ahat: np.ndarray, Bhat: np.ndarray, a: float, T: int
             ) -> tuple[np.ndarray, np.ndarray]:
    """Degree-<=T coefficients of div and curl of the flux whose components
    times cos(phi), divided by (1-mu^2), have analysis coefficients Ahat, Bhat
    (dense, degree <= T+1).

    div_n  = [i m Ahat_n + n eps_{n+1} Bhat_{n+1} - (n+1) eps_n Bhat_{n-1}] / a
    curl_n = [i m Bhat_n - n eps_{n+1} Ahat_{n+1} + (n+1) eps_n Ahat_{n-1}] / a
    """
    from .sht import epsilon
    L = T + 1
    eps = epsilon(T + 2)
    m = np.arange(L, dtype=np.float64)[:, None]
    n = np.arange(L, dtype=np.float64)[None, :]
    A = Ahat[..., :L, :T + 2]
    B = Bhat[..., :L, :T + 2]
    e_n = eps[:L, :L]
    e_n1 = eps[:L, 1:T + 2]
    A_n, B_n = A[..., :, :L], B[..., :, :L]
    A_up, B_up = A[..., :, 1:T + 2], B[..., :, 1:T + 2]
    A_dn = np.zeros_like(A_n)
    B_dn = np.zeros_like(B_n)
    A_dn[..., 1:] = A[..., :L - 1]
    B_dn[..., 1:] = B[..., :L - 1]
    div = (1j * m * A_n + n * e_n1 * B_up - (n + 1) * e_n * B_dn) / a
    curl = (1j * m * B_n - n * e_n1 * A_up + (n + 1) * e_n * A_dn) / a
    valid = n >= m
    return np.where(valid, div, 0.0), np.where(valid, curl, 0.0)


def mu_times(c: np.ndarray) -> np.ndarray:
    """Coefficients (degree < L) of mu times the series c (dense [..., L, L]):
    (mu X)_n = eps_n X_{n-1} + eps_{n+1} X_{n+1} (the degree-L term is cut)."""
    from .sht import epsilon
    L = c.shape[-1]
    eps = epsilon(L + 1)
    out = np.zeros_like(c)
    out[..., :, 1:] += eps[:L, 1:L] * c[..., :, :L - 1]
    out[..., :, :L - 1] += eps[:L, 1:L] * c[..., :, 1:]
    return out


def coriolis_linear(state: np.ndarray, p: SWEParams) -> np.ndarray:
    """C(state) = [0, -div(f V), curl(f V)], degree <= T, dense [..., 3, L, L]:
    -f delta - 2 Omega V / a and f zeta - 2 Omega U / a with f = 2 Omega mu."""
    L = state.shape[-1]
    zeta, delta = state[..., 1, :, :], state[..., 2, :, :]
    U, V = velocity_coefficients(zeta, delta, p.a)
    zeta_l, delta_l = zeta.copy(), delta.copy()     # lap psi, lap chi
    zeta_l[..., 0, 0] = 0.0
    delta_l[..., 0, 0] = 0.0
    out = np.zeros_like(state)
    out[..., 1, :, :] = -2.0 * p.omega * (mu_times(delta_l) + V[..., :L, :L] / p.a)
    out[..., 2, :, :] = 2.0 * p.omega * (mu_times(zeta_l) - U[..., :L, :L] / p.a)
    return out


def linear_part(state: np.ndarray, p: SWEParams) -> np.ndarray:
    """F_I = L(state) (+ C(state) when the Coriolis term is implicit), dense
    [..., 3, L, L]."""
    k = kappa(state.shape[-1], p.a)
    Phi, zeta, delta = state[..., 0, :, :], state[..., 1, :, :], state[..., 2, :, :]
    out = np.empty_like(state)
    out[..., 0, :, :] = -p.phibar * delta - p.nu * k * Phi
    out[..., 1, :, :] = -p.nu * k * zeta
    out[..., 2, :, :] = k * Phi - p.nu * k * delta
    if p.coriolis_implicit:
        out += coriolis_linear(state, p)
    return out


def nonlinear_part(state: np.ndarray, sht: SHT, p: SWEParams) -> np.ndarray:
    """F_E = N(state) by the spectral transform method (grid products); with
    the Coriolis term implicit, eta = zeta (f moves to F_I)."""
    T = state.shape[-1] - 1
    Phi, zeta, delta = state[..., 0, :, :], state[..., 1, :, :], state[..., 2, :, :]
    U, V = velocity_coefficients(zeta, delta, p.a)
    mu = sht.mu[:, None]
    one_m_mu2 = (1.0 - mu) * (1.0 + mu)
    Ug = sht.synthesis(U)
    Vg = sht.synthesis(V)
    f = 0.0 if p.coriolis_implicit else 2.0 * p.omega * mu
    eta = sht.synthesis(zeta) + f                            # zeta + f
    phip = sht.synthesis(Phi) - p.phibar                     # Phi'
    L2 = T + 2
    A1 = sht.analysis(eta * Ug / one_m_mu2, L2)
    B1 = sht.analysis(eta * Vg / one_m_mu2, L2)
    A2 = sht.analysis(phip * Ug / one_m_mu2, L2)
    B2 = sht.analysis(phip * Vg / one_m_mu2, L2)
    E = sht.analysis((Ug * Ug + Vg * Vg) / (2.0 * one_m_mu2), L2)[..., :T + 1, :T + 1]
    div1, curl1 = div_curl(A1, B1, p.a, T)
    div2, _ = div_curl(A2, B2, p.a, T)
    k = kappa(T + 1, p.a)
    out = np.empty_like(state)
    out[..., 0, :, :] = -div2
    out[..., 1, :, :] = -div1
    out[..., 2, :, :] = curl1 + k * E
    return out


def rhs(state: np.ndarray, sht: SHT, p: SWEParams) -> tuple[np.ndarray, np.ndarray]:
    """(F_E, F_I) of a state (Section 4, Eqs. "system_of_odes_*")."""
    return nonlinear_part(state, sht, p), linear_part(state, p)


def diffusion_part(state: np.ndarray, p: SWEParams) -> np.ndarray:
    """The diffusion terms of F_I, nu lap [Phi', zeta, delta] = -nu k state."""
    return -p.nu * kappa(state.shape[-1], p.a) * state


def implicit_solve(b: np.ndarray, h: float, p: SWEParams) -> np.ndarray:
    """x with x - h L(x) = b (Section 5.4, Eq. "implicit_systems").

    Per coefficient with k = n(n+1)/a^2 and s = 1 + h nu k:
      zeta  = b_zeta / s
      [ s        h Phibar ] [Phi  ]   [b_Phi  ]
      [ -h k     s        ] [delta] = [b_delta]
    """
    if p.coriolis_implicit:
        return _implicit_solve_orders(b, h, p)
    k = kappa(b.shape[-1], p.a)
    s = 1.0 + h * p.nu * k
    det = s * s + h * h * p.phibar * k
    bP, bz, bd = b[..., 0, :, :], b[..., 1, :, :], b[..., 2, :, :]
    x = np.empty_like(b)
    x[..., 0, :, :] = (s * bP - h * p.phibar * bd) / det
    x[..., 1, :, :] = bz / s
    x[..., 2, :, :] = (s * bd + h * k * bP) / det
    return x


_order_inverses: dict = {}


def implicit_solve_split(b: np.ndarray, h: float, old: np.ndarray, p: SWEParams) -> np.ndarray:
    """The node solve of an SDC sweep in two substeps, physical linear terms
    first, then diffusion (Section 5.1.1; reading: each substep carries its
    own correction term, as in multi-implicit SDC, so that the fixed point of
    the sweep is unchanged).  With D = the diffusion part of F_I, F_I = L0 + D
    (L0: gravity waves, plus Coriolis when it is implicit) and `old` the
    previous iterate of the node, whose right-hand side b already contains
    -h F_I(old):
        x* - h L0(x*) = b + h D(old),      x - h D(x) = x* - h D(old)."""
    from dataclasses import replace
    xs = implicit_solve(b + h * diffusion_part(old, p), h, replace(p, nu=0.0))
    s = 1.0 + h * p.nu * kappa(b.shape[-1], p.a)
    return (xs - h * diffusion_part(old, p)) / s


def _implicit_solve_orders(b: np.ndarray, h: float, p: SWEParams) -> np.ndarray:
    """x - h (L + C)(x) = b with the Coriolis term implicit: orders m do not
    couple, so each order's 3(T+1-m) unknowns solve a dense system whose
    matrix I - h J_m is read off the operator itself (J_m column (f, n) =
    F_I of the unit coefficient (f, m, n); one application per (f, j = n - m)
    fills that column for every order at once)."""
    L = b.shape[-1]
    key = (L, h, p.a, p.omega, p.nu, p.phibar)
    if key not in _order_inverses:
        cols = np.zeros((3, L, 3, L, L), dtype=np.complex128)   # [f, j][out f, m, n]
        for f in range(3):
            for j in range(L):
                e = np.zeros((3, L, L), dtype=np.complex128)
                for m in range(L - j):
                    e[f, m, m + j] = 1.0
                cols[f, j] = linear_part(e, p)
        inv = []
        for m in range(L):
            K = L - m
            A = np.empty((3 * K, 3 * K), dtype=np.complex128)
            for f in range(3):
                for j in range(K):
                    A[:, f * K + j] = -h * cols[f, j][:, m, m:].reshape(-1)
            A += np.eye(3 * K)
            inv.append(np.linalg.inv(A))
        if len(_order_inverses) > 16:
            _order_inverses.clear()
        _order_inverses[key] = inv
    inv = _order_inverses[key]
    x = np.zeros_like(b)
    for m in range(L):
        K = L - m
        rhs_m = b[..., :, m, m:].reshape(b.shape[:-3] + (3 * K,))
        x[..., :, m, m:] = (rhs_m @ inv[m].T).reshape(b.shape[:-3] + (3, K))
    return x
