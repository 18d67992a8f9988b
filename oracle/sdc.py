"""IMEX spectral deferred corrections on Gauss-Lobatto nodes (Section 5.1.1).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

* Nodes: M+1 Gauss-Lobatto points on [t^n, t^n + dt] (Eq.
  "time_discretization_sdc_nodes"), here as fractions tau_0 = 0 < ... < tau_M = 1.
* Q[i][j] = integral from 0 to tau_i of the Lagrange polynomial l_j on the
  nodes, so that sum_j Q[i][j] F_j approximates the integral of F from t^n to
  t^{n,i} (third line of Eq. "update_equation_sdcq_discrete_form").
* QE: forward Euler, QE[i][j] = tau_{j+1} - tau_j for j < i.
* QI: upper factor of the LU decomposition of Q^T (Weiser 2015).  The first
  row of Q is zero, so Q^T is singular; the reading taken is the pivot-free
  Doolittle LU of Q[1:,1:]^T = L U and QI = [[0, 0], [0, U^T]] (lower
  triangular: node i is implicit in itself and explicit in earlier nodes).
* Sweep (Eq. "update_equation_sdcq_discrete_form", plus the FAS term of
  Eq. "modified_update_equation_sdcq_discrete_form" on the coarse level), for
  node i = 1..M in order:
      b_i = Theta_0 + dt sum_{1<=j<i} QE[i][j] (FE_j^new - FE_j^old)
                    + dt sum_{1<=j<i} QI[i][j] (FI_j^new - FI_j^old)
                    - dt QI[i][i] FI_i^old
                    + dt sum_{0<=j<=M} Q[i][j] (FE_j^old + FI_j^old) + tau_i
      Theta_i solves Theta_i - dt QI[i][i] F_I(Theta_i) = b_i
      (FE_i, FI_i) = F(Theta_i)
  The right-hand side at node 0 must be current (F(Theta_0)) when a sweep
  starts; callers refresh it whenever Theta_0 changes.
* Collocation operator (Eq. "collocation_problem"): A(Theta) = Theta - dt (Q x I) F.

Pins (tests/test_oracle_sdc.py): closed-form nodes and Q rows for 3 and 5
nodes; QI lower-triangular with L U = Q[1:,1:]^T; a converged sweep solves
the collocation problem; accuracy order on dt refinement for scalar IMEX
test equations with known solution and for the SWE.
"""
from __future__ import annotations

import math

import numpy as np
from numpy.polynomial import Polynomial
from numpy.polynomial import legendre as npleg

from .sht import SHT
from .swe import SWEParams, implicit_solve, implicit_solve_split, rhs


def lobatto_nodes(num_nodes: int) -> np.ndarray:
    """Gauss-Lobatto nodes on [0, 1]: 0, 1 and the roots of P'_{num_nodes-1}."""
    M = num_nodes - 1
    if M < 1:
        raise ValueError("need at least 2 nodes")
    inner = np.sort(npleg.legroots(npleg.legder([0] * M + [1]))) if M >= 2 else np.array([])
    x = np.concatenate([[-1.0], inner, [1.0]])
    return 0.5 * (np.real(x) + 1.0)


def lagrange_basis(tau: np.ndarray) -> list[Polynomial]:
    polys = []
    for j in range(tau.size):
        p = Polynomial([1.0])
        for k in range(tau.size):
            if k != j:
                p = p * Polynomial([-tau[k], 1.0]) / (tau[j] - tau[k])
        polys.append(p)
    return polys


def q_matrix(tau: np.ndarray) -> np.ndarray:
    """Q[i][j] = integral_0^{tau_i} l_j(s) ds."""
    n = tau.size
    Q = np.zeros((n, n))
    for j, lj in enumerate(lagrange_basis(tau)):
        Lj = lj.integ()
        for i in range(n):
            Q[i, j] = Lj(tau[i]) - Lj(0.0)
    return Q


def qe_matrix(tau: np.ndarray) -> np.ndarray:
    n = tau.size
    QE = np.zeros((n, n))
    for i in range(n):
        for j in range(i):
            QE[i, j] = tau[j + 1] - tau[j]
    return QE


def doolittle_lu(A: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """A = L U with L unit lower triangular, no pivoting."""
    n = A.shape[0]
    L = np.eye(n)
    U = np.zeros((n, n))
    for i in range(n):
        for k in range(i, n):
            U[i, k] = A[i, k] - sum(L[i, s] * U[s, k] for s in range(i))
        for k in range(i + 1, n):
            L[k, i] = (A[k, i] - sum(L[k, s] * U[s, i] for s in range(i))) / U[i, i]
    return L, U


def qi_matrix(Q: np.ndarray) -> np.ndarray:
    n = Q.shape[0]
    _, U = doolittle_lu(Q[1:, 1:].T)
    QI = np.zeros((n, n))
    QI[1:, 1:] = U.T
    return QI


def lagrange_matrix(src: np.ndarray, dst: np.ndarray) -> np.ndarray:
    """Pi[i][j] = l_j^{src}(dst_i): interpolation from nodes src to nodes dst."""
    basis = lagrange_basis(src)
    return np.array([[b(t) for b in basis] for t in dst])


class SDCLevel:
    """One time level: truncation, grid, nodes and the SWE right-hand side."""

    def __init__(self, T: int, nlat: int, nlon: int, num_nodes: int, dt: float,
                 params: SWEParams):
        self.args = (T, nlat, nlon, num_nodes, dt, params)   # to rebuild it in a worker process
        self.T = T
        self.sht = SHT(T, nlat, nlon)
        self.p = params
        self.dt = dt
        self.tau = lobatto_nodes(num_nodes)
        self.M = num_nodes - 1
        self.Q = q_matrix(self.tau)
        self.QE = qe_matrix(self.tau)
        self.QI = qi_matrix(self.Q)

    def eval_f(self, theta: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
        return rhs(theta, self.sht, self.p)

    def eval_nodes(self, theta: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
        """F_E, F_I at every node of theta [M+1, 3, L, L]."""
        FE = np.empty_like(theta)
        FI = np.empty_like(theta)
        for i in range(theta.shape[0]):
            FE[i], FI[i] = self.eval_f(theta[i])
        return FE, FI

    def sweep(self, theta: np.ndarray, FE: np.ndarray, FI: np.ndarray,
              tau: np.ndarray | None = None):
        """One IMEX-SDC sweep.  theta, FE, FI: [M+1, 3, L, L]; node 0 is the
        initial value with current F.  Returns new (theta, FE, FI)."""
        dt, Q, QE, QI, M = self.dt, self.Q, self.QE, self.QI, self.M
        th_new, FE_new, FI_new = theta.copy(), FE.copy(), FI.copy()
        for i in range(1, M + 1):
            b = theta[0].copy()
            for j in range(1, i):
                b += dt * QE[i, j] * (FE_new[j] - FE[j])
                b += dt * QI[i, j] * (FI_new[j] - FI[j])
            b -= dt * QI[i, i] * FI[i]
            for j in range(M + 1):
                b += dt * Q[i, j] * (FE[j] + FI[j])
            if tau is not None:
                b += tau[i]
            if self.p.implicit_split:
                th_new[i] = implicit_solve_split(b, dt * QI[i, i], theta[i], self.p)
            else:
                th_new[i] = implicit_solve(b, dt * QI[i, i], self.p)
            FE_new[i], FI_new[i] = self.eval_f(th_new[i])
        return th_new, FE_new, FI_new

    def spread(self, theta0: np.ndarray):
        """Initial iterate: theta0 copied to every node with F(theta0)."""
        fe, fi = self.eval_f(theta0)
        theta = np.repeat(theta0[None], self.M + 1, axis=0)
        return theta, np.repeat(fe[None], self.M + 1, axis=0), np.repeat(fi[None], self.M + 1, axis=0)

    def collocation_residual(self, theta: np.ndarray, FE: np.ndarray,
                             FI: np.ndarray) -> np.ndarray:
        """A(Theta) - 1 x Theta_0 (zero at the collocation solution)."""
        F = FE + FI
        QF = np.einsum("ij,j...->i...", self.Q, F)
        return theta - self.dt * QF - theta[0][None]


def sdc_step(level: SDCLevel, theta0: np.ndarray, n_sweeps: int) -> np.ndarray:
    """SDC(M+1, n_sweeps) over one step: spread, sweep, return the last node."""
    theta, FE, FI = level.spread(theta0)
    for _ in range(n_sweeps):
        theta, FE, FI = level.sweep(theta, FE, FI)
    return theta[-1]


def sdc_run(level: SDCLevel, theta0: np.ndarray, n_steps: int, n_sweeps: int) -> np.ndarray:
    th = theta0
    for _ in range(n_steps):
        th = sdc_step(level, th, n_sweeps)
    return th
