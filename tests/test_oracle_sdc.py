"""Pins of the oracle's IMEX-SDC (Section 5.1.1) against closed forms and invariants."""
import math

import numpy as np
import pytest

from oracle.sdc import (lobatto_nodes, q_matrix, qe_matrix, qi_matrix, doolittle_lu,
                        SDCLevel, sdc_run)
from oracle.sht import unpack
from oracle.swe import SWEParams
import synthetic as syn


def test_lobatto_nodes_closed_forms():
    assert np.allclose(lobatto_nodes(2), [0.0, 1.0], atol=0, rtol=0)
    assert np.max(np.abs(lobatto_nodes(3) - [0.0, 0.5, 1.0])) < 1e-16
    r = math.sqrt(3.0 / 7.0)
    ref = [0.0, (1 - r) / 2, 0.5, (1 + r) / 2, 1.0]
    assert np.max(np.abs(lobatto_nodes(5) - ref)) < 1e-15


def test_q_matrix_closed_form_rows():
    Q3 = q_matrix(lobatto_nodes(3))
    assert np.max(np.abs(Q3[0])) == 0.0
    assert np.max(np.abs(Q3[1] - [5 / 24, 1 / 3, -1 / 24])) < 1e-14
    assert np.max(np.abs(Q3[2] - [1 / 6, 2 / 3, 1 / 6])) < 1e-14          # Simpson
    Q5 = q_matrix(lobatto_nodes(5))
    assert np.max(np.abs(Q5[4] - [1 / 20, 49 / 180, 16 / 45, 49 / 180, 1 / 20])) < 1e-14


@pytest.mark.parametrize("nodes", [2, 3, 5])
def test_q_matrix_integrates_polynomials_exactly(nodes):
    tau = lobatto_nodes(nodes)
    Q = q_matrix(tau)
    for k in range(nodes):
        assert np.max(np.abs(Q @ tau ** k - tau ** (k + 1) / (k + 1))) < 1e-14


@pytest.mark.parametrize("nodes", [2, 3, 5])
def test_qe_qi_structure(nodes):
    tau = lobatto_nodes(nodes)
    Q = q_matrix(tau)
    QE = qe_matrix(tau)
    QI = qi_matrix(Q)
    # forward Euler rows integrate constants exactly
    assert np.max(np.abs(QE.sum(axis=1) - tau)) < 1e-15
    assert np.allclose(np.triu(QE), 0.0)
    assert np.allclose(np.triu(QI, 1), 0.0)
    assert np.all(QI[0] == 0.0) and np.all(QI[:, 0] == 0.0)
    Lf, U = doolittle_lu(Q[1:, 1:].T)
    assert np.max(np.abs(Lf @ U - Q[1:, 1:].T)) < 1e-15
    assert np.allclose(np.diag(Lf), 1.0) and np.allclose(np.triu(Lf, 1), 0.0)
    assert np.max(np.abs(QI[1:, 1:] - U.T)) == 0.0


def _params(nu=1e5):
    return SWEParams(a=syn.EARTH_RADIUS, omega=syn.OMEGA, g=syn.GRAVITY, nu=nu,
                     phibar=syn.GRAVITY * syn.MEAN_DEPTH)


def _state(T, seed=1):
    return unpack(syn.zonal_jet(T), T) + unpack(
        syn.random_spectrum(T, (3,), seed=seed, rms=1e-5), T) * np.array([1e3, 1, 1])[:, None, None]


def test_converged_sweeps_solve_the_collocation_problem():
    T = 15
    lvl = SDCLevel(T, *syn.gaussian_grid_size(T), 5, 600.0, _params())
    th, FE, FI = lvl.spread(_state(T))
    for _ in range(30):
        th, FE, FI = lvl.sweep(th, FE, FI)
    res = lvl.collocation_residual(th, FE, FI)
    assert np.max(np.abs(res)) < 1e-14 * np.max(np.abs(th))


@pytest.mark.parametrize("nodes,sweeps,order", [(3, 1, 1), (3, 2, 2)])
def test_accuracy_order_on_dt_refinement(nodes, sweeps, order):
    """Each sweep raises the order by one up to the quadrature order."""
    T = 15
    nlat, nlon = syn.gaussian_grid_size(T)
    th0 = _state(T)
    t_end = 3600.0
    ref = sdc_run(SDCLevel(T, nlat, nlon, 5, t_end / 32, _params()), th0, 32, 8)
    errs = []
    for n in (4, 8, 16):
        out = sdc_run(SDCLevel(T, nlat, nlon, nodes, t_end / n, _params()), th0, n, sweeps)
        errs.append(np.max(np.abs(out - ref)[1]))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(r - order) < 0.25 for r in rates), rates
