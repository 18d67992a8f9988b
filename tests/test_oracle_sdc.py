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


# ---------------------------------------------------------------------------
# Node solve in two substeps (physical linear terms, then diffusion), each
# with its own correction term
# ---------------------------------------------------------------------------
def _split(nu=syn.NU, coriolis=False):
    p = _params()
    return SWEParams(a=p.a, omega=p.omega, g=p.g, nu=nu, phibar=p.phibar, coriolis_implicit=coriolis,
                     implicit_split=True)


@pytest.mark.parametrize("coriolis", [False, True])
def test_split_sweeps_converge_to_the_collocation_solution(coriolis):
    """The substeps change every sweep but not its fixed point: iterated,
    the split sweep solves the same collocation problem as the one-solve
    sweep (and leaves a zero collocation residual)."""
    T = 15
    nlat, nlon = syn.gaussian_grid_size(T)
    nu = 5e5     # strong diffusion: the splitting error of one sweep is large
    comb = SDCLevel(T, nlat, nlon, 5, 600.0, SWEParams(a=syn.EARTH_RADIUS, omega=syn.OMEGA, g=syn.GRAVITY, nu=nu,
                                                        phibar=syn.GRAVITY * syn.MEAN_DEPTH,
                                                        coriolis_implicit=coriolis))
    split = SDCLevel(T, nlat, nlon, 5, 600.0, _split(nu, coriolis))
    x0 = _state(T)
    a = comb.spread(x0)
    b = split.spread(x0)
    a1 = comb.sweep(*a)
    b1 = split.sweep(*b)
    assert np.max(np.abs(a1[0] - b1[0])) > 1e-9 * np.max(np.abs(a1[0] - x0))    # one sweep differs
    for _ in range(40):
        a = comb.sweep(*a)
        b = split.sweep(*b)
    change = np.max(np.abs(a[0][-1] - x0))
    assert np.max(np.abs(a[0] - b[0])) < 1e-12 * change
    res = split.collocation_residual(*b)
    assert np.max(np.abs(res)) < 1e-14 * np.max(np.abs(b[0]))


def test_split_sweep_without_diffusion_is_the_one_solve_sweep():
    T = 12
    nlat, nlon = syn.gaussian_grid_size(T)
    p0 = _params()
    comb = SDCLevel(T, nlat, nlon, 3, 600.0, SWEParams(a=p0.a, omega=p0.omega, g=p0.g, nu=0.0, phibar=p0.phibar))
    split = SDCLevel(T, nlat, nlon, 3, 600.0, _split(nu=0.0))
    x0 = _state(T, 4)
    a = comb.sweep(*comb.spread(x0))
    b = split.sweep(*split.spread(x0))
    assert np.max(np.abs(a[0] - b[0])) <= 1e-15 * np.max(np.abs(a[0]))


def test_split_sweeps_keep_the_accuracy_order():
    """Two sweeps on 3 nodes stay second order in dt with the split solve."""
    T = 15
    nlat, nlon = syn.gaussian_grid_size(T)
    th0 = _state(T)
    t_end = 3600.0
    ref = sdc_run(SDCLevel(T, nlat, nlon, 5, t_end / 32, _params()), th0, 32, 8)
    errs = []
    for n in (4, 8, 16):
        out = sdc_run(SDCLevel(T, nlat, nlon, 3, t_end / n, _split()), th0, n, 2)
        errs.append(np.max(np.abs(out - ref)[1]))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(r - 2) < 0.25 for r in rates), rates
