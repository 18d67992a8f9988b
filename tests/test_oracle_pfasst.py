"""Pins of the oracle's FAS/PFASST (Sections 5.1.2, 5.2, 5.3, Algorithm 1)."""
import numpy as np
import pytest

from oracle.pfasst import PFASST, restrict_space, interpolate_space
from oracle.sdc import SDCLevel, lagrange_matrix, lobatto_nodes
from oracle.sht import unpack
from oracle.swe import SWEParams
import synthetic as syn


def _params():
    return SWEParams(a=syn.EARTH_RADIUS, omega=syn.OMEGA, g=syn.GRAVITY, nu=1e5,
                     phibar=syn.GRAVITY * syn.MEAN_DEPTH)


def _state(T, seed=1):
    return unpack(syn.zonal_jet(T), T) + unpack(
        syn.random_spectrum(T, (3,), seed=seed, rms=1e-5), T) * np.array([1e3, 1, 1])[:, None, None]


def _levels(Tf, Tc, dt):
    f = SDCLevel(Tf, *syn.gaussian_grid_size(Tf), 5, dt, _params())
    c = SDCLevel(Tc, *syn.gaussian_grid_size(Tc), 3, dt, _params())
    return f, c


def test_space_restriction_of_interpolation_is_identity():
    x = unpack(syn.random_spectrum(7, (3,), seed=2, nmin=0), 7)
    y = interpolate_space(x, 16)
    assert np.array_equal(restrict_space(y, 8), x)
    assert np.all(y[..., 8:, :] == 0) and np.all(y[..., :, 8:] == 0)


@pytest.mark.parametrize("fine,coarse,inj", [(5, 3, [0, 2, 4]), (3, 2, [0, 2]), (5, 2, [0, 4])])
def test_nested_lobatto_time_restriction_is_injection(fine, coarse, inj):
    R = lagrange_matrix(lobatto_nodes(fine), lobatto_nodes(coarse))
    E = np.zeros_like(R)
    for i, j in enumerate(inj):
        E[i, j] = 1.0
    assert np.max(np.abs(R - E)) < 1e-14
    # interpolation reproduces the coarse values at the shared nodes
    P = lagrange_matrix(lobatto_nodes(coarse), lobatto_nodes(fine))
    assert np.max(np.abs(R @ P - np.eye(coarse))) < 1e-14


def test_fas_invariant_restricted_fine_solution_solves_coarse_problem():
    """Section 5.1.2: with tau_c, R Theta_f is a solution of the coarse problem."""
    f, c = _levels(15, 7, 600.0)
    th, FE, FI = f.spread(_state(15))
    for _ in range(30):
        th, FE, FI = f.sweep(th, FE, FI)
    pf = PFASST(f, c, 1)
    thc = pf.restrict(th)
    FEc = np.empty_like(thc)
    FIc = np.empty_like(thc)
    for i in range(3):
        FEc[i], FIc[i] = c.eval_f(thc[i])
    tau = pf.fas(FE, FI, FEc, FIc)
    thc2, _, _ = c.sweep(thc, FEc, FIc, tau)
    assert np.max(np.abs(thc2 - thc)) < 1e-14 * np.max(np.abs(thc))


def _serial(f, th0, n_ts):
    out, x = [], th0
    for _ in range(n_ts):
        th, FE, FI = f.spread(x)
        for _ in range(40):
            th, FE, FI = f.sweep(th, FE, FI)
        x = th[-1]
        out.append(x)
    return np.array(out)


@pytest.mark.parametrize("Tc", [15, 7])
def test_pfasst_converges_to_serial_collocation(Tc):
    Tf, n_ts = 15, 4
    f, c = _levels(Tf, Tc, 600.0)
    th0 = _state(Tf)
    ref = _serial(f, th0, n_ts)
    pf = PFASST(f, c, n_ts)
    errs = [np.max(np.abs(pf.run(th0, k) - ref)) for k in (2, 12)]
    scale = np.max(np.abs(ref[:, 1]))
    assert errs[1] < 1e-12 * np.max(np.abs(ref))
    assert errs[1] < errs[0]
    assert scale > 0


def test_pfasst_single_slice_is_two_level_sdc():
    f, c = _levels(15, 7, 600.0)
    th0 = _state(15)
    ref = _serial(f, th0, 1)
    out = PFASST(f, c, 1).run(th0, 8)
    assert np.max(np.abs(out - ref)) < 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("coriolis,split", [(True, False), (False, True), (True, True)])
def test_pfasst_with_other_splits_converges_to_the_same_collocation_solution(coriolis, split):
    """The Coriolis term in F_I (which couples degrees n +- 1, so that
    restriction and F_I no longer commute at the top coarse degree: the FAS
    term absorbs it) and the two-substep node solve leave the fixed point of
    Algorithm 1 unchanged: PFASST converges to the serial fine collocation
    solution of the paper's split, for alpha < 1."""
    Tf, Tc, n_ts, dt = 15, 7, 4, 600.0
    f, _ = _levels(Tf, Tc, dt)
    th0 = _state(Tf)
    ref = _serial(f, th0, n_ts)
    p = SWEParams(a=syn.EARTH_RADIUS, omega=syn.OMEGA, g=syn.GRAVITY, nu=1e5, phibar=syn.GRAVITY * syn.MEAN_DEPTH,
                  coriolis_implicit=coriolis, implicit_split=split)
    fo = SDCLevel(Tf, *syn.gaussian_grid_size(Tf), 5, dt, p)
    co = SDCLevel(Tc, *syn.gaussian_grid_size(Tc), 3, dt, p)
    errs = [np.max(np.abs(PFASST(fo, co, n_ts).run(th0, k) - ref)) for k in (2, 14)]
    assert errs[1] < 1e-12 * np.max(np.abs(ref))
    assert errs[1] < errs[0]


@pytest.mark.parametrize("npf,order", [(1, 1), (2, 2), (3, 3)])
def test_pfasst_iterations_add_one_order_each(npf, order):
    """alpha = 1: a fixed number N_PF of PFASST iterations per block converges
    with order N_PF in dt (each iteration adds one order below the collocation
    order, as for SDC sweeps; the paper prints no rates, so this pins the
    iteration structure).  T10, 4 slices, 5/3 nodes, window 19200 s in 1, 2
    and 4 blocks, against SDC(5) run to convergence with 1/8 of the step."""
    import math
    from oracle.sdc import sdc_run
    T, n_ts, t_end = 10, 4, 19200.0
    th0 = _state(T)
    gf = syn.gaussian_grid_size(T)
    ref = sdc_run(SDCLevel(T, *gf, 5, t_end / 32, _params()), th0, 32, 10)
    errs = []
    for blocks in (1, 2, 4):
        dt = t_end / (n_ts * blocks)
        f, c = _levels(T, T, dt)
        x = th0
        for _ in range(blocks):
            x = PFASST(f, c, n_ts).run(x, npf)[-1]
        errs.append(np.max(np.abs(x - ref)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert abs(rates[-1] - order) < 0.3, rates


def _spread_coarse(c, th0_c):
    fe, fi = c.eval_f(th0_c)
    M = c.M
    return (np.repeat(th0_c[None], M + 1, 0), np.repeat(fe[None], M + 1, 0), np.repeat(fi[None], M + 1, 0))


@pytest.mark.parametrize("Tf,Tc,n_ts", [(9, 9, 1), (9, 6, 1), (9, 6, 4)])
def test_predictor_round_structure(Tf, Tc, n_ts):
    """Section 5.2.1 written out slice by slice instead of round by round:
    slice n sweeps n + 1 times on the coarse level; before its r-th sweep
    (r >= 1) it takes as node-0 value the end value slice n-1 had after its
    own r-th sweep (round r-1) and refreshes F there; every slice starts from
    the spread restricted initial value.  The fine iterate is the initial
    value plus the coarse increment interpolated in space (zero-padding) and
    time (Lagrange), with F evaluated at every fine node.  With n_ts = 1 this
    is one coarse sweep from the spread state.  A schedule with n sweeps for
    slice n, or a receive from the wrong round, fails the equality."""
    f, c = _levels(Tf, Tc, 600.0)
    th0 = _state(Tf, seed=3)
    pf = PFASST(f, c, n_ts)
    pf.predict(th0)
    base = _spread_coarse(c, restrict_space(th0, Tc + 1))
    E = {}
    finals = []
    for n in range(n_ts):
        th, FE, FI = (a.copy() for a in base)
        for r in range(n + 1):
            if r > 0:
                th[0] = E[n - 1, r - 1]
                FE[0], FI[0] = c.eval_f(th[0])
            th, FE, FI = c.sweep(th, FE, FI)
            E[n, r] = th[-1].copy()
        finals.append(th)
        assert np.array_equal(pf.th_c[n], th), n
    P = lagrange_matrix(c.tau, f.tau)
    for n in range(n_ts):
        inc = interpolate_space(finals[n] - base[0], Tf + 1)
        exp = th0[None] + np.einsum("ij,j...->i...", P, inc)
        assert np.max(np.abs(pf.th_f[n] - exp)) <= 1e-15 * np.max(np.abs(exp))
        for i in range(f.M + 1):
            fe, fi = f.eval_f(pf.th_f[n, i])
            assert np.array_equal(pf.FE_f[n, i], fe) and np.array_equal(pf.FI_f[n, i], fi)
    if n_ts > 1:   # the later slices saw their predecessors' values: they differ from slice 0
        assert np.max(np.abs(pf.th_c[n_ts - 1] - pf.th_c[0])) > 0


def test_slice_pool_changes_no_arithmetic():
    """The worker-process pool runs the same level methods: predictor + one
    iteration give bitwise the same space-time arrays with and without it."""
    from oracle.pool import SlicePool
    f, c = _levels(9, 6, 600.0)
    th0 = _state(9, seed=4)
    a = PFASST(f, c, 3)
    a.run(th0, 2)
    with SlicePool({"f": f.args, "c": c.args}, workers=2) as pool:
        b = PFASST(f, c, 3, pool=pool)
        b.run(th0, 2)
    for name in ("th_f", "FE_f", "FI_f", "th_c", "FE_c", "FI_c"):
        assert np.array_equal(getattr(a, name), getattr(b, name)), name
