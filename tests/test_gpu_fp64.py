"""Parity of the FP64 CUDA path with the oracle, element by element, through
the C ABI (Python binding = argument marshalling only).

Tolerances (FP64): rel-L2 <= 1e-12 for a transform; <= 5e-11 for one RHS
evaluation (RHS_TOL); <= 1e-10 for 20 SDC steps; <= 1e-11 for PFASST.

Why the RHS bound is looser than the transform bound: the flux products are
divided by 1 - mu^2, which near the poles turns a one-ulp difference in the
Gaussian latitudes (the two sides compute them independently) into a relative
change of up to ~1e-11 in the tendencies.  Measured on the oracle alone:
moving mu by one ulp changes its delta tendency by 3.3e-12 (T85) and 2.9e-11
(T170) in rel-L2; RHS_TOL sits just above that.
"""
import numpy as np
import pytest

import synthetic as syn
from oracle.sht import SHT, pack, unpack
from oracle.swe import SWEParams, rhs, implicit_solve
from oracle.sdc import SDCLevel
from oracle.pfasst import PFASST
from _lib import ensure_built

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
ensure_built()
import paper_1904_05988_gb300 as ps  # noqa: E402

DEV = torch.device("cuda:0")
A, OM, G = syn.EARTH_RADIUS, syn.OMEGA, syn.GRAVITY
PHIBAR = G * syn.MEAN_DEPTH
RHS_TOL = 5e-11


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


def cuda(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.complex128, device=DEV)


def state_of(T, seed, batch=1):
    s = syn.random_spectrum(T, (batch, 3), seed=seed, rms=1e-5)
    s[:, 0] *= 1e3
    return s + syn.zonal_jet(T)[None]


# ---------------------------------------------------------------------------
# transforms
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("T", [31, 63, 85, 170])
def test_sht_inverse_and_forward_match_oracle(T):
    nlat, nlon = syn.gaussian_grid_size(T)
    plan = ps.sht_plan_create(T, nlat, nlon, 12, "fp64")
    assert np.max(np.abs(np.array(plan.mu) - SHT(T, nlat, nlon, L=T + 1).mu)) < 1e-15
    nf = 20   # passes of 12 (tiled kernels) and 8 (small-batch kernels)
    spec = syn.random_spectrum(T, (nf,), seed=T, nmin=0)
    grid = torch.empty((nf, nlat, nlon), dtype=torch.float64, device=DEV)
    ps.sht_inverse(plan, cuda(spec), grid)
    ps.pfsh_sync_status()
    o = SHT(T, nlat, nlon, L=T + 1)
    ref = o.synthesis(unpack(spec, T))
    assert rel(grid.cpu().numpy(), ref) < 1e-12
    back = torch.empty((nf, syn.ncoef(T)), dtype=torch.complex128, device=DEV)
    ps.sht_forward(plan, torch.tensor(ref, device=DEV), back)
    ps.pfsh_sync_status()
    ref_spec = pack(o.analysis(ref, T + 1), T)
    assert rel(back.cpu().numpy(), ref_spec) < 1e-12
    assert rel(back.cpu().numpy(), spec) < 1e-12


def test_sht_empty_batch_is_a_no_op():
    plan = ps.sht_plan_create(15, 24, 48, 2, "fp64")
    g = torch.zeros((0, 24, 48), dtype=torch.float64, device=DEV)
    s = torch.zeros((0, syn.ncoef(15)), dtype=torch.complex128, device=DEV)
    ps.sht_inverse(plan, s, g)
    ps.sht_forward(plan, g, s)
    ps.pfsh_sync_status()


# ---------------------------------------------------------------------------
# RHS and implicit solve
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("T,B", [(21, 1), (63, 3), (85, 2), (170, 1)])
def test_swe_rhs_matches_oracle(T, B):
    nlat, nlon = syn.gaussian_grid_size(T)
    plan = ps.sht_plan_create(T, nlat, nlon, 10, "fp64")   # 2 states per pass -> ragged chunks
    ctx = ps.swe_ctx_create(plan, A, OM, syn.NU, PHIBAR)
    st = state_of(T, 100 + T, B)
    fE = torch.empty((B, 3, syn.ncoef(T)), dtype=torch.complex128, device=DEV)
    fI = torch.empty_like(fE)
    ps.swe_rhs(ctx, cuda(st), fE, fI)
    ps.pfsh_sync_status()
    p = SWEParams(a=A, omega=OM, g=G, nu=syn.NU, phibar=PHIBAR)
    FE, FI = rhs(unpack(st, T), SHT(T, nlat, nlon), p)
    for b in range(B):
        for f in range(3):
            assert rel(fE.cpu().numpy()[b, f], pack(FE[b, f], T)) < RHS_TOL, (b, f)
            assert rel(fI.cpu().numpy()[b, f], pack(FI[b, f], T)) < 1e-13, (b, f)


def test_swe_rhs_t255_full_grid():
    T = 255
    nlat, nlon = syn.gaussian_grid_size(T)
    plan = ps.sht_plan_create(T, nlat, nlon, 10, "fp64")
    ctx = ps.swe_ctx_create(plan, A, OM, syn.NU, PHIBAR)
    st = state_of(T, 7, 2)
    fE = torch.empty((2, 3, syn.ncoef(T)), dtype=torch.complex128, device=DEV)
    ps.swe_rhs(ctx, cuda(st), fE, None)
    ps.pfsh_sync_status()
    p = SWEParams(a=A, omega=OM, g=G, nu=syn.NU, phibar=PHIBAR)
    FE, _ = rhs(unpack(st[1], T), SHT(T, nlat, nlon), p)
    assert rel(fE.cpu().numpy()[1], pack(FE, T)) < RHS_TOL


def test_swe_rhs_t511_long_rows():
    """T511 on 768 x 1536 in FP64: ten padded transforms of 1536 points exceed
    the shared memory of a block, so the grid stage takes the long-row kernel
    (products transformed one after the other).  Batched path (3 states) and
    batch-1 path (1 state) against the oracle on the same state."""
    T = 511
    nlat, nlon = syn.gaussian_grid_size(T)
    plan = ps.sht_plan_create(T, nlat, nlon, 15, "fp64")
    ctx = ps.swe_ctx_create(plan, A, OM, syn.NU, PHIBAR)
    st = state_of(T, 511, 3)
    fE3 = torch.empty((3, 3, syn.ncoef(T)), dtype=torch.complex128, device=DEV)
    fE1 = torch.empty((1, 3, syn.ncoef(T)), dtype=torch.complex128, device=DEV)
    ps.swe_rhs(ctx, cuda(st), fE3, None)
    ps.swe_rhs(ctx, cuda(st[:1]), fE1, None)
    ps.pfsh_sync_status()
    p = SWEParams(a=A, omega=OM, g=G, nu=syn.NU, phibar=PHIBAR)
    FE, _ = rhs(unpack(st[0], T), SHT(T, nlat, nlon), p)
    assert rel(fE3.cpu().numpy()[0], pack(FE, T)) < RHS_TOL
    assert rel(fE1.cpu().numpy()[0], pack(FE, T)) < RHS_TOL


def test_balanced_jet_is_steady_on_gpu():
    T = 63
    nlat, nlon = syn.gaussian_grid_size(T)
    plan = ps.sht_plan_create(T, nlat, nlon, 5, "fp64")
    ctx = ps.swe_ctx_create(plan, A, OM, 0.0, PHIBAR)
    st = cuda(syn.zonal_jet(T)[None])
    fE = torch.empty_like(st)
    fI = torch.empty_like(st)
    ps.swe_rhs(ctx, st, fE, fI)
    ps.pfsh_sync_status()
    tot = (fE + fI).abs().max().item()
    assert tot < 1e-11 * fI.abs().max().item()


def test_implicit_solve_matches_oracle_and_aliases():
    T = 63
    nlat, nlon = syn.gaussian_grid_size(T)
    plan = ps.sht_plan_create(T, nlat, nlon, 5, "fp64")
    ctx = ps.swe_ctx_create(plan, A, OM, syn.NU, PHIBAR)
    b = state_of(T, 3, 4)
    x = torch.empty((4, 3, syn.ncoef(T)), dtype=torch.complex128, device=DEV)
    ps.swe_implicit_solve(ctx, cuda(b), x, 45.0)
    bb = cuda(b)
    ps.swe_implicit_solve(ctx, bb, bb, 45.0)      # in place
    ps.pfsh_sync_status()
    p = SWEParams(a=A, omega=OM, g=G, nu=syn.NU, phibar=PHIBAR)
    ref = pack(implicit_solve(unpack(b, T), 45.0, p), T)
    assert rel(x.cpu().numpy(), ref) < 1e-14
    assert torch.equal(x, bb)


# ---------------------------------------------------------------------------
# SDC
# ---------------------------------------------------------------------------
def test_sdc_twenty_steps_t63_matches_oracle():
    """Plain method, FP64, single slice: T63 on 96x192, 3 Lobatto nodes, 2 sweeps,
    dt = 180 s, 20 steps, balanced jet plus n^-3 vorticity perturbation."""
    T, nodes, sweeps, dt, steps = 63, 3, 2, 180.0, 20
    nlat, nlon = syn.gaussian_grid_size(T)
    st0 = syn.zonal_jet(T)
    st0[1] += syn.random_spectrum(T, (1,), seed=1, rms=1e-6)[0]
    plan = ps.sht_plan_create(T, nlat, nlon, 5, "fp64")
    ctx = ps.swe_ctx_create(plan, A, OM, syn.NU, PHIBAR)
    lvl = ps.sdc_level_create(ctx, nodes, dt, 1)
    th = torch.empty((nodes, 1, 3, syn.ncoef(T)), dtype=torch.complex128, device=DEV)
    fE, fI = torch.empty_like(th), torch.empty_like(th)
    x = cuda(st0[None])
    for _ in range(steps):
        ps.sdc_spread(lvl, x, th, fE, fI)
        for _ in range(sweeps):
            ps.sdc_sweep(lvl, th, fE, fI)
        x = th[-1].clone()
    ps.pfsh_sync_status()
    p = SWEParams(a=A, omega=OM, g=G, nu=syn.NU, phibar=PHIBAR)
    lv = SDCLevel(T, nlat, nlon, nodes, dt, p)
    y = unpack(st0, T)
    for _ in range(steps):
        y = sdc_step_ref(lv, y, sweeps)
    ref = pack(y, T)
    got = x.cpu().numpy()[0]
    assert rel(got, ref) < 1e-10
    # the perturbation itself (not just the jet) is matched
    assert rel(got[1] - syn.zonal_jet(T)[1], ref[1] - syn.zonal_jet(T)[1]) < 1e-9


def sdc_step_ref(lv, y, sweeps):
    th, FE, FI = lv.spread(y)
    for _ in range(sweeps):
        th, FE, FI = lv.sweep(th, FE, FI)
    return th[-1]


def test_sdc_sweep_with_tau_and_batch_matches_oracle():
    T, nodes, dt, B = 31, 5, 300.0, 3
    nlat, nlon = syn.gaussian_grid_size(T)
    plan = ps.sht_plan_create(T, nlat, nlon, 10, "fp64")
    ctx = ps.swe_ctx_create(plan, A, OM, syn.NU, PHIBAR)
    lvl = ps.sdc_level_create(ctx, nodes, dt, B)
    st = state_of(T, 11, B)
    tau = syn.random_spectrum(T, (nodes, B, 3), seed=12, rms=1e-9)
    tau[0] = 0
    th = torch.empty((nodes, B, 3, syn.ncoef(T)), dtype=torch.complex128, device=DEV)
    fE, fI = torch.empty_like(th), torch.empty_like(th)
    ps.sdc_spread(lvl, cuda(st), th, fE, fI)
    ps.sdc_sweep(lvl, th, fE, fI, cuda(tau))
    ps.sdc_sweep(lvl, th, fE, fI, cuda(tau))
    ps.pfsh_sync_status()
    p = SWEParams(a=A, omega=OM, g=G, nu=syn.NU, phibar=PHIBAR)
    lv = SDCLevel(T, nlat, nlon, nodes, dt, p)
    for b in range(B):
        t_, e_, i_ = lv.spread(unpack(st[b], T))
        for _ in range(2):
            t_, e_, i_ = lv.sweep(t_, e_, i_, unpack(tau[:, b], T))
        assert rel(th.cpu().numpy()[:, b], pack(t_, T)) < 1e-12
        assert rel(fE.cpu().numpy()[:, b], pack(e_, T)) < 1e-11


# ---------------------------------------------------------------------------
# PFASST
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("Tf,Tc,nts,groups", [(21, 10, 4, 0), (31, 31, 3, 0), (21, 10, 9, 2)])
def test_pfasst_predict_and_iterations_match_oracle(Tf, Tc, nts, groups):
    """groups = 2 with 9 slices: the coarse chain of slices 0-3 overlaps the
    fine sweep of slices 4-8 (uneven groups of 4 and 5)."""
    dt, nf, nc, iters = 600.0, 5, 3, 3
    gf, gc = syn.gaussian_grid_size(Tf), syn.gaussian_grid_size(Tc)
    st0 = state_of(Tf, 21)[0]
    pf = ps.pfasst_create(nts, nf, nc, Tf, *gf, Tc, *gc, dt, A, OM, syn.NU, PHIBAR, "fp64", slice_groups=groups)
    ps.pfasst_set_initial(pf, cuda(st0))
    ps.pfasst_predict(pf)
    p = SWEParams(a=A, omega=OM, g=G, nu=syn.NU, phibar=PHIBAR)
    o = PFASST(SDCLevel(Tf, *gf, nf, dt, p), SDCLevel(Tc, *gc, nc, dt, p), nts)
    o.predict(unpack(st0, Tf))
    out = torch.empty((3, syn.ncoef(Tf)), dtype=torch.complex128, device=DEV)
    outc = torch.empty((3, syn.ncoef(Tc)), dtype=torch.complex128, device=DEV)

    def compare(tol):
        for n in range(nts):
            for k in range(nf):
                ps.pfasst_get(pf, 0, n, k, out)
                assert rel(out.cpu().numpy(), pack(o.th_f[n, k], Tf)) < tol, (n, k)
            ps.pfasst_get(pf, 1, n, nc - 1, outc)
            assert rel(outc.cpu().numpy(), pack(o.th_c[n, nc - 1], Tc)) < tol, n

    compare(1e-12)
    for it in range(iters):
        last = it == iters - 1
        ps.pfasst_iteration(pf, last)
        o.iteration(last)
        ps.pfsh_sync_status()
        compare(1e-11)


@pytest.mark.parametrize("form", ["fp64", "bf16x3"])
def test_pfasst_slice_groups_leave_results_unchanged(form):
    """The pipelined iteration (coarse chain of a slice group overlapping the
    fine sweeps of the next groups) and the wavefront block of iterations
    (groups of iteration k+1 starting beside the chain of iteration k)
    compute exactly what one-group single iterations compute: same kernels,
    same batch paths, same order of arithmetic per slice.  The block is
    checked eagerly, when captured into a graph and when replayed."""
    if form not in ps.available_precisions():
        pytest.skip(f"{form} not built")
    Tf, Tc, nts, dt = 63, 31, 12, 600.0
    gf, gc = syn.gaussian_grid_size(Tf), syn.gaussian_grid_size(Tc)
    st0 = cuda(state_of(Tf, 23)[0])

    def run(groups, mode):
        pf = ps.pfasst_create(nts, 5, 3, Tf, *gf, Tc, *gc, dt, A, OM, syn.NU, PHIBAR, form, slice_groups=groups)
        rounds = 3 if mode == "block" else 1       # block: eager, capture, replay
        for _ in range(rounds):
            ps.pfasst_set_initial(pf, st0)
            ps.pfasst_predict(pf)
            if mode == "single":
                for it in range(3):   # eager, graph capture, graph replay
                    ps.pfasst_iteration(pf, False)
                ps.pfasst_iteration(pf, True)
            else:
                ps.pfasst_iterations(pf, 4, True)
        res = torch.empty((nts, 5, 3, syn.ncoef(Tf)), dtype=torch.complex128, device=DEV)
        for n in range(nts):
            for k in range(5):
                ps.pfasst_get(pf, 0, n, k, res[n, k])
        ps.pfsh_sync_status()
        pf.close()
        return res.cpu().numpy()

    ref = run(1, "single")
    assert np.array_equal(ref, run(3, "single"))
    assert np.array_equal(ref, run(3, "block"))
    assert np.array_equal(ref, run(1, "block"))


def test_pfasst_residual_tracks_the_iteration():
    """pfasst_residual equals the relative max-norm change of every slice's
    fine end value between calls (computed here from pfasst_get), and the
    PFASST iteration contracts it."""
    Tf, Tc, nts, dt = 21, 10, 4, 600.0
    gf, gc = syn.gaussian_grid_size(Tf), syn.gaussian_grid_size(Tc)
    pf = ps.pfasst_create(nts, 5, 3, Tf, *gf, Tc, *gc, dt, A, OM, syn.NU, PHIBAR, "fp64")
    ps.pfasst_set_initial(pf, cuda(state_of(Tf, 31)[0]))
    ps.pfasst_predict(pf)
    res = torch.empty(nts, dtype=torch.float64, device=DEV)
    out = torch.empty((3, syn.ncoef(Tf)), dtype=torch.complex128, device=DEV)

    def ends():
        v = []
        for n in range(nts):
            ps.pfasst_get(pf, 0, n, 4, out)
            ps.pfsh_sync_status()
            v.append(out.cpu().numpy().copy())
        return v

    ps.pfasst_residual(pf, res)
    prev = ends()
    history = []
    for it in range(6):
        ps.pfasst_iteration(pf, False)
        ps.pfasst_residual(pf, res)
        cur = ends()
        got = res.cpu().numpy()
        for n in range(nts):
            d = max(np.abs(cur[n].real - prev[n].real).max(), np.abs(cur[n].imag - prev[n].imag).max())
            v = max(np.abs(cur[n].real).max(), np.abs(cur[n].imag).max())
            assert got[n] == pytest.approx(d / v, rel=1e-12, abs=1e-300), (it, n)
        history.append(got.max())
        prev = cur
    # measured: 1.2e-4, 1.0e-4, 7.2e-5, 3.6e-5, 2.5e-5, 2.4e-6
    assert all(b < a for a, b in zip(history, history[1:])), history
    assert history[-1] < 0.05 * history[0], history
    pf.close()
