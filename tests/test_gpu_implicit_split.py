"""The SDC node solve in two substeps (swe_params.implicit_split: physical
linear terms with the previous iterate's diffusion, then diffusion, each with
its own correction term) against the oracle, for the paper's split and with
the Coriolis term implicit: SDC sweeps of the batched node update and PFASST
(whose coarse chain runs the substeps inside the fused chain step).

The substeps change each sweep (checked: one sweep differs from the
one-solve sweep) but not its fixed point (pinned in the oracle tests).
nu = 5e5 m^2/s makes the difference large.  Bounds as for the one-solve
forms (FP64).
"""
import numpy as np
import pytest

import synthetic as syn
from oracle.sht import pack, unpack
from oracle.swe import SWEParams
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
NU = 5e5


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


def cuda(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.complex128, device=DEV)


def state_of(T, seed, batch=1):
    s = syn.random_spectrum(T, (batch, 3), seed=seed, rms=1e-5)
    s[:, 0] *= 1e3
    return s + syn.zonal_jet(T)[None]


def oparams(coriolis, split=True):
    return SWEParams(a=A, omega=OM, g=G, nu=NU, phibar=PHIBAR, coriolis_implicit=coriolis, implicit_split=split)


@pytest.mark.parametrize("coriolis", [False, True])
@pytest.mark.parametrize("B", [3, 1])
def test_split_sdc_sweeps_with_tau_match_oracle(coriolis, B):
    T, nodes, dt = 31, 5, 600.0
    nlat, nlon = syn.gaussian_grid_size(T)
    st = state_of(T, 15, B)
    tau = syn.random_spectrum(T, (nodes, B, 3), seed=16, rms=1e-9)
    tau[0] = 0

    def gpu(split):
        plan = ps.sht_plan_create(T, nlat, nlon, 10, "fp64")
        ctx = ps.swe_ctx_create(plan, A, OM, NU, PHIBAR, coriolis_implicit=coriolis, implicit_split=split)
        lvl = ps.sdc_level_create(ctx, nodes, dt, B)
        th = torch.empty((nodes, B, 3, syn.ncoef(T)), dtype=torch.complex128, device=DEV)
        fE, fI = torch.empty_like(th), torch.empty_like(th)
        ps.sdc_spread(lvl, cuda(st), th, fE, fI)
        ps.sdc_sweep(lvl, th, fE, fI, cuda(tau))
        first = th.clone()
        ps.sdc_sweep(lvl, th, fE, fI, cuda(tau))
        ps.pfsh_sync_status()
        return first.cpu().numpy(), th.cpu().numpy(), fI.cpu().numpy()

    first, th, fI = gpu(True)
    first_one, _, _ = gpu(False)
    assert rel(first, first_one) > 1e-9          # the substeps change a sweep
    lv = SDCLevel(T, nlat, nlon, nodes, dt, oparams(coriolis))
    for b in range(B):
        t_, e_, i_ = lv.spread(unpack(st[b], T))
        for _ in range(2):
            t_, e_, i_ = lv.sweep(t_, e_, i_, unpack(tau[:, b], T))
        assert rel(th[:, b], pack(t_, T)) < 1e-12
        assert rel(fI[:, b], pack(i_, T)) < 1e-12


@pytest.mark.parametrize("coriolis", [False, True])
@pytest.mark.parametrize("nts,groups", [(4, 0), (9, 2)])
def test_split_pfasst_matches_oracle(coriolis, nts, groups):
    Tf, Tc, dt, nf, nc, iters = 21, 10, 600.0, 5, 3, 3
    gf, gc = syn.gaussian_grid_size(Tf), syn.gaussian_grid_size(Tc)
    st0 = state_of(Tf, 24)[0]
    pf = ps.pfasst_create(nts, nf, nc, Tf, *gf, Tc, *gc, dt, A, OM, NU, PHIBAR, "fp64", slice_groups=groups,
                          coriolis_implicit=coriolis, implicit_split=True)
    ps.pfasst_set_initial(pf, cuda(st0))
    ps.pfasst_predict(pf)
    p = oparams(coriolis)
    o = PFASST(SDCLevel(Tf, *gf, nf, dt, p), SDCLevel(Tc, *gc, nc, dt, p), nts)
    o.predict(unpack(st0, Tf))
    out = torch.empty((3, syn.ncoef(Tf)), dtype=torch.complex128, device=DEV)
    for it in range(iters):
        last = it == iters - 1
        ps.pfasst_iteration(pf, last)
        o.iteration(last)
    ps.pfsh_sync_status()
    for n in range(nts):
        for k in range(nf):
            ps.pfasst_get(pf, 0, n, k, out)
            assert rel(out.cpu().numpy(), pack(o.th_f[n, k], Tf)) < 1e-11, (n, k)
    pf.close()
