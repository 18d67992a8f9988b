"""Propagation of a Gaussian dome (Section 6.1): accuracy of PFASST-SH against
a serial SDC reference, in the paper's normalised error norm
E_{R_norm} = max_{m <= n <= R_norm} |phi - phi_ref| / max_{m <= n <= R_norm} |phi_ref|
(Eq. error_norm_r_norm) on the geopotential.

Set-up as in the paper: u = v = 0, h = 29400 m + 6000 m exp(-alpha (d/a)^2)
centred at lambda = pi, phi = pi/4 (chordal distance d), nu = 1e5 m^2/s,
T255 (R_f = 256) on 384 x 768; PFASST(n_ts = 16, 5 / 3 Gauss-Lobatto nodes,
N_PF = 8 iterations, coarse truncation 4/5: T203 on 306 x 612) with dt = 100 s;
reference SDC(5 nodes, 8 sweeps) in FP64 with dt_ref = 60 s on the same grid.
Readings: the dome sharpness alpha is not printed; alpha = 225 (the width
1/15 rad of the benchmark's bump).  The comparison is made at t = 4800 s,
the first time both step sizes reach (3 PFASST blocks of 16 x 100 s, 80
reference steps), instead of the paper's 102,400 s window.

Both runs are GPU runs of the library (the reference is the serial method the
paper uses as reference); the oracle projects the dome and checks the first
two reference steps.  The printed
values and the readings come from tests/golden/gaussian_dome_sec6_1.json.
Bounds: measured values on GB300 in brackets.
"""
import json
import math
import os

import numpy as np
import pytest

import synthetic as syn
from oracle.sht import SHT, pack
from _lib import ensure_built

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
ensure_built()
import paper_1904_05988_gb300 as ps  # noqa: E402
import sys  # noqa: E402
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

DEV = torch.device("cuda:0")
with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "gaussian_dome_sec6_1.json")) as _fh:
    _G = json.load(_fh)       # the printed set-up of Section 6.1 and the readings around it
_P, _R = _G["printed"], _G["readings"]
TF = _P["R_f"] - 1
TC = _P["R_f"] * _P["pfasst"]["alpha"][0] // _P["pfasst"]["alpha"][1] - 1
NTS, NF, NC, NPF = (_P["pfasst"][k] for k in ("n_ts", "fine_nodes", "coarse_nodes", "N_PF"))
DT, DT_REF, T_END = _P["dt_s"], _R["reference_dt_s"], _R["window_used_s"]
HBAR, AMP, ALPHA = _P["h_bar_m"], _P["A_m"], _R["dome_sharpness_alpha"]
assert (TF, TC, NTS, NF, NC, NPF) == (255, 203, 16, 5, 3, 8)
BOUNDS = {  # E_32, E_64, E_256 of PFASST against the reference
    "fp64": (1e-11, 5e-11, 2e-7),       # (1.3e-12, 6.4e-12, 3.5e-8)
    "bf16x3": (5e-10, 5e-10, 2e-7),     # (1.0e-10, 1.0e-10, 3.5e-8)
}


def e_norm(phi, ref, T, R):
    """Eq. error_norm_r_norm on packed triangles (m-major, n = m..T)."""
    ms = np.concatenate([np.full(T + 1 - m, m) for m in range(T + 1)])
    ns = np.concatenate([np.arange(m, T + 1) for m in range(T + 1)])
    keep = (ms <= R) & (ns <= R)
    return float(np.abs(phi[keep] - ref[keep]).max() / np.abs(ref[keep]).max())


@pytest.fixture(scope="module")
def dome():
    nlat, nlon = syn.gaussian_grid_size(TF)
    o = SHT(TF, nlat, nlon, L=TF + 1)
    lam = 2.0 * math.pi * np.arange(nlon) / nlon
    h = HBAR + syn.gaussian_bump(o.mu, lam, amplitude=AMP, width=1.0 / math.sqrt(ALPHA), lam_c=math.pi,
                                 phi_c=math.pi / 4)
    st = np.zeros((3, TF + 1, TF + 1), dtype=np.complex128)
    st[0] = o.analysis(syn.GRAVITY * h, TF + 1)
    st = pack(st, TF)
    st[0, 0] = st[0, 0].real
    phibar = st[0, 0].real / math.sqrt(2.0)
    return st, phibar


@pytest.fixture(scope="module")
def reference(dome):
    """SDC(5, 8) in FP64, dt_ref = 60 s, to T_END."""
    st, phibar = dome
    nlat, nlon = syn.gaussian_grid_size(TF)
    plan = ps.sht_plan_create(TF, nlat, nlon, 5, "fp64")
    ctx = ps.swe_ctx_create(plan, syn.EARTH_RADIUS, syn.OMEGA, syn.NU, phibar)
    lvl = ps.sdc_level_create(ctx, NF, DT_REF, 1)
    x = torch.tensor(st[None], dtype=torch.complex128, device=DEV)
    th = torch.empty((NF, 1, 3, syn.ncoef(TF)), dtype=torch.complex128, device=DEV)
    fE, fI = torch.empty_like(th), torch.empty_like(th)
    for _ in range(int(round(T_END / DT_REF))):
        ps.sdc_spread(lvl, x, th, fE, fI)
        for _ in range(8):
            ps.sdc_sweep(lvl, th, fE, fI, None)
        x = th[NF - 1].clone()
    ps.pfsh_sync_status()
    return x[0].cpu().numpy()


def test_reference_steps_match_oracle(dome):
    """The reference integrator against the oracle on the dome itself: two
    SDC(5, 8) steps of dt_ref in FP64 at T255 (oracle.sdc: spread, then 8
    sweeps per step).  Bounds: the FP64 right-hand side matches the oracle to
    ~5e-11 relative (test_gpu_fp64.py), and the change of the state over the
    two steps integrates it (1e-9); the state's own error is then bounded by
    that times the size of the change relative to the state."""
    from oracle.sdc import SDCLevel
    from oracle.sht import unpack
    from oracle.swe import SWEParams
    st, phibar = dome
    nlat, nlon = syn.gaussian_grid_size(TF)
    plan = ps.sht_plan_create(TF, nlat, nlon, 5, "fp64")
    ctx = ps.swe_ctx_create(plan, syn.EARTH_RADIUS, syn.OMEGA, syn.NU, phibar)
    lvl = ps.sdc_level_create(ctx, NF, DT_REF, 1)
    x = torch.tensor(st[None], dtype=torch.complex128, device=DEV)
    th = torch.empty((NF, 1, 3, syn.ncoef(TF)), dtype=torch.complex128, device=DEV)
    fE, fI = torch.empty_like(th), torch.empty_like(th)
    for _ in range(2):
        ps.sdc_spread(lvl, x, th, fE, fI)
        for _ in range(8):
            ps.sdc_sweep(lvl, th, fE, fI, None)
        x = th[NF - 1].clone()
    ps.pfsh_sync_status()
    got = x[0].cpu().numpy()
    p = SWEParams(a=syn.EARTH_RADIUS, omega=syn.OMEGA, g=syn.GRAVITY, nu=syn.NU, phibar=phibar)
    lv = SDCLevel(TF, nlat, nlon, NF, DT_REF, p)
    y = unpack(st, TF)
    for _ in range(2):
        t, FE, FI = lv.spread(y)
        for _ in range(8):
            t, FE, FI = lv.sweep(t, FE, FI)
        y = t[-1]
    ref = pack(y, TF)
    e_state = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    e_change = np.linalg.norm((got - st) - (ref - st)) / np.linalg.norm(ref - st)
    print(f"\ndome reference, 2 SDC(5,8) steps of {DT_REF:.0f} s vs oracle: state {e_state:.2e}, change {e_change:.2e}")
    moved = np.linalg.norm(ref - st) / np.linalg.norm(ref)
    assert e_change < 1e-9 and e_state < 1e-9 * moved + 1e-15, (e_change, e_state, moved)


@pytest.mark.parametrize("form", ["fp64", "bf16x3"])
def test_gaussian_dome_pfasst_against_sdc_reference(form, dome, reference):
    if form not in ps.available_precisions():
        pytest.skip(f"{form} not built")
    st, phibar = dome
    gf, gc = syn.gaussian_grid_size(TF), syn.gaussian_grid_size(TC)
    pf = ps.pfasst_create(NTS, NF, NC, TF, *gf, TC, *gc, DT, syn.EARTH_RADIUS, syn.OMEGA, syn.NU, phibar, form)
    x = torch.tensor(st, dtype=torch.complex128, device=DEV)
    out = torch.empty_like(x)
    for _ in range(int(round(T_END / (NTS * DT)))):
        ps.pfasst_set_initial(pf, x)
        ps.pfasst_predict(pf)
        ps.pfasst_iterations(pf, NPF, True)
        ps.pfasst_get(pf, 0, NTS - 1, NF - 1, out)
        x = out.clone()
    ps.pfsh_sync_status()
    phi = x.cpu().numpy()[0]
    errs = [e_norm(phi, reference[0], TF, R) for R in (32, 64, 255)]
    print(f"\nGaussian dome, t = {T_END:.0f} s, PFASST({NTS},{NF},{NC},{NPF}, T{TC}) {form} vs SDC(5,8): "
          f"E_32 {errs[0]:.3e}  E_64 {errs[1]:.3e}  E_256 {errs[2]:.3e}")
    assert all(e < b for e, b in zip(errs, BOUNDS[form])), errs
    pf.close()


# ---------------------------------------------------------------------------
# Sensitivity to the number of iterations (the closing study of Section 6.1):
# with dt = 100 s fixed, the error stops decreasing beyond a threshold N_PF,
# because the coarse level cannot represent the modes above T_c; the paper
# reads the thresholds N_PF = 2, 4 and 6 for alpha = 1/5, 1/2 and 4/5 off its
# R_norm = 256 figure over 102,400 s, and the plateau error falls as alpha
# grows.  This test runs 12,800 s (8 PFASST blocks).  Over that window the
# alpha = 1/5 error on the full spectrum is dominated from N_PF = 1 on by the
# modes the T50 coarse level cannot carry (it falls less than 2x from 1 to 8
# iterations), so the threshold is read on the large scales (R_norm = 32),
# where the iteration converges what the coarse levels represent; it is taken
# as the first N_PF after which no later N_PF cuts the error by 4x or more.
# The full-window thresholds on R_norm = 256 come from tests/dome_study.py
# and are reported beside the paper's, not asserted.
# ---------------------------------------------------------------------------
STUDY_WINDOW, STUDY_NPF = 12800.0, (1, 2, 4, 6, 8)


def threshold(errs):
    """First N_PF after which no later N_PF reduces the error by 4x or more."""
    return min(n for n in STUDY_NPF if min(errs[k] for k in STUDY_NPF if k >= n) > errs[n] / 4.0)


def test_iteration_count_thresholds_follow_the_coarsening_ratio(dome):
    import dome_study as ds
    st, phibar = dome
    ref, _ = ds.sdc_reference(ps, torch, st, phibar, STUDY_WINDOW)
    e32, e256 = {}, {}
    for name, alpha in ds.ALPHAS.items():
        e32[name], e256[name] = {}, {}
        for npf in STUDY_NPF:
            phi = ds.pfasst_run(ps, torch, st, phibar, STUDY_WINDOW, 100.0, alpha, npf)[0]
            e32[name][npf] = ds.e_norm(phi, ref[0], TF, 32)
            e256[name][npf] = ds.e_norm(phi, ref[0], TF, 255)
        print(f"\nalpha {name}: E_32 " + " ".join(f"{e32[name][n]:.2e}" for n in STUDY_NPF) +
              "  E_256 " + " ".join(f"{e256[name][n]:.2e}" for n in STUDY_NPF))
    t32 = {a: threshold(e32[a]) for a in ds.ALPHAS}
    print("thresholds (R_norm = 32):", t32)
    # iterating pays before the threshold, for every ratio
    for a in ds.ALPHAS:
        assert e32[a][1] > 4 * e32[a][8] and e256[a][1] > 1.2 * e256[a][8], a
    # the paper's end points: 2 iterations for alpha = 1/5, 6 for alpha = 4/5;
    # thresholds do not decrease as alpha grows
    assert t32["1/5"] == 2 and t32["4/5"] == 6, t32
    assert t32["1/5"] <= t32["1/2"] <= t32["4/5"], t32
    # past the threshold the error stays put (within 3x from 6 to 8 iterations)
    for a in ds.ALPHAS:
        assert e32[a][8] > e32[a][6] / 3 and e256[a][8] > e256[a][6] / 3, a
    # the plateau error falls as alpha grows; aggressive coarsening stagnates
    assert e256["1/5"][8] > 3 * e256["1/2"][8] > 3 * 3 * e256["4/5"][8]
    assert e256["1/5"][8] > 0.5 * e256["1/5"][2]
