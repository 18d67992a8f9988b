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
paper uses as reference); the oracle only projects the dome.  The printed
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
