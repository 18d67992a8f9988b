"""Gaussian-dome study of Section 6.1 on the GPU (error against a serial SDC
reference as a function of time-step size and of the number of PFASST
iterations, for the coarsening ratios alpha = 1/5, 1/2, 4/5).

Run on a GPU:  python tests/dome_study.py [--window 102400] [--out study.json]

The set-up and the readings are those of tests/golden/gaussian_dome_sec6_1.json
(the same file test_gpu_dome.py reads): u = v = 0, h = 29400 m + 6000 m
exp(-alpha_d (d/a)^2) centred at lambda = pi, phi = pi/4, alpha_d = 225, nu =
1e5 m^2/s, T255 (R_f = 256) on 384 x 768; PFASST(16, 5, 3, N_PF, alpha) with
coarse truncation T_c = floor(alpha R_f) - 1 on its own Gaussian grid;
reference SDC(5 nodes, 8 sweeps) in FP64 on the fine grid with the step
window / ceil(window / 60 s) (60 s in the paper, which does not divide its
102,400 s window; the nearest step that does).  Errors: Eq. error_norm_r_norm
on the geopotential at the end of the window, R_norm = 32 and 256.  All runs
are FP64 GPU runs of the library; the oracle only projects the dome.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
for _p in (ROOT, HERE):
    if _p not in sys.path:
        sys.path.insert(0, _p)

import synthetic as syn  # noqa: E402

with open(os.path.join(HERE, "golden", "gaussian_dome_sec6_1.json")) as _fh:
    GOLDEN = json.load(_fh)
P, R = GOLDEN["printed"], GOLDEN["readings"]
TF = P["R_f"] - 1
NTS, NF, NC = P["pfasst"]["n_ts"], P["pfasst"]["fine_nodes"], P["pfasst"]["coarse_nodes"]
ALPHAS = {"1/5": (1, 5), "1/2": (1, 2), "4/5": (4, 5)}


def coarse_T(alpha):
    """Reading R20: R_c = floor(alpha R_f) zonal wavenumbers, T_c = R_c - 1."""
    num, den = alpha
    return P["R_f"] * num // den - 1


def e_norm(phi, ref, T, Rn):
    """Eq. error_norm_r_norm on packed triangles (m-major, n = m..T)."""
    ms = np.concatenate([np.full(T + 1 - m, m) for m in range(T + 1)])
    ns = np.concatenate([np.arange(m, T + 1) for m in range(T + 1)])
    keep = (ms <= Rn) & (ns <= Rn)
    return float(np.abs(phi[keep] - ref[keep]).max() / np.abs(ref[keep]).max())


def dome_state():
    """The dome projected by the oracle's analysis (packed [3][ncoef]) and Phibar."""
    from oracle.sht import SHT, pack
    nlat, nlon = syn.gaussian_grid_size(TF)
    o = SHT(TF, nlat, nlon, L=TF + 1)
    lam = 2.0 * math.pi * np.arange(nlon) / nlon
    h = P["h_bar_m"] + syn.gaussian_bump(o.mu, lam, amplitude=P["A_m"],
                                         width=1.0 / math.sqrt(R["dome_sharpness_alpha"]),
                                         lam_c=math.pi, phi_c=math.pi / 4)
    st = np.zeros((3, TF + 1, TF + 1), dtype=np.complex128)
    st[0] = o.analysis(syn.GRAVITY * h, TF + 1)
    st = pack(st, TF)
    st[0, 0] = st[0, 0].real
    return st, st[0, 0].real / math.sqrt(2.0)


def sdc_reference(ps, torch, st, phibar, window, dt_target=60.0):
    """SDC(5, 8) in FP64 with the step window / ceil(window / dt_target)."""
    steps = int(math.ceil(window / dt_target - 1e-9))
    dt = window / steps
    nlat, nlon = syn.gaussian_grid_size(TF)
    plan = ps.sht_plan_create(TF, nlat, nlon, 5, "fp64")
    ctx = ps.swe_ctx_create(plan, syn.EARTH_RADIUS, syn.OMEGA, syn.NU, phibar)
    lvl = ps.sdc_level_create(ctx, NF, dt, 1)
    x = torch.tensor(st[None], dtype=torch.complex128, device="cuda")
    th = torch.empty((NF, 1, 3, syn.ncoef(TF)), dtype=torch.complex128, device="cuda")
    fE, fI = torch.empty_like(th), torch.empty_like(th)
    for _ in range(steps):
        ps.sdc_spread(lvl, x, th, fE, fI)
        for _ in range(P["reference_sdc"]["sweeps"]):
            ps.sdc_sweep(lvl, th, fE, fI, None)
        x = th[NF - 1].clone()
    ps.pfsh_sync_status()
    return x[0].cpu().numpy(), dt


def pfasst_run(ps, torch, st, phibar, window, dt, alpha, npf, prec="fp64"):
    """PFASST(16, 5, 3, npf, alpha) over the window in blocks of 16 slices."""
    Tc = coarse_T(alpha)
    gf, gc = syn.gaussian_grid_size(TF), syn.gaussian_grid_size(Tc)
    blocks = int(round(window / (NTS * dt)))
    if abs(blocks * NTS * dt - window) > 1e-6 * window:
        raise ValueError("the window must be a whole number of PFASST blocks")
    pf = ps.pfasst_create(NTS, NF, NC, TF, *gf, Tc, *gc, dt, syn.EARTH_RADIUS, syn.OMEGA, syn.NU, phibar, prec)
    x = torch.tensor(st, dtype=torch.complex128, device="cuda")
    out = torch.empty_like(x)
    for _ in range(blocks):
        ps.pfasst_set_initial(pf, x)
        ps.pfasst_predict(pf)
        ps.pfasst_iterations(pf, npf, True)
        ps.pfasst_get(pf, 0, NTS - 1, NF - 1, out)
        x = out.clone()
    ps.pfsh_sync_status()
    pf.close()
    return x.cpu().numpy()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--window", type=float, default=P["window_s"])
    ap.add_argument("--dts", default="400,200,100,50")
    ap.add_argument("--npf", default="1,2,3,4,5,6,8,10")
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    import torch
    from _lib import ensure_built
    ensure_built()
    import paper_1904_05988_gb300 as ps
    st, phibar = dome_state()
    t0 = time.time()
    ref, dt_ref = sdc_reference(ps, torch, st, phibar, args.window)
    res = {"window_s": args.window, "reference": f"SDC(5,8) FP64, dt_ref = {dt_ref:.4f} s",
           "reference_s": time.time() - t0, "dt_sweep": {}, "npf_sweep": {}}
    print(json.dumps({"reference": res["reference"], "seconds": res["reference_s"]}), flush=True)
    for name, alpha in ALPHAS.items():
        for dt in [float(v) for v in args.dts.split(",")]:
            try:
                phi = pfasst_run(ps, torch, st, phibar, args.window, dt, alpha, 8)[0]
                e = [e_norm(phi, ref[0], TF, Rn) for Rn in (32, 255)]
                if not np.all(np.isfinite(phi.view(np.float64))) or max(e) > 1.0:
                    e = None   # unstable at this step
            except ValueError:
                e = None
            res["dt_sweep"].setdefault(name, {})[str(dt)] = e
            print(json.dumps({"alpha": name, "dt": dt, "N_PF": 8, "E32_E256": e}), flush=True)
        for npf in [int(v) for v in args.npf.split(",")]:
            phi = pfasst_run(ps, torch, st, phibar, args.window, 100.0, alpha, npf)[0]
            e = [e_norm(phi, ref[0], TF, Rn) for Rn in (32, 255)]
            res["npf_sweep"].setdefault(name, {})[str(npf)] = e
            print(json.dumps({"alpha": name, "dt": 100.0, "N_PF": npf, "E32_E256": e}), flush=True)
    res["seconds"] = time.time() - t0
    if args.out:
        with open(args.out, "w") as fh:
            json.dump(res, fh, indent=1)
    print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
