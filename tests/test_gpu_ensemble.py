"""Ensembles of independent PFASST instances (uneven batches): members with
different truncations, grids, slice counts and precisions advanced together,
each member on its own stream pair, iteration blocks in one CUDA graph.

Parity: an ensemble member computes exactly what the same configuration run
alone computes (same kernels, same batch paths, its own buffers), so the
members are compared bitwise with individual runs; the individual path is
itself checked against the oracle in test_gpu_fp64 / test_gpu_mixed.

The uneven batch of 48 instances draws T from {63, 127, 170, 255} (seed 4),
coarse level T/2, 8 slices, 5/3 Gauss-Lobatto nodes, dt = 120 * 256/(T+1) s;
initial states are the balanced jet plus seeded n^-3 vorticity and
divergence perturbations (generated on the host, no transform needed).
"""
import numpy as np
import pytest

import synthetic as syn
from _lib import ensure_built

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
ensure_built()
import paper_1904_05988_gb300 as ps  # noqa: E402

DEV = torch.device("cuda:0")
A, OM, G = syn.EARTH_RADIUS, syn.OMEGA, syn.GRAVITY
PHIBAR = G * syn.MEAN_DEPTH


def initial_state(T, seed):
    st = syn.zonal_jet(T)
    pert = syn.random_spectrum(T, (2,), seed=seed, rms=1e-6)
    st[1] += pert[0]
    st[2] += pert[1]
    return st


def config(T, Tc, nts, prec, dt=None, groups=0):
    gf, gc = syn.gaussian_grid_size(T), syn.gaussian_grid_size(Tc)
    dt = 120.0 * 256 / (T + 1) if dt is None else dt
    return ps.pfasst_config(nts, 5, 3, T, *gf, Tc, *gc, dt, A, OM, syn.NU, PHIBAR, prec, groups)


def end_values(pf, cfg):
    out = torch.empty((cfg.n_ts, 3, syn.ncoef(cfg.Tf)), dtype=torch.complex128, device=DEV)
    for n in range(cfg.n_ts):
        ps.pfasst_get(pf, 0, n, 4, out[n])
    ps.pfsh_sync_status()
    return out.cpu().numpy()


def run_alone(cfg, st, iters):
    pf = ps.pfasst_create(cfg.n_ts, 5, 3, cfg.Tf, cfg.nlat_f, cfg.nlon_f, cfg.Tc, cfg.nlat_c, cfg.nlon_c, cfg.dt,
                          A, OM, syn.NU, PHIBAR, cfg.prec, cfg.slice_groups)
    ps.pfasst_set_initial(pf, torch.tensor(st, dtype=torch.complex128, device=DEV))
    ps.pfasst_predict(pf)
    ps.pfasst_iterations(pf, iters, True)
    res = end_values(pf, cfg)
    pf.close()
    return res


def run_ensemble(cfgs, states, iters, rounds):
    ens = ps.pfasst_ensemble_create(cfgs)
    for _ in range(rounds):    # eager, graph capture, graph replay
        for i, st in enumerate(states):
            ps.pfasst_set_initial(ps.pfasst_ensemble_member(ens, i), torch.tensor(st, dtype=torch.complex128,
                                                                                  device=DEV))
        ps.pfasst_ensemble_predict(ens)
        ps.pfasst_ensemble_iterations(ens, iters, True)
    res = [end_values(m, c) for m, c in zip(ens.members, cfgs)]
    ens.close()
    return res


def test_mixed_ensemble_matches_members_run_alone():
    forms = ps.available_precisions()
    specs = [(21, 10, 4, "fp64", 0), (31, 15, 8, "bf16x3", 2), (42, 21, 4, "fp32", 0), (63, 31, 8, "bf16x3", 0),
             (21, 21, 3, "fp64", 0)]
    specs = [s for s in specs if s[3] in forms]
    cfgs = [config(T, Tc, nts, prec, dt=600.0, groups=g) for T, Tc, nts, prec, g in specs]
    states = [initial_state(s[0], 40 + i) for i, s in enumerate(specs)]
    together = run_ensemble(cfgs, states, 3, rounds=3)
    for cfg, st, got in zip(cfgs, states, together):
        assert np.all(np.isfinite(got.view(np.float64)))
        assert np.array_equal(got, run_alone(cfg, st, 3)), (cfg.Tf, cfg.prec)


def test_uneven_batch_of_48_instances():
    if "bf16x3" not in ps.available_precisions():
        pytest.skip("bf16x3 not built")
    rng = np.random.default_rng(4)
    Ts = [int(t) for t in rng.choice([63, 127, 170, 255], size=48)]
    cfgs = [config(T, T // 2, 8, "bf16x3") for T in Ts]
    states = [initial_state(T, 100 + i) for i, T in enumerate(Ts)]
    together = run_ensemble(cfgs, states, 4, rounds=2)
    for got in together:
        assert np.all(np.isfinite(got.view(np.float64)))
    picks = {}
    for i, T in enumerate(Ts):
        picks.setdefault(T, i)
    for T, i in picks.items():   # one member of every truncation, including T170 (nlon 516 = 2^2 3 43)
        assert np.array_equal(together[i], run_alone(cfgs[i], states[i], 4)), T


def test_ensemble_member_T170_matches_oracle():
    """An ensemble member at the uneven batch's odd size, T170/T85 on 258 x 516
    / 130 x 260 (nlon = 2^2 3 43, 2^2 5 13: the run-time FFT path and row
    centring), beside a T63/T31 member, against the oracle: predictor and a
    block of two iterations, end values of every slice (3xBF16: the end-value
    bound of the mixed PFASST tests and the low-band change law of
    tests/_lib.py).  The oracle runs its slice-independent steps on all host
    cores."""
    import os
    from oracle.pfasst import PFASST
    from oracle.pool import SlicePool
    from oracle.sdc import SDCLevel
    from oracle.sht import pack, unpack
    from oracle.swe import SWEParams
    from _lib import change_bound
    if "bf16x3" not in ps.available_precisions():
        pytest.skip("bf16x3 not built")
    specs = [(170, 85, 4), (63, 31, 4)]
    cfgs = [config(T, Tc, nts, "bf16x3") for T, Tc, nts in specs]
    states = [initial_state(T, 60 + i) for i, (T, _, _) in enumerate(specs)]
    got = run_ensemble(cfgs, states, 2, rounds=1)[0]
    T, Tc, nts = specs[0]
    p = SWEParams(a=A, omega=OM, g=G, nu=syn.NU, phibar=PHIBAR)
    gf, gc = syn.gaussian_grid_size(T), syn.gaussian_grid_size(Tc)
    f, c = SDCLevel(T, *gf, 5, cfgs[0].dt, p), SDCLevel(Tc, *gc, 3, cfgs[0].dt, p)
    with SlicePool({"f": f.args, "c": c.args}, workers=min(nts, os.cpu_count() or 1)) as pool:
        ref = PFASST(f, c, nts, pool=pool).run(unpack(states[0], T), 2)
    st0 = states[0]
    errs = [np.linalg.norm(got[n] - pack(ref[n], T)) / np.linalg.norm(pack(ref[n], T)) for n in range(nts)]
    chg = np.linalg.norm((got[-1] - st0) - (pack(ref[-1], T) - st0)) / np.linalg.norm(pack(ref[-1], T) - st0)
    print(f"\nensemble member T{T}/T{Tc} x {nts}: end values {max(errs):.2e}, change {chg:.2e}")
    assert max(errs) < 5e-7
    assert chg < change_bound("bf16x3", T)
