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
