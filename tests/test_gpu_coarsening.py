"""Spatial coarsening ratios alpha (Section 5.1.2: the coarse level keeps
R_c = floor(alpha R_f) zonal wavenumbers) on Gaussian grids whose longitude
counts are not powers of two.

* Parity at T63 (R_f = 64) for alpha in {1/5, 4/5, 19/20, 1}: coarse T11 on
  18 x 36, T50 on 78 x 156 (2^2 3 13), T59 on 90 x 180 (2^2 3^2 5), T63 on
  96 x 192; predictor and two iterations against the oracle (FP64).
* The benchmark's fine level T255 with every ratio, FP64: coarse T50 on
  78 x 156, T203 on 306 x 612 (2^2 3^2 17), T242 on 366 x 732 (2^2 3 61),
  T255 on 384 x 768.  8 slices from the jet plus the Gaussian height bump.
  Every ratio approaches the same solution (the fixed point of Algorithm 1
  is set by the fine level; the ratio only changes how fast it is reached):
  the error of the end values' change from the initial value, against
  alpha = 1 iterated to convergence, must fall over 6 iterations, and reach
  1e-2 for alpha >= 4/5.
"""
import math

import numpy as np
import pytest

import synthetic as syn
from oracle.sht import SHT, pack, unpack
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
ALPHAS = [(1, 5), (4, 5), (19, 20), (1, 1)]


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


def cuda(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.complex128, device=DEV)


def coarse_T(Tf, alpha):
    return (Tf + 1) * alpha[0] // alpha[1] - 1


@pytest.mark.parametrize("alpha", ALPHAS)
def test_coarsening_ratio_matches_oracle_T63(alpha):
    Tf, nts, dt = 63, 4, 600.0
    Tc = coarse_T(Tf, alpha)
    gf, gc = syn.gaussian_grid_size(Tf), syn.gaussian_grid_size(Tc)
    s = syn.random_spectrum(Tf, (3,), seed=63, rms=1e-5)
    s[0] *= 1e3
    st0 = s + syn.zonal_jet(Tf)
    pf = ps.pfasst_create(nts, 5, 3, Tf, *gf, Tc, *gc, dt, A, OM, syn.NU, PHIBAR, "fp64")
    ps.pfasst_set_initial(pf, cuda(st0))
    ps.pfasst_predict(pf)
    ps.pfasst_iteration(pf, False)
    ps.pfasst_iteration(pf, True)
    ps.pfsh_sync_status()
    p = SWEParams(a=A, omega=OM, g=G, nu=syn.NU, phibar=PHIBAR)
    o = PFASST(SDCLevel(Tf, *gf, 5, dt, p), SDCLevel(Tc, *gc, 3, dt, p), nts)
    ref = o.run(unpack(st0, Tf), 2)
    out = torch.empty((3, syn.ncoef(Tf)), dtype=torch.complex128, device=DEV)
    for n in range(nts):
        ps.pfasst_get(pf, 0, n, 4, out)
        assert rel(out.cpu().numpy(), pack(ref[n], Tf)) < 1e-11, (alpha, n)
    pf.close()


def test_coarsening_ratios_at_T255():
    Tf, nts, dt, iters = 255, 8, 120.0, 6
    gf = syn.gaussian_grid_size(Tf)
    sht = SHT(Tf, *gf, L=Tf + 1)
    lam = 2.0 * math.pi * np.arange(gf[1]) / gf[1]
    lam_c, phi_c = syn.bump_center(2)
    st = unpack(syn.zonal_jet(Tf), Tf)
    st[0] += sht.analysis(G * syn.gaussian_bump(sht.mu, lam, amplitude=120.0, width=1.0 / 15.0, lam_c=lam_c,
                                                phi_c=phi_c), Tf + 1)
    st0 = pack(st, Tf)
    phibar = st[0, 0, 0].real / math.sqrt(2.0)
    out = torch.empty((nts, 3, syn.ncoef(Tf)), dtype=torch.complex128, device=DEV)

    def run(alpha, n_iter):
        Tc = coarse_T(Tf, alpha)
        gc = syn.gaussian_grid_size(Tc)
        pf = ps.pfasst_create(nts, 5, 3, Tf, *gf, Tc, *gc, dt, A, OM, syn.NU, phibar, "fp64")
        ps.pfasst_set_initial(pf, cuda(st0))
        ps.pfasst_predict(pf)
        ends = []
        for it in range(n_iter):
            ps.pfasst_iteration(pf, it == n_iter - 1)
            for n in range(nts):
                ps.pfasst_get(pf, 0, n, 4, out[n])
            ends.append(out.cpu().numpy() - st0[None])
        ps.pfsh_sync_status()
        pf.close()
        return ends, Tc, gc

    # converged reference: alpha = 1 iterated to the fixed point of Algorithm 1
    ref_runs, _, _ = run((1, 1), 2 * nts)
    ref = ref_runs[-1]
    assert rel(ref_runs[-1], ref_runs[-2]) < 1e-9
    lines = []
    for alpha in ALPHAS:
        ends, Tc, gc = run(alpha, iters)
        errs = [rel(e, ref) for e in ends]
        assert np.all(np.isfinite(ends[-1].view(np.float64)))
        lines.append(f"alpha {alpha[0]:>2}/{alpha[1]:<2} T{Tc} on {gc[0]}x{gc[1]}: error of the change after "
                     f"k = 1..{iters} iterations " + " ".join(f"{e:.1e}" for e in errs))
        assert errs[-1] < 0.5 * errs[0], (alpha, errs)
        if alpha[0] * 5 >= alpha[1] * 4:
            assert errs[-1] < 1e-2, (alpha, errs)
    print("\n" + "\n".join(lines))
