"""Parity of the mixed-precision CUDA paths with the FP64 oracle.

Every mixed form keeps spectral data, the Legendre recurrence, Gaussian
nodes/weights and all SDC/FAS bookkeeping in FP64; the Legendre contractions
run in the form's precision and the FFT/grid stage in FP32.

Bounds (rel-L2 against the oracle):

* transform pair: the form's measured bound (fp32 1e-6, bf16 5e-3, 3xBF16
  1e-5; largest measured on GB300 over T63/T170/T255: 3.5e-7, 3.0e-3, 5.5e-6),
  a few units of the operand rounding u of the form; the three-part split
  6xBF16 2.5e-6 (measured 6.4e-7, 1.2e-6, 1.6e-6 at T63, T170, T255: its
  operands keep 24 bits, the tensor cores' fp32 accumulation limits it);
* one RHS F_E: the rounding laws of tests/_lib.py, one set of constants for
  every form and truncation -- the error at degree n at most 24 u (n+1) |F_E|
  (the spectral derivatives amplify the analysed fluxes' rounding by ~n),
  the whole field within 48 u (T+1) and the band n <= T/4 within 8 u (T/4+1);
* PFASST end values: the form's measured bound (fp32 and 6xBF16 1e-8, bf16
  2e-4, 3xBF16 5e-7); their change from the initial value: the low-band law of F_E
  (8 u (T/4+1)), since the change integrates the tendencies.
"""
import numpy as np
import pytest

import synthetic as syn
from oracle.sht import SHT, pack, unpack
from oracle.swe import SWEParams, rhs
from oracle.sdc import SDCLevel
from oracle.pfasst import PFASST
from _lib import C_DEGREE, change_bound, ensure_built, low_band_rel, per_degree_excess, rhs_bounds

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
ensure_built()
import paper_1904_05988_gb300 as ps  # noqa: E402

DEV = torch.device("cuda:0")
A, OM, G = syn.EARTH_RADIUS, syn.OMEGA, syn.GRAVITY
PHIBAR = G * syn.MEAN_DEPTH
BOUNDS = {  # transform pair, PFASST end values
    "fp32": (1e-6, 1e-8),
    "bf16": (5e-3, 2e-4),
    "bf16x3": (1e-5, 5e-7),
    "bf16x6": (2.5e-6, 1e-8),
}
FORMS = [f for f in BOUNDS if f in ps.available_precisions()]


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


def cuda(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.complex128, device=DEV)


def state_of(T, seed, batch=1):
    s = syn.random_spectrum(T, (batch, 3), seed=seed, rms=1e-5)
    s[:, 0] *= 1e3
    return s + syn.zonal_jet(T)[None]


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("T", [63, 170, 255])
def test_transform_pair(form, T):
    """40 fields in passes of 16, 16 and 8: the first two take the form's
    contraction (tensor cores for bf16/3xbf16), the ragged last one the
    small-batch CUDA-core kernels; the error is over all 40."""
    nlat, nlon = syn.gaussian_grid_size(T)
    plan = ps.sht_plan_create(T, nlat, nlon, 16, form)
    nf = 40
    spec = syn.random_spectrum(T, (nf,), seed=30 + T, nmin=1)
    grid = torch.empty((nf, nlat, nlon), dtype=torch.float32, device=DEV)
    ps.sht_inverse(plan, cuda(spec), grid)
    back = torch.empty((nf, syn.ncoef(T)), dtype=torch.complex128, device=DEV)
    ps.sht_forward(plan, grid, back)
    ps.pfsh_sync_status()
    o = SHT(T, nlat, nlon, L=T + 1)
    ref_grid = o.synthesis(unpack(spec, T))
    e_inv = rel(grid.cpu().numpy().astype(np.float64), ref_grid)
    e_pair = rel(back.cpu().numpy(), spec)
    print(f"\n[{form} T{T}] inverse {e_inv:.2e}  pair {e_pair:.2e}")
    assert e_inv < BOUNDS[form][0] and e_pair < BOUNDS[form][0]


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("T,B", [(63, 3), (170, 3), (255, 3), (127, 1)])
def test_swe_rhs(form, T, B):
    """B = 3 states (12 synthesis / 15 analysis columns) takes the form's
    contraction; B = 1 the small-batch path of the serial coarse chain."""
    nlat, nlon = syn.gaussian_grid_size(T)
    plan = ps.sht_plan_create(T, nlat, nlon, 5 * B, form)
    ctx = ps.swe_ctx_create(plan, A, OM, syn.NU, PHIBAR)
    st = state_of(T, 200 + T, B)
    fE = torch.empty((B, 3, syn.ncoef(T)), dtype=torch.complex128, device=DEV)
    fI = torch.empty_like(fE)
    ps.swe_rhs(ctx, cuda(st), fE, fI)
    ps.pfsh_sync_status()
    p = SWEParams(a=A, omega=OM, g=G, nu=syn.NU, phibar=PHIBAR)
    FE, FI = rhs(unpack(st[B - 1], T), SHT(T, nlat, nlon), p)
    got = fE.cpu().numpy()[B - 1]
    _, b_whole, b_low = rhs_bounds(form, T)
    for f in range(3):
        ref = pack(FE[f], T)
        e_whole, e_low = rel(got[f], ref), low_band_rel(got[f], ref, T)
        exc = per_degree_excess(got[f], ref, T, form)
        print(f"\n[{form} T{T}] F_E field {f}: rel-L2 {e_whole:.2e} (bound {b_whole:.1e}), n <= T/4 {e_low:.2e} "
              f"(bound {b_low:.1e}), max_n e_n/(u (n+1) |F|) {exc:.2f}")
        assert e_whole < b_whole and e_low < b_low
        assert exc <= C_DEGREE
    assert rel(fI.cpu().numpy()[B - 1], pack(FI, T)) < 1e-13    # F_I stays FP64


@pytest.mark.parametrize("form", FORMS)
def test_pfasst_two_iterations(form):
    Tf, Tc, nts, dt = 63, 31, 4, 600.0
    gf, gc = syn.gaussian_grid_size(Tf), syn.gaussian_grid_size(Tc)
    st0 = state_of(Tf, 41)[0]
    pf = ps.pfasst_create(nts, 5, 3, Tf, *gf, Tc, *gc, dt, A, OM, syn.NU, PHIBAR, form)
    ps.pfasst_set_initial(pf, cuda(st0))
    ps.pfasst_predict(pf)
    ps.pfasst_iteration(pf, False)
    ps.pfasst_iteration(pf, True)
    ps.pfsh_sync_status()
    p = SWEParams(a=A, omega=OM, g=G, nu=syn.NU, phibar=PHIBAR)
    o = PFASST(SDCLevel(Tf, *gf, 5, dt, p), SDCLevel(Tc, *gc, 3, dt, p), nts)
    ref = o.run(unpack(st0, Tf), 2)
    out = torch.empty((3, syn.ncoef(Tf)), dtype=torch.complex128, device=DEV)
    errs = []
    for n in range(nts):
        ps.pfasst_get(pf, 0, n, 4, out)
        errs.append(rel(out.cpu().numpy(), pack(ref[n], Tf)))
    # the perturbation (state minus initial value) is matched too, not just the jet
    ps.pfasst_get(pf, 0, nts - 1, 4, out)
    d_got = out.cpu().numpy() - st0
    d_ref = pack(ref[nts - 1], Tf) - st0
    e_inc = rel(d_got, d_ref)
    print(f"\n[{form}] PFASST end values rel-L2 max {max(errs):.2e}, increment {e_inc:.2e}")
    assert max(errs) < BOUNDS[form][1]
    assert e_inc < change_bound(form, Tf)
