"""Precision sweep of the transform pair at T511 on the 768 x 1536 Gaussian
grid: 3 fields x 5 nodes x 16 slices = 240 seeded spectra with per-degree
power ~ n^-3 (unit area-rms) through every form of the build, each form's
rel-L2 error against the FP64 oracle reported and bounded.

The GPU transforms all 240 fields in one call; the oracle computes two
sampled fields in full (its table at T511 takes seconds), and the round trip
analysis(synthesis(x)) = x, which holds at any size, is checked on all 240:

  synthesis  GPU inverse of the sampled spectra vs the oracle's grids
  analysis   GPU forward of the oracle's grids (rounded to the plan's grid
             type), tiled to 16 columns so that the form's contraction (not
             the batch-1/2 CUDA-core kernels) runs, vs the sampled spectra
  pair       GPU forward(GPU inverse(x)) vs x over all 240 fields

Bounds (measured on GB300 in brackets) follow the operand rounding of each
form: bf16 keeps 8 mantissa bits, fp16 11, the hi/lo split of 3xBF16 about
16, the three-part split of 6xBF16 and fp32 24.  6xBF16 stays about 3.5x
above the fp32 CUDA-core form: its operands keep fp32's 24 bits, but the
tensor cores' fp32 accumulation over K = 128..384 terms loses more than the
CUDA cores' FMA chains.
"""
import numpy as np
import pytest

import synthetic as syn
from oracle.sht import SHT, unpack, pack
from _lib import ensure_built

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
ensure_built()
import paper_1904_05988_gb300 as ps  # noqa: E402

DEV = torch.device("cuda:0")
T = 511
NFIELDS = 3 * 5 * 16
SAMPLE = (0, 137)
BOUNDS = {  # synthesis, analysis, pair
    "fp64": (1e-13, 1e-12, 1e-12),      # (1.2e-15, 2.1e-14, 1.9e-14)
    "fp32": (1e-6, 1e-6, 1e-6),         # (4.2e-7, 4.7e-7, 4.6e-7)
    "bf16": (5e-3, 5e-3, 6e-3),         # (2.1e-3, 1.9e-3, 2.8e-3)
    "fp16": (6e-4, 6e-4, 8e-4),         # (2.3e-4, 2.6e-4, 3.7e-4)
    "bf16x3": (1e-5, 1e-5, 1.5e-5),     # (4.1e-6, 3.7e-6, 5.7e-6)
    "bf16x6": (2.5e-6, 2.5e-6, 5e-6),    # (1.7e-6, 1.6e-6, 3.1e-6)
}
FORMS = [f for f in BOUNDS if f in ps.available_precisions()]


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def sweep_data():
    nlat, nlon = syn.gaussian_grid_size(T)
    assert (nlat, nlon) == (768, 1536)
    spec = syn.random_spectrum(T, (NFIELDS,), seed=511)
    o = SHT(T, nlat, nlon, L=T + 1)
    grids = o.synthesis(unpack(spec[list(SAMPLE)], T))
    return spec, grids


@pytest.mark.parametrize("form", FORMS)
def test_transform_pair_T511_240_fields(form, sweep_data):
    spec, grids = sweep_data
    nlat, nlon = syn.gaussian_grid_size(T)
    gdtype = torch.float64 if form == "fp64" else torch.float32
    plan = ps.sht_plan_create(T, nlat, nlon, NFIELDS, form)
    d_spec = torch.tensor(spec, dtype=torch.complex128, device=DEV)
    grid = torch.empty((NFIELDS, nlat, nlon), dtype=gdtype, device=DEV)
    back = torch.empty_like(d_spec)
    ps.sht_inverse(plan, d_spec, grid)
    ps.sht_forward(plan, grid, back)
    reps = 8
    g_o = torch.tensor(np.tile(grids, (reps, 1, 1)), dtype=gdtype, device=DEV)
    b_o = torch.empty((reps * len(SAMPLE), syn.ncoef(T)), dtype=torch.complex128, device=DEV)
    ps.sht_forward(plan, g_o, b_o)
    ps.pfsh_sync_status()
    e_syn = rel(grid[list(SAMPLE)].cpu().numpy().astype(np.float64), grids)
    e_ana = rel(b_o.cpu().numpy(), np.tile(spec[list(SAMPLE)], (reps, 1)))
    e_pair = rel(back.cpu().numpy(), spec)
    print(f"\nT511 x {NFIELDS} fields, {form}: synthesis {e_syn:.3e}  analysis {e_ana:.3e}  pair {e_pair:.3e}")
    bs, ba, bp = BOUNDS[form]
    assert e_syn < bs and e_ana < ba and e_pair < bp, (e_syn, e_ana, e_pair)
    plan.close()


def test_fp16_plan_refuses_the_rhs():
    """The FP16 form serves transforms only: the flux products of the
    right-hand side leave the fp16 range, so a context on an FP16 plan is
    refused."""
    if "fp16" not in ps.available_precisions():
        pytest.skip("fp16 not built")
    plan = ps.sht_plan_create(31, 48, 96, 5, "fp16")
    with pytest.raises(ps.PfshError):
        ps.swe_ctx_create(plan, syn.EARTH_RADIUS, syn.OMEGA, syn.NU, 1e5)
    plan.close()
