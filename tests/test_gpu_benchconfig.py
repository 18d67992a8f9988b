"""PFASST at exactly the benchmark's set-up against the oracle.

T255 on 384 x 768 with 5 Gauss-Lobatto nodes / T127 on 192 x 384 with 3,
32 time slices, dt = 120 s, the balanced jet plus the 120 m Gaussian height
bump at the seed-2 location: the predictor, then a block of two iterations of
Algorithm 1 through ``pfasst_iterations`` (a full iteration and a last one of
Step A only) -- the call the benchmark times, in the launch configuration it
times: 3xBF16 with the slices in 2 groups of 16 (16-state tensor-core batches,
the chain of one group overlapping the fine sweeps of the other, the
wavefront across iterations), and FP64 in one group of 32 (the FP64 GPU path
the benchmark reports beside it).  Every slice's fine end value is compared
with the oracle's, element by element over the whole state.

The oracle runs its slice-independent steps in spawned worker processes on
every host core (``oracle.pool``); the whole reference takes about a minute
on 16 cores.  The oracle projects the bump with its own analysis and the GPU
receives that state.

Bounds: FP64 1e-11 on every slice's end value (rounding of ~1e5 FP64
operations per coefficient along the chain of 32 slices).  3xBF16: the
end-value bound is the one of the 4-slice full-size test (5e-8); the change
of the state from its initial value integrates the tendencies, so its
relative error obeys the low-band rounding law of F_E, 8 u (T/4 + 1) with
u = 2^-17 (tests/_lib.py).
"""
import math
import os

import numpy as np
import pytest

import synthetic as syn
from oracle.pfasst import PFASST
from oracle.pool import SlicePool
from oracle.sdc import SDCLevel
from oracle.sht import SHT, pack, unpack
from oracle.swe import SWEParams
from _lib import change_bound, ensure_built

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
ensure_built()
import paper_1904_05988_gb300 as ps  # noqa: E402

DEV = torch.device("cuda:0")
TF, TC, NTS, NF, NC, DT = 255, 127, 32, 5, 3, 120.0
CASES = {  # form: (slice groups, end-value bound, change bound)
    "fp64": (1, 1e-11, 1e-8),
    "bf16x3": (2, 5e-8, change_bound("bf16x3", TF)),
}


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.fixture(scope="module")
def reference():
    gf, gc = syn.gaussian_grid_size(TF), syn.gaussian_grid_size(TC)
    sht = SHT(TF, *gf, L=TF + 1)
    lam = 2.0 * math.pi * np.arange(gf[1]) / gf[1]
    lam_c, phi_c = syn.bump_center(2)
    bump = syn.GRAVITY * syn.gaussian_bump(sht.mu, lam, amplitude=120.0, width=1.0 / 15.0, lam_c=lam_c, phi_c=phi_c)
    st = unpack(syn.zonal_jet(TF), TF)
    st[0] += sht.analysis(bump, TF + 1)
    phibar = st[0, 0, 0].real / math.sqrt(2.0)
    p = SWEParams(a=syn.EARTH_RADIUS, omega=syn.OMEGA, g=syn.GRAVITY, nu=syn.NU, phibar=phibar)
    f, c = SDCLevel(TF, *gf, NF, DT, p), SDCLevel(TC, *gc, NC, DT, p)
    with SlicePool({"f": f.args, "c": c.args}, workers=min(NTS, os.cpu_count() or 1)) as pool:
        ends = PFASST(f, c, NTS, pool=pool).run(st, 2)
    return pack(st, TF), phibar, np.stack([pack(ends[n], TF) for n in range(NTS)])


@pytest.mark.parametrize("form", list(CASES))
def test_pfasst_bench_configuration_matches_oracle(form, reference):
    if form not in ps.available_precisions():
        pytest.skip(f"{form} not built")
    groups, b_end, b_change = CASES[form]
    st0, phibar, ends = reference
    gf, gc = syn.gaussian_grid_size(TF), syn.gaussian_grid_size(TC)
    pf = ps.pfasst_create(NTS, NF, NC, TF, *gf, TC, *gc, DT, syn.EARTH_RADIUS, syn.OMEGA, syn.NU, phibar, form,
                          slice_groups=groups)
    ps.pfasst_set_initial(pf, torch.tensor(st0, dtype=torch.complex128, device=DEV))
    ps.pfasst_predict(pf)
    ps.pfasst_iterations(pf, 2, True)
    out = torch.empty((NTS, 3, syn.ncoef(TF)), dtype=torch.complex128, device=DEV)
    for n in range(NTS):
        ps.pfasst_get(pf, 0, n, NF - 1, out[n])
    ps.pfsh_sync_status()
    got = out.cpu().numpy()
    pf.close()
    errs = [rel(got[n], ends[n]) for n in range(NTS)]
    changes = [rel(got[n] - st0, ends[n] - st0) for n in range(NTS)]
    assert np.all(np.isfinite(got.view(np.float64)))
    print(f"\nT255/T127 x {NTS} slices, {form}, {groups} group(s): end values max {max(errs):.3e} "
          f"(slice {int(np.argmax(errs))}), change max {max(changes):.3e}")
    assert max(errs) < b_end, errs
    assert max(changes) < b_change, changes
