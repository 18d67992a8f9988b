"""Failure detection on the GPU without faulting it.

* Non-finite values: with pfsh_set_check_finite on, a NaN planted on the host
  in an input state makes swe_rhs / the PFASST calls record ST_NUMERIC, and
  pfsh_sync_status raises PFSH_ENUMERIC; the status word is then clear and
  the next call runs normally.  With the check off the NaN passes silently
  (the check is what detects it).
* Bounded waits: pfsh_selftest_wait runs one CTA that waits on an mbarrier
  nothing arms, with a short poll limit: the wait gives up, the CTA frees its
  tensor memory, pfsh_sync_status raises PFSH_ETIMEOUT, and the context stays
  usable for the next computation.
No test traps, faults or hangs the GPU: every wait is bounded.
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
A, OM, PHIBAR = syn.EARTH_RADIUS, syn.OMEGA, syn.GRAVITY * syn.MEAN_DEPTH


def state(T, seed):
    s = syn.zonal_jet(T) + syn.random_spectrum(T, (3,), seed=seed, rms=1e-5) * np.array([1e3, 1, 1])[:, None]
    return torch.tensor(s[None], dtype=torch.complex128, device=DEV)


@pytest.fixture
def check_on():
    ps.pfsh_set_check_finite(True)
    yield
    ps.pfsh_set_check_finite(False)


@pytest.mark.parametrize("form", ["fp64", "bf16x3"])
def test_nan_in_rhs_input_is_reported(form, check_on):
    if form not in ps.available_precisions():
        pytest.skip(f"{form} not built")
    T = 31
    plan = ps.sht_plan_create(T, *syn.gaussian_grid_size(T), 10, form)
    ctx = ps.swe_ctx_create(plan, A, OM, syn.NU, PHIBAR)
    st = state(T, 81)
    fE, fI = torch.empty_like(st), torch.empty_like(st)
    ps.swe_rhs(ctx, st, fE, fI)
    ps.pfsh_sync_status()                                  # finite input: no report
    bad = st.clone()
    bad[0, 1, 7] = complex(float("nan"), 0.0)              # planted on the host side of the ABI
    ps.swe_rhs(ctx, bad, fE, fI)
    with pytest.raises(ps.PfshError) as e:
        ps.pfsh_sync_status()
    assert e.value.code == ps.PFSH_ENUMERIC
    ps.swe_rhs(ctx, st, fE, fI)                            # status cleared, context usable
    ps.pfsh_sync_status()
    assert torch.isfinite(torch.view_as_real(fE)).all()


def test_nan_passes_silently_without_the_check():
    T = 21
    plan = ps.sht_plan_create(T, *syn.gaussian_grid_size(T), 10, "fp64")
    ctx = ps.swe_ctx_create(plan, A, OM, syn.NU, PHIBAR)
    bad = state(T, 82)
    bad[0, 0, 3] = complex(float("inf"), 0.0)
    fE, fI = torch.empty_like(bad), torch.empty_like(bad)
    ps.swe_rhs(ctx, bad, fE, fI)
    ps.pfsh_sync_status()
    assert not torch.isfinite(torch.view_as_real(fE)).all()


def test_nan_in_pfasst_initial_value_is_reported(check_on):
    form = "bf16x3" if "bf16x3" in ps.available_precisions() else "fp64"
    Tf, Tc = 31, 15
    gf, gc = syn.gaussian_grid_size(Tf), syn.gaussian_grid_size(Tc)
    pf = ps.pfasst_create(4, 5, 3, Tf, *gf, Tc, *gc, 600.0, A, OM, syn.NU, PHIBAR, form)
    st = state(Tf, 83)[0]
    bad = st.clone()
    bad[2, 40] = complex(0.0, float("nan"))
    ps.pfasst_set_initial(pf, bad)
    ps.pfasst_predict(pf)
    ps.pfasst_iterations(pf, 2, True)
    with pytest.raises(ps.PfshError) as e:
        ps.pfsh_sync_status()
    assert e.value.code == ps.PFSH_ENUMERIC
    ps.pfasst_set_initial(pf, st)                          # a finite run afterwards is clean
    ps.pfasst_predict(pf)
    ps.pfasst_iterations(pf, 2, True)
    ps.pfsh_sync_status()
    pf.close()


def test_bounded_wait_gives_up_and_leaves_the_context_usable():
    ps.pfsh_selftest_wait(4096)
    with pytest.raises(ps.PfshError) as e:
        ps.pfsh_sync_status()
    assert e.value.code == ps.PFSH_ETIMEOUT
    T = 21
    plan = ps.sht_plan_create(T, *syn.gaussian_grid_size(T), 10, "fp64")
    ctx = ps.swe_ctx_create(plan, A, OM, syn.NU, PHIBAR)
    st = state(T, 84)
    fE = torch.empty_like(st)
    ps.swe_rhs(ctx, st, fE, None)
    ps.pfsh_sync_status()
    assert torch.isfinite(torch.view_as_real(fE)).all()
