"""The allocation-free synthesis entry point (sht_inverse_noalloc) against
the plan-based sht_inverse, through the C ABI.

Callers that may not allocate device memory (no-allocation policies after
start-up, applications that own all device memory through their own pool)
use sht_inverse_noalloc instead of a plan.  This file is collected last on
purpose, and each test works both alone in a fresh process and after the
rest of the suite: two calls in a row must each reproduce sht_inverse within
the FP64 transform tolerance of the other GPU tests (rel-L2 1e-12), and a
request beyond the fixed scratch size must be refused before any work.
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
TOL = 1e-12


def rel(a, b):
    return (torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)).item()


@pytest.mark.parametrize("T", [31, 85])
def test_noalloc_synthesis_matches_plan_twice(T):
    nlat, nlon = syn.gaussian_grid_size(T)
    plan = ps.sht_plan_create(T, nlat, nlon, 4, "fp64")
    for call, seed in enumerate((71, 72)):
        spec = torch.tensor(syn.random_spectrum(T, (3,), seed=seed + T, nmin=0), dtype=torch.complex128,
                            device=DEV)
        ref = torch.empty((3, nlat, nlon), dtype=torch.float64, device=DEV)
        ps.sht_inverse(plan, spec, ref)
        got = torch.full((3, nlat, nlon), float("nan"), dtype=torch.float64, device=DEV)
        ps.sht_inverse_noalloc(T, nlat, nlon, spec, got)
        ps.pfsh_sync_status()
        err = rel(got, ref)
        assert err < TOL, (call, err)


def test_noalloc_refuses_requests_beyond_its_scratch():
    T = 127
    nlat, nlon = syn.gaussian_grid_size(T)
    too_many = 20                                  # 128*192*20*16 B > 4 MiB
    spec = torch.zeros((too_many, syn.ncoef(T)), dtype=torch.complex128, device=DEV)
    grid = torch.zeros((too_many, nlat, nlon), dtype=torch.float64, device=DEV)
    with pytest.raises(ps.PfshError) as e:
        ps.sht_inverse_noalloc(T, nlat, nlon, spec, grid)
    assert e.value.code == ps.PFSH_EINVAL
    spec255 = torch.zeros((1, syn.ncoef(255)), dtype=torch.complex128, device=DEV)
    grid255 = torch.zeros((1, 384, 768), dtype=torch.float64, device=DEV)
    with pytest.raises(ps.PfshError):                # T above the on-the-fly limit of 127
        ps.sht_inverse_noalloc(255, 384, 768, spec255, grid255)


def test_noalloc_synthesis_matches_oracle():
    """The allocation-free synthesis against the oracle's definition of the
    synthesis (Section 3), not only against the plan path."""
    from oracle.sht import SHT, unpack
    T = 42
    nlat, nlon = syn.gaussian_grid_size(T)
    spec = syn.random_spectrum(T, (2,), seed=73, nmin=0)
    got = torch.empty((2, nlat, nlon), dtype=torch.float64, device=DEV)
    ps.sht_inverse_noalloc(T, nlat, nlon, torch.tensor(spec, dtype=torch.complex128, device=DEV), got)
    ps.pfsh_sync_status()
    ref = SHT(T, nlat, nlon).synthesis(unpack(spec, T))
    err = float(np.linalg.norm(got.cpu().numpy() - ref) / np.linalg.norm(ref))
    assert err < TOL, err


def test_noalloc_refuses_rows_too_long_for_shared_memory():
    """An nlon whose row transform needs more than 227 KiB of shared memory is
    refused before any work is queued, although its scratch would fit."""
    spec = torch.zeros((1, syn.ncoef(1)), dtype=torch.complex128, device=DEV)
    nlon = 2 ** 13                                   # 2 * 8705 * 16 B > 227 KiB
    grid = torch.zeros((1, 4, nlon), dtype=torch.float64, device=DEV)
    with pytest.raises(ps.PfshError) as e:
        ps.sht_inverse_noalloc(1, 4, nlon, spec, grid)
    assert e.value.code == ps.PFSH_EINVAL
