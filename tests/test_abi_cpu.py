"""The C-ABI library builds for sm_103a, loads without a GPU and exports
every function that include/pfsh.h declares (no compute calls)."""
import ctypes

from _lib import declared_functions, ensure_built


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["sht_plan_create", "sht_forward", "sht_inverse", "swe_rhs", "swe_implicit_solve",
                     "sdc_sweep", "pfasst_iteration"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(ensure_built())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    ensure_built()
    import paper_1904_05988_gb300 as ps
    for n in declared_functions():
        if n in ("pfsh_last_error",):
            continue
        assert hasattr(ps, n) or n.endswith("_destroy") or n == "sht_plan_query", n


def test_argument_errors_are_reported_without_a_gpu():
    ensure_built()
    import paper_1904_05988_gb300 as ps
    import pytest
    with pytest.raises(ps.PfshError) as e:
        ps.sht_plan_create(0, 4, 8, 1, "fp64")
    assert e.value.code == ps.PFSH_EINVAL
    with pytest.raises(ps.PfshError):
        ps.sht_plan_create(31, 47, 96, 5, "fp64")   # odd nlat
    with pytest.raises(ps.PfshError):
        ps.sht_plan_create(31, 48, 62, 5, "fp64")   # nlon <= 2(T+1)


def test_noalloc_binding_rejects_a_ragged_spectrum_before_the_library():
    """A spectrum whose size is not a whole number of ncoef(T) fields is an
    error in the binding (it would otherwise be truncated silently)."""
    ensure_built()
    import paper_1904_05988_gb300 as ps
    import pytest
    import torch
    spec = torch.zeros(ps.ncoef(31) + 1, dtype=torch.complex128)
    grid = torch.zeros((1, 48, 96), dtype=torch.float64)
    with pytest.raises(ValueError):
        ps.sht_inverse_noalloc(31, 48, 96, spec, grid)


def test_failure_detection_arguments_checked_without_a_gpu():
    ensure_built()
    import paper_1904_05988_gb300 as ps
    import pytest
    with pytest.raises(ps.PfshError) as e:
        ps.pfsh_selftest_wait(0, stream=0)
    assert e.value.code == ps.PFSH_EINVAL
    ps.pfsh_set_check_finite(False)
