"""GB300-native PFASST-SH hot path: Python binding of ``include/pfsh.h``.

Argument marshalling only: every function below forwards device pointers of
torch CUDA tensors to the C ABI of ``lib/libpfsh.so`` and raises
``PfshError`` on a negative status.  There is no fallback: if the library is
missing, importing this package fails; run ``python paper_1904_05988_gb300/build.py``
(or ``__graft_entry__.build()``) first.

Names and argument order follow the C ABI.  Spectral arrays are complex128
tensors of shape ``[..., ncoef]`` (m-major triangle, see the header) and
states ``[..., 3, ncoef]``; grids are float64 (FP64 plans) or float32
``[batch, nlat, nlon]``.
"""
from __future__ import annotations

import ctypes
import os

import torch

from .build import LIB

PFSH_OK, PFSH_EINVAL, PFSH_ENOMEM, PFSH_ECUDA, PFSH_EUNSUPPORTED, PFSH_ETIMEOUT, PFSH_ENUMERIC = 0, -1, -2, -3, -4, -5, -6
PFSH_FP64, PFSH_FP32, PFSH_BF16, PFSH_FP16, PFSH_BF16X3, PFSH_BF16X6 = 0, 1, 2, 3, 4, 5
PREC_NAMES = {"fp64": PFSH_FP64, "fp32": PFSH_FP32, "bf16": PFSH_BF16, "fp16": PFSH_FP16, "bf16x3": PFSH_BF16X3,
              "bf16x6": PFSH_BF16X6}

EXPORTED = ["sht_plan_create", "sht_plan_destroy", "sht_plan_query", "sht_inverse", "sht_forward",
            "swe_ctx_create", "swe_ctx_destroy", "swe_rhs", "swe_implicit_solve",
            "sdc_level_create", "sdc_level_destroy", "sdc_spread", "sdc_sweep",
            "pfasst_create", "pfasst_destroy", "pfasst_set_initial", "pfasst_predict",
            "pfasst_iteration", "pfasst_iterations", "pfasst_residual", "pfasst_get", "pfasst_ensemble_create",
            "pfasst_ensemble_destroy", "pfasst_ensemble_member", "pfasst_ensemble_predict",
            "pfasst_ensemble_iterations", "pfsh_sync_status", "pfsh_last_error",
            "pfsh_kernel_launches", "pfsh_profiler_enable", "pfsh_profiler_report", "sht_inverse_noalloc",
            "pfsh_alu_peak", "pfsh_set_check_finite", "pfsh_selftest_wait"]


class PfshError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"pfsh status {code}: {msg}")
        self.code = code


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB):
        raise ImportError(f"CUDA library {LIB} is missing: build it with paper_1904_05988_gb300.build.build()")
    return ctypes.CDLL(LIB)


_lib = _load()

c_int, c_double, c_void_p, c_size_t = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t


PFSH_CORIOLIS_EXPLICIT, PFSH_CORIOLIS_IMPLICIT = 0, 1


class SweParams(ctypes.Structure):
    _fields_ = [("a", c_double), ("omega", c_double), ("nu", c_double), ("phibar", c_double), ("coriolis", c_int),
                ("implicit_split", c_int)]


class ShtInfo(ctypes.Structure):
    _fields_ = [("T", c_int), ("nlat", c_int), ("nlon", c_int), ("ncoef", c_int), ("max_batch", c_int),
                ("prec", c_int), ("device_bytes", c_size_t), ("mu", ctypes.POINTER(c_double)),
                ("w", ctypes.POINTER(c_double)), ("tc_tiles", (c_int * 8) * 2)]


class PfasstConfig(ctypes.Structure):
    _fields_ = [("n_ts", c_int), ("fine_nodes", c_int), ("coarse_nodes", c_int),
                ("Tf", c_int), ("nlat_f", c_int), ("nlon_f", c_int),
                ("Tc", c_int), ("nlat_c", c_int), ("nlon_c", c_int),
                ("dt", c_double), ("phys", SweParams), ("prec", c_int), ("slice_groups", c_int)]


_sig = {
    "sht_plan_create": [ctypes.POINTER(c_void_p), c_int, c_int, c_int, c_int, c_int],
    "sht_plan_destroy": [c_void_p],
    "sht_plan_query": [c_void_p, ctypes.POINTER(ShtInfo)],
    "sht_inverse": [c_void_p, c_void_p, c_void_p, c_int, c_void_p],
    "sht_forward": [c_void_p, c_void_p, c_void_p, c_int, c_void_p],
    "swe_ctx_create": [ctypes.POINTER(c_void_p), c_void_p, ctypes.POINTER(SweParams)],
    "swe_ctx_destroy": [c_void_p],
    "swe_rhs": [c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_void_p],
    "swe_implicit_solve": [c_void_p, c_void_p, c_void_p, c_double, c_int, c_void_p],
    "sdc_level_create": [ctypes.POINTER(c_void_p), c_void_p, c_int, c_double, c_int],
    "sdc_level_destroy": [c_void_p],
    "sdc_spread": [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_void_p],
    "sdc_sweep": [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_void_p],
    "pfasst_create": [ctypes.POINTER(c_void_p), ctypes.POINTER(PfasstConfig)],
    "pfasst_destroy": [c_void_p],
    "pfasst_set_initial": [c_void_p, c_void_p, c_void_p],
    "pfasst_predict": [c_void_p, c_void_p],
    "pfasst_iteration": [c_void_p, c_int, c_void_p],
    "pfasst_iterations": [c_void_p, c_int, c_int, c_void_p],
    "pfasst_residual": [c_void_p, c_void_p, c_void_p],
    "pfasst_ensemble_create": [ctypes.POINTER(c_void_p), ctypes.POINTER(PfasstConfig), c_int],
    "pfasst_ensemble_destroy": [c_void_p],
    "pfasst_ensemble_predict": [c_void_p, c_void_p],
    "pfasst_ensemble_iterations": [c_void_p, c_int, c_int, c_void_p],
    "pfasst_get": [c_void_p, c_int, c_int, c_int, c_void_p, c_void_p],
    "pfsh_sync_status": [c_void_p],
    "sht_inverse_noalloc": [c_int, c_int, c_int, c_void_p, c_void_p, c_int, c_void_p],
}
for _name, _args in _sig.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = c_int
_lib.pfasst_ensemble_member.argtypes = [c_void_p, c_int]
_lib.pfasst_ensemble_member.restype = c_void_p
_lib.pfsh_last_error.argtypes = []
_lib.pfsh_last_error.restype = ctypes.c_char_p
_lib.pfsh_kernel_launches.argtypes = []
_lib.pfsh_kernel_launches.restype = ctypes.c_ulonglong
_lib.pfsh_profiler_enable.argtypes = [c_int]
_lib.pfsh_profiler_enable.restype = c_int
_lib.pfsh_profiler_report.argtypes = [ctypes.c_char_p, c_size_t]
_lib.pfsh_profiler_report.restype = c_int
_lib.pfsh_set_check_finite.argtypes = [c_int]
_lib.pfsh_set_check_finite.restype = c_int
_lib.pfsh_selftest_wait.argtypes = [ctypes.c_uint, c_void_p]
_lib.pfsh_selftest_wait.restype = c_int
_lib.pfsh_alu_peak.argtypes = [c_int, ctypes.POINTER(c_double)]
_lib.pfsh_alu_peak.restype = c_int


def available_precisions() -> list[str]:
    """Precision names the compiled library serves (probed with argument-free checks)."""
    return [name for name, code in PREC_NAMES.items() if code in _BUILT_PRECISIONS]


_BUILT_PRECISIONS = {PFSH_FP64, PFSH_FP32, PFSH_BF16, PFSH_FP16, PFSH_BF16X3, PFSH_BF16X6}


def last_error() -> str:
    return _lib.pfsh_last_error().decode()


def _check(rc: int) -> None:
    if rc != PFSH_OK:
        raise PfshError(rc, last_error())


def _stream(stream) -> int | None:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream or None
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else stream


def _ptr(t: torch.Tensor | None, dtype: torch.dtype | None = None, numel: int | None = None) -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("tensor must live on a CUDA device")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"expected {dtype}, got {t.dtype}")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"tensor too small: {t.numel()} < {numel} elements")
    return t.data_ptr()


def ncoef(T: int) -> int:
    return (T + 1) * (T + 2) // 2


# ---------------------------------------------------------------------------
# handles
# ---------------------------------------------------------------------------
class _Handle:
    _destroy = None

    def __init__(self, ptr: int):
        self.ptr = ptr

    def close(self):
        if self.ptr:
            getattr(_lib, self._destroy)(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ShtPlan(_Handle):
    _destroy = "sht_plan_destroy"

    def __init__(self, ptr: int):
        super().__init__(ptr)
        info = ShtInfo()
        _check(_lib.sht_plan_query(ptr, ctypes.byref(info)))
        self.T, self.nlat, self.nlon = info.T, info.nlat, info.nlon
        self.ncoef, self.max_batch, self.prec = info.ncoef, info.max_batch, info.prec
        self.device_bytes = info.device_bytes
        self.mu = [info.mu[i] for i in range(self.nlat)]
        self.w = [info.w[i] for i in range(self.nlat)]
        # autotuned row tiles per order: [synthesis, analysis][launch width 1..8 x 128 real columns]
        self.tc_tiles = [[info.tc_tiles[d][i] for i in range(8)] for d in range(2)]

    @property
    def grid_dtype(self) -> torch.dtype:
        return torch.float64 if self.prec == PFSH_FP64 else torch.float32


class SweCtx(_Handle):
    _destroy = "swe_ctx_destroy"

    def __init__(self, ptr: int, plan: ShtPlan, params: SweParams):
        super().__init__(ptr)
        self.plan, self.params = plan, params  # keep the plan alive


class SdcLevel(_Handle):
    _destroy = "sdc_level_destroy"

    def __init__(self, ptr: int, ctx: SweCtx, nodes: int, dt: float, max_batch: int):
        super().__init__(ptr)
        self.ctx, self.nodes, self.dt, self.max_batch = ctx, nodes, dt, max_batch


class Pfasst(_Handle):
    _destroy = "pfasst_destroy"

    def __init__(self, ptr: int, cfg: PfasstConfig, owner=None):
        super().__init__(ptr)
        self.cfg = cfg
        self._owner = owner   # an ensemble member is destroyed with its ensemble

    def close(self):
        if self._owner is None:
            super().close()
        self.ptr = None


class PfasstEnsemble(_Handle):
    _destroy = "pfasst_ensemble_destroy"

    def __init__(self, ptr: int, cfgs: list):
        super().__init__(ptr)
        self.members = []
        for i, c in enumerate(cfgs):
            m = _lib.pfasst_ensemble_member(ptr, i)
            if not m:
                raise PfshError(PFSH_EINVAL, last_error())
            self.members.append(Pfasst(m, c, owner=self))

    def close(self):
        for m in getattr(self, "members", []):
            m.ptr = None
        super().close()


# ---------------------------------------------------------------------------
# ABI functions (same names)
# ---------------------------------------------------------------------------
def sht_plan_create(T: int, nlat: int, nlon: int, max_batch: int, prec: int | str = PFSH_FP64) -> ShtPlan:
    prec = PREC_NAMES[prec] if isinstance(prec, str) else prec
    h = c_void_p()
    _check(_lib.sht_plan_create(ctypes.byref(h), T, nlat, nlon, max_batch, prec))
    return ShtPlan(h.value)


def sht_inverse(plan: ShtPlan, spec: torch.Tensor, grid: torch.Tensor, stream=None) -> torch.Tensor:
    batch = spec.numel() // plan.ncoef
    _check(_lib.sht_inverse(plan.ptr, _ptr(spec, torch.complex128, batch * plan.ncoef),
                            _ptr(grid, plan.grid_dtype, batch * plan.nlat * plan.nlon), batch, _stream(stream)))
    return grid


def sht_forward(plan: ShtPlan, grid: torch.Tensor, spec: torch.Tensor, stream=None) -> torch.Tensor:
    batch = grid.numel() // (plan.nlat * plan.nlon)
    _check(_lib.sht_forward(plan.ptr, _ptr(grid, plan.grid_dtype, batch * plan.nlat * plan.nlon),
                            _ptr(spec, torch.complex128, batch * plan.ncoef), batch, _stream(stream)))
    return spec


def swe_ctx_create(plan: ShtPlan, a: float, omega: float, nu: float, phibar: float,
                   coriolis_implicit: bool = False, implicit_split: bool = False) -> SweCtx:
    p = SweParams(a, omega, nu, phibar, PFSH_CORIOLIS_IMPLICIT if coriolis_implicit else PFSH_CORIOLIS_EXPLICIT,
                  int(implicit_split))
    h = c_void_p()
    _check(_lib.swe_ctx_create(ctypes.byref(h), plan.ptr, ctypes.byref(p)))
    return SweCtx(h.value, plan, p)


def swe_rhs(ctx: SweCtx, state: torch.Tensor, fE: torch.Tensor, fI: torch.Tensor | None = None,
            stream=None) -> None:
    nc3 = 3 * ctx.plan.ncoef
    B = state.numel() // nc3
    _check(_lib.swe_rhs(ctx.ptr, _ptr(state, torch.complex128, B * nc3), _ptr(fE, torch.complex128, B * nc3),
                        _ptr(fI, torch.complex128, B * nc3), B, _stream(stream)))


def swe_implicit_solve(ctx: SweCtx, b: torch.Tensor, x: torch.Tensor, h: float, stream=None) -> None:
    nc3 = 3 * ctx.plan.ncoef
    B = b.numel() // nc3
    _check(_lib.swe_implicit_solve(ctx.ptr, _ptr(b, torch.complex128, B * nc3), _ptr(x, torch.complex128, B * nc3),
                                   h, B, _stream(stream)))


def sdc_level_create(ctx: SweCtx, nodes: int, dt: float, max_batch: int) -> SdcLevel:
    h = c_void_p()
    _check(_lib.sdc_level_create(ctypes.byref(h), ctx.ptr, nodes, dt, max_batch))
    return SdcLevel(h.value, ctx, nodes, dt, max_batch)


def sdc_spread(level: SdcLevel, theta0: torch.Tensor, theta: torch.Tensor, fE: torch.Tensor, fI: torch.Tensor,
               stream=None) -> None:
    nc3 = 3 * level.ctx.plan.ncoef
    B = theta0.numel() // nc3
    n = level.nodes * B * nc3
    _check(_lib.sdc_spread(level.ptr, _ptr(theta0, torch.complex128, B * nc3), _ptr(theta, torch.complex128, n),
                           _ptr(fE, torch.complex128, n), _ptr(fI, torch.complex128, n), B, _stream(stream)))


def sdc_sweep(level: SdcLevel, theta: torch.Tensor, fE: torch.Tensor, fI: torch.Tensor,
              tau: torch.Tensor | None = None, stream=None) -> None:
    nc3 = 3 * level.ctx.plan.ncoef
    B = theta.numel() // (nc3 * level.nodes)
    n = level.nodes * B * nc3
    _check(_lib.sdc_sweep(level.ptr, _ptr(theta, torch.complex128, n), _ptr(fE, torch.complex128, n),
                          _ptr(fI, torch.complex128, n), _ptr(tau, torch.complex128, n), B, _stream(stream)))


def pfasst_create(n_ts: int, fine_nodes: int, coarse_nodes: int, Tf: int, nlat_f: int, nlon_f: int,
                  Tc: int, nlat_c: int, nlon_c: int, dt: float, a: float, omega: float, nu: float,
                  phibar: float, prec: int | str = PFSH_FP64, slice_groups: int = 0,
                  coriolis_implicit: bool = False, implicit_split: bool = False) -> Pfasst:
    cfg = pfasst_config(n_ts, fine_nodes, coarse_nodes, Tf, nlat_f, nlon_f, Tc, nlat_c, nlon_c, dt, a, omega, nu,
                        phibar, prec, slice_groups, coriolis_implicit, implicit_split)
    h = c_void_p()
    _check(_lib.pfasst_create(ctypes.byref(h), ctypes.byref(cfg)))
    return Pfasst(h.value, cfg)


def pfasst_set_initial(pf: Pfasst, theta0: torch.Tensor, stream=None) -> None:
    _check(_lib.pfasst_set_initial(pf.ptr, _ptr(theta0, torch.complex128, 3 * ncoef(pf.cfg.Tf)), _stream(stream)))


def pfasst_predict(pf: Pfasst, stream=None) -> None:
    _check(_lib.pfasst_predict(pf.ptr, _stream(stream)))


def pfasst_iteration(pf: Pfasst, last: bool = False, stream=None) -> None:
    _check(_lib.pfasst_iteration(pf.ptr, 1 if last else 0, _stream(stream)))


def pfasst_iterations(pf: Pfasst, count: int, last: bool = False, stream=None) -> None:
    _check(_lib.pfasst_iterations(pf.ptr, count, 1 if last else 0, _stream(stream)))


def pfasst_residual(pf: Pfasst, res: torch.Tensor, stream=None) -> torch.Tensor:
    """res: float64 [n_ts] on the device; res[n] = max |change of slice n's fine
    end value since the previous call| / max |its end value|."""
    _check(_lib.pfasst_residual(pf.ptr, _ptr(res, torch.float64, pf.cfg.n_ts), _stream(stream)))
    return res


def pfasst_config(n_ts: int, fine_nodes: int, coarse_nodes: int, Tf: int, nlat_f: int, nlon_f: int,
                  Tc: int, nlat_c: int, nlon_c: int, dt: float, a: float, omega: float, nu: float,
                  phibar: float, prec: int | str = PFSH_FP64, slice_groups: int = 0,
                  coriolis_implicit: bool = False, implicit_split: bool = False) -> PfasstConfig:
    prec = PREC_NAMES[prec] if isinstance(prec, str) else prec
    cor = PFSH_CORIOLIS_IMPLICIT if coriolis_implicit else PFSH_CORIOLIS_EXPLICIT
    return PfasstConfig(n_ts, fine_nodes, coarse_nodes, Tf, nlat_f, nlon_f, Tc, nlat_c, nlon_c, dt,
                        SweParams(a, omega, nu, phibar, cor, int(implicit_split)), prec, slice_groups)


def pfasst_ensemble_create(cfgs: list) -> PfasstEnsemble:
    arr = (PfasstConfig * len(cfgs))(*cfgs)
    h = c_void_p()
    _check(_lib.pfasst_ensemble_create(ctypes.byref(h), arr, len(cfgs)))
    return PfasstEnsemble(h.value, list(cfgs))


def pfasst_ensemble_member(ens: PfasstEnsemble, i: int) -> Pfasst:
    """Member i (owned by the ensemble), for pfasst_set_initial / pfasst_get."""
    if not 0 <= i < len(ens.members):
        raise PfshError(PFSH_EINVAL, "pfasst_ensemble_member: index out of range")
    return ens.members[i]


def pfasst_ensemble_predict(ens: PfasstEnsemble, stream=None) -> None:
    _check(_lib.pfasst_ensemble_predict(ens.ptr, _stream(stream)))


def pfasst_ensemble_iterations(ens: PfasstEnsemble, count: int, last: bool = False, stream=None) -> None:
    _check(_lib.pfasst_ensemble_iterations(ens.ptr, count, 1 if last else 0, _stream(stream)))


def pfasst_get(pf: Pfasst, level: int, slice_: int, node: int, out: torch.Tensor, stream=None) -> torch.Tensor:
    T = pf.cfg.Tf if level == 0 else pf.cfg.Tc
    _check(_lib.pfasst_get(pf.ptr, level, slice_, node, _ptr(out, torch.complex128, 3 * ncoef(T)), _stream(stream)))
    return out


def pfsh_sync_status(stream=None) -> None:
    _check(_lib.pfsh_sync_status(_stream(stream)))


def pfsh_kernel_launches() -> int:
    return int(_lib.pfsh_kernel_launches())


def pfsh_profiler_enable(on: bool) -> None:
    _check(_lib.pfsh_profiler_enable(1 if on else 0))


def pfsh_profiler_report() -> dict:
    """{kernel: [launches, total_ms]} of the launches recorded while enabled."""
    import json
    need = _lib.pfsh_profiler_report(None, 0)
    buf = ctypes.create_string_buffer(need + 16)
    _lib.pfsh_profiler_report(buf, len(buf))
    return json.loads(buf.value.decode())


def pfsh_set_check_finite(on: bool) -> None:
    """Opt-in device-side non-finite check of the results of swe_rhs, sdc_sweep
    and the PFASST calls (PFSH_ENUMERIC at the next pfsh_sync_status)."""
    _check(_lib.pfsh_set_check_finite(1 if on else 0))


def pfsh_selftest_wait(polls: int, stream=None) -> None:
    """One CTA waits on an mbarrier nothing arms, with a limit of `polls` polls;
    the next pfsh_sync_status raises PfshError(PFSH_ETIMEOUT)."""
    _check(_lib.pfsh_selftest_wait(polls, _stream(stream)))


def pfsh_alu_peak(prec: int | str) -> float:
    """Measured FMA throughput (TFLOP/s) of the FP64 or FP32 pipe of the current device."""
    prec = PREC_NAMES[prec] if isinstance(prec, str) else prec
    out = c_double()
    _check(_lib.pfsh_alu_peak(prec, ctypes.byref(out)))
    return out.value


def sht_inverse_noalloc(T: int, nlat: int, nlon: int, spec: torch.Tensor, grid: torch.Tensor,
                        stream=None) -> torch.Tensor:
    """FP64 synthesis that allocates no device memory (see include/pfsh.h):
    spec complex128 [batch, ncoef(T)] -> grid float64 [batch, nlat, nlon]."""
    if spec.numel() % ncoef(T):
        raise ValueError(f"spec holds {spec.numel()} coefficients, not a multiple of ncoef({T}) = {ncoef(T)}")
    if spec.device != grid.device:
        raise ValueError("spec and grid must live on the same device")
    batch = spec.numel() // ncoef(T)
    # the library launches on the current device: make it the tensors' device
    with torch.cuda.device(spec.device):
        _check(_lib.sht_inverse_noalloc(T, nlat, nlon, _ptr(spec, torch.complex128, batch * ncoef(T)),
                                        _ptr(grid, torch.float64, batch * nlat * nlon), batch, _stream(stream)))
    return grid
