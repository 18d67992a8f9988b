"""Helpers shared by the tests: build/load the CUDA library on demand."""
import importlib.util
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pfsh.h")


def ensure_built() -> str:
    path = os.path.join(ROOT, "paper_1904_05988_gb300", "build.py")
    spec = importlib.util.spec_from_file_location("_pfsh_build", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.build()


def declared_functions() -> list[str]:
    """Names of the functions declared in include/pfsh.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_]\w*\s*\**\s*([A-Za-z_]\w*)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if n not in ("defined",)))


# Error laws of the mixed-precision forms (rounding-derived bounds of the GPU tests).
# u = unit rounding of the form's operands: fp32 2^-24; bf16 2^-9 (8 stored
# mantissa bits); 3xBF16 2^-17 (the hi/lo split keeps about 16 bits); 6xBF16
# 2^-24 (the three-part split keeps about 24 bits, the precision of fp32).  The
# transforms lose a few u; the nonlinear tendency F_E is a spectral derivative
# (div/curl, factors n eps ~ n/2, and n(n+1)/a^2 on E) of analysed fluxes, so its
# rounding error at degree n grows like u (n+1).  Measured on GB300 over
# T63/T170/T255 and all three fields, max_n e_n / (u (n+1) |F_E|) <= 11.2 (fp32
# delta tendency at T255; bf16 <= 3.4, 3xBF16 <= 1.2), the whole-field error
# <= 37 u (T+1) and the error over the band n <= T/4 <= 5.1 u (T/4 + 1).
U_FORM = {"fp32": 2.0 ** -24, "bf16": 2.0 ** -9, "bf16x3": 2.0 ** -17, "bf16x6": 2.0 ** -24, "fp16": 2.0 ** -11}
C_DEGREE, C_WHOLE, C_LOWBAND = 24.0, 48.0, 8.0


def rhs_bounds(form, T):
    """(per-degree constant, whole-field rel-L2 bound, low-band rel-L2 bound) of F_E."""
    u = U_FORM[form]
    return C_DEGREE * u, C_WHOLE * u * (T + 1), C_LOWBAND * u * (T // 4 + 1)


def change_bound(form, T):
    """Bound on the relative L2 error of the change of a state over a PFASST block
    (fine level at truncation T): the change integrates the tendencies, whose
    low-degree band carries it (n^-3 spectra, jet, bump), so it inherits the
    low-band law of F_E."""
    return C_LOWBAND * U_FORM[form] * (T // 4 + 1)


def per_degree_excess(got, ref, T, form):
    """max over degrees n of e_n / (u (n+1) |ref|) for packed spectra of one field
    (e_n = L2 error over the orders of degree n)."""
    import numpy as np
    deg = np.concatenate([np.arange(m, T + 1) for m in range(T + 1)])
    en = np.sqrt(np.bincount(deg, weights=np.abs(np.asarray(got) - np.asarray(ref)) ** 2, minlength=T + 1))
    return float((en / (np.linalg.norm(ref) * U_FORM[form] * (np.arange(T + 1) + 1))).max())


def low_band_rel(got, ref, T):
    import numpy as np
    deg = np.concatenate([np.arange(m, T + 1) for m in range(T + 1)])
    sel = deg <= T // 4
    return float(np.linalg.norm((np.asarray(got) - np.asarray(ref))[sel]) / np.linalg.norm(np.asarray(ref)[sel]))
