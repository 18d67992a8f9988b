"""Small self-contained GPU cases for ncu captures of single kernels.

Each case builds what its kernel needs, runs it a few times and exits; run one
case per process.  Sizes exceed the 129 MB L2 while the process holds a few GB
of device memory.

  python tests/profile_cases.py grid_long
      k_grid_rhs_long (fp32, nlon = 3840: six padded rows in shared memory,
      row means centred because nlon / 5 <= T): T767 on 1920 x 3840, 4 states,
      seeded n^-3 spectra, 4 swe_rhs calls.
"""
from __future__ import annotations

import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
for _p in (ROOT, HERE):
    if _p not in sys.path:
        sys.path.insert(0, _p)

import synthetic as syn  # noqa: E402


def grid_long(ps, torch):
    T, nlat, nlon, B = 767, 1920, 3840, 4
    free0 = torch.cuda.mem_get_info()[0]
    st = syn.zonal_jet(T)[None].repeat(B, axis=0)
    phibar = st[0, 0, 0].real / 2 ** 0.5
    plan = ps.sht_plan_create(T, nlat, nlon, 5 * B, "fp32")   # 5 transform columns per state
    ctx = ps.swe_ctx_create(plan, syn.EARTH_RADIUS, syn.OMEGA, syn.NU, phibar)
    pert = syn.random_spectrum(T, (B, 2), seed=767, rms=1e-6)
    st[:, 1:] += pert
    x = torch.tensor(st, dtype=torch.complex128, device="cuda")
    fE, fI = torch.empty_like(x), torch.empty_like(x)
    for _ in range(4):
        ps.swe_rhs(ctx, x, fE, fI)
    ps.pfsh_sync_status()
    used = (free0 - torch.cuda.mem_get_info()[0]) / 1e9
    print(f"grid_long: T{T} on {nlat} x {nlon}, {B} states, fp32; {used:.2f} GB on the device; "
          f"|F_E| {float(fE.abs().max()):.3e}")
    ctx.close()
    plan.close()


CASES = {"grid_long": grid_long}


def main():
    if len(sys.argv) != 2 or sys.argv[1] not in CASES:
        raise SystemExit(f"usage: {sys.argv[0]} {'|'.join(CASES)}")
    import torch
    from _lib import ensure_built
    ensure_built()
    import paper_1904_05988_gb300 as ps
    CASES[sys.argv[1]](ps, torch)


if __name__ == "__main__":
    main()
