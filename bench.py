"""Benchmark: two-level PFASST-SH on one GB300 (fine T255 on 384x768, coarse
T127 on 192x384, 32 time slices, 5/3 Gauss-Lobatto nodes, dt = 120 s).

A step is one PFASST iteration (Algorithm 1: fine sweeps, restriction + FAS,
serial coarse chain, interpolation) over all 32 slices -- every stage of the
hot path.  The JSON line reports PFASST iterations/s of the mixed-precision
path (3xBF16 Legendre GEMMs on tensor cores, FP32 FFT/grid, FP64 spectral
bookkeeping; the headline), the same for the plain FP64 GPU path and the
speedup over it, the difference of the two paths' end states, SWE RHS
evaluations/s at T255 with 32 states per call, an end-to-end block solve
through the C ABI with host buffers, the rooflines of the top kernels and the
FP64 CPU oracle timed on a bounded sample.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--prec bf16x3] [--impl reference]

Under torchrun (N > 1) every rank solves an independent replica of the
workload (different bump location); `value` is the whole-job rate.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthetic as syn  # noqa: E402

TF, TC, NTS, NF, NC, DT, NPF = 255, 127, 32, 5, 3, 120.0, 4
GRID_F = syn.gaussian_grid_size(TF)
GRID_C = syn.gaussian_grid_size(TC)
BUMP_AMPLITUDE, BUMP_WIDTH = 120.0, 1.0 / 15.0
WORKLOAD = ("two-level PFASST-SH: T255 (384x768, 5 Lobatto nodes) / T127 (192x384, 3 nodes), "
            "32 time slices, dt=120 s, balanced jet + 120 m Gaussian bump")
# one metric string and unit for both arms (the GPU path and the oracle)
METRIC = "PFASST iterations/s (T255/T127, 32 slices, 5/3 nodes)"
UNIT = "PFASST iterations/s"
ORACLE_SLICES = 16   # slices the oracle advances per timed iteration (scaled to 32)


def env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


# ---------------------------------------------------------------------------
# algorithmic work per unit (flops or bytes one launch must move)
# ---------------------------------------------------------------------------
def legendre_flops(T: int, nlat: int, cols_complex: int) -> float:
    """Real flops of one synthesis or analysis pass over `cols_complex` complex
    columns: per m, 2 (FMA) * 2 (re/im) * (nlat/2) * K_m * cols with K_m = T+2-m."""
    K = sum(T + 2 - m for m in range(T + 1))
    return 4.0 * (nlat // 2) * K * cols_complex


def grid_long_rows(nlon: int, elem: int) -> bool:
    """True when the grid stage of rows of nlon points takes the long-row
    kernel: 10 padded transforms (nlon + nlon/16 + 1 complex entries each)
    exceed the 227 KB of shared memory of a block."""
    return 10 * (nlon + nlon // 16 + 1) * 2 * elem > 227 * 1024


def grid_rhs_bytes(T: int, nlat: int, B: int, elem: int) -> float:
    """HBM bytes of the fused FFT/grid kernel: read 4 spectra (m <= T) of every
    latitude, write 5 hemispheric spectra, complex of `elem`-byte reals."""
    return B * nlat * (T + 1) * (4 + 5) * 2 * elem


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax.append(float(f[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
            os.unlink(self.path)
        except Exception:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------
def initial_state(ps, torch, dev, seed: int):
    """Balanced jet + Gaussian height bump, projected with an FP64 plan of the library."""
    nlat, nlon = GRID_F
    plan = ps.sht_plan_create(TF, nlat, nlon, 1, "fp64")
    lam_c, phi_c = syn.bump_center(seed)
    lam = 2.0 * math.pi * np.arange(nlon) / nlon
    grid = syn.GRAVITY * syn.gaussian_bump(np.array(plan.mu), lam, amplitude=BUMP_AMPLITUDE, width=BUMP_WIDTH,
                                           lam_c=lam_c, phi_c=phi_c)
    d_grid = torch.tensor(grid[None], dtype=torch.float64, device=dev)
    d_spec = torch.empty((1, syn.ncoef(TF)), dtype=torch.complex128, device=dev)
    ps.sht_forward(plan, d_grid, d_spec)
    ps.pfsh_sync_status()
    st = syn.zonal_jet(TF)
    st[0] += d_spec[0].cpu().numpy()
    st[0, 0] = st[0, 0].real
    plan.close()
    phibar = st[0, 0].real / math.sqrt(2.0)
    return st, phibar


def time_iterations(ps, torch, pf, stream, steps: int) -> float:
    """Device time (ms) of one block of `steps` iterations on `stream` (one
    CUDA-graph launch once the block has been captured)."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ps.pfasst_iterations(pf, steps, False)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def prepare_block(ps, pf, steps: int, warmup: int) -> int:
    """Untimed: `warmup` single iterations, then the block of `steps`
    iterations twice (its first call runs eagerly, the second records the
    graph that the timed call replays).  Returns the iterations run."""
    for _ in range(warmup):
        ps.pfasst_iteration(pf, False)
    for _ in range(2):
        ps.pfasst_iterations(pf, steps, False)
    ps.pfsh_sync_status()
    return warmup + 2 * steps


def block_solve(ps, torch, pf, h_in, h_out, d_in, d_out):
    """One block of the user's workflow: H2D initial value, predictor, NPF
    iterations, D2H of the last slice's end value."""
    d_in.copy_(h_in, non_blocking=True)
    ps.pfasst_set_initial(pf, d_in)
    ps.pfasst_predict(pf)
    ps.pfasst_iterations(pf, NPF, True)
    ps.pfasst_get(pf, 0, NTS - 1, NF - 1, d_out)
    h_out.copy_(d_out, non_blocking=True)


def job_time(ms_local: float, dist, device) -> float:
    """Duration of the timed region for the whole job: the maximum over ranks
    (every rank runs its own replica; the job is as slow as its slowest rank)."""
    import torch
    t = torch.tensor([ms_local], device=device, dtype=torch.float64)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(ms_max: float, world: int, steps: int) -> float:
    """Whole-job PFASST iterations/s: every rank advanced its replica by
    `steps` iterations within ms_max."""
    return world * steps / (ms_max / 1e3)


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_1904_05988_gb300 as ps

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    st0, phibar = initial_state(ps, torch, dev, seed=2 + rank)

    def make(prec, **kw):
        return ps.pfasst_create(NTS, NF, NC, TF, *GRID_F, TC, *GRID_C, DT, syn.EARTH_RADIUS, syn.OMEGA, syn.NU,
                                phibar, prec, **kw)

    pf = make(args.prec)
    d_st0 = torch.tensor(st0, dtype=torch.complex128, device=dev)
    stream = torch.cuda.current_stream()
    ps.pfasst_set_initial(pf, d_st0)
    ps.pfasst_predict(pf)
    warmup_run = prepare_block(ps, pf, args.steps, args.warmup)

    # ---- timed region: K iterations of Algorithm 1 over all slices ----
    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.3)
    barrier()
    n0 = ps.pfsh_kernel_launches()
    torch.cuda.nvtx.range_push("pfasst_timed")
    ms = time_iterations(ps, torch, pf, stream, args.steps)
    torch.cuda.nvtx.range_pop()
    barrier()
    launches = ps.pfsh_kernel_launches() - n0
    clk = clocks.stop()
    ps.pfsh_sync_status()
    ms_max = job_time(ms, dist, dev)
    ms_per_step = ms_max / args.steps
    value = job_value(ms_max, world, args.steps)

    # ---- SWE RHS evaluations/s at T255, 32 states per call ----
    def rhs_rate(prec):
        plan_r = ps.sht_plan_create(TF, *GRID_F, 5 * NTS, prec)
        ctx_r = ps.swe_ctx_create(plan_r, syn.EARTH_RADIUS, syn.OMEGA, syn.NU, phibar)
        rhs_in = d_st0[None].repeat(NTS, 1, 1).contiguous()
        rhs_fe, rhs_fi = torch.empty_like(rhs_in), torch.empty_like(rhs_in)
        for _ in range(3):
            ps.swe_rhs(ctx_r, rhs_in, rhs_fe, rhs_fi)
        torch.cuda.synchronize()
        r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        nrhs = 10
        r0.record(stream)
        for _ in range(nrhs):
            ps.swe_rhs(ctx_r, rhs_in, rhs_fe, rhs_fi)
        r1.record(stream)
        torch.cuda.synchronize()
        ctx_r.close()
        plan_r.close()
        return nrhs * NTS / (r0.elapsed_time(r1) / 1e3)

    rhs_per_s = rhs_rate(args.prec)

    # ---- measured FP64/FP32 pipe peaks, then the profiled pass (same workload,
    #      separate from the timed region) ----
    alu = measure_alu_peaks(ps, torch, dev)
    ALU_PEAKS["fp64"], ALU_PEAKS["fp32"] = alu["fp64"], alu["fp32"]
    ps.pfsh_profiler_enable(True)
    ps.pfasst_iterations(pf, 2, False)
    ps.pfsh_profiler_enable(False)
    prof = ps.pfsh_profiler_report()
    rooflines = rooflines_of(prof, args.prec, 2)

    # ---- end to end: host initial value -> block solve -> host end value ----
    h_in = torch.tensor(st0, dtype=torch.complex128).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    d_in = torch.empty_like(d_st0)
    d_out = torch.empty_like(d_st0)
    blocks = max(1, min(3, args.steps))
    for _ in range(2):   # eager run, graph capture
        block_solve(ps, torch, pf, h_in, h_out, d_in, d_out)
    torch.cuda.synchronize()
    b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b0.record(stream)
    for _ in range(blocks):
        block_solve(ps, torch, pf, h_in, h_out, d_in, d_out)
    b1.record(stream)
    torch.cuda.synchronize()
    ms_block = b0.elapsed_time(b1) / blocks
    end_state = h_out.numpy().copy()
    if not np.all(np.isfinite(end_state.view(np.float64))):
        raise RuntimeError("non-finite solution")
    e2e_val = world * NPF / (ms_block / 1e3)
    state_bytes = 3 * syn.ncoef(TF) * 16
    pf.close()

    # ---- the plain FP64 GPU path on the same workload, for the speedup ----
    fp64 = None
    fp64_end = None
    if args.prec != "fp64" and not args.no_fp64_path:
        pf64 = make("fp64")
        ps.pfasst_set_initial(pf64, d_st0)
        ps.pfasst_predict(pf64)
        k64 = max(2, min(5, args.steps))
        prepare_block(ps, pf64, k64, 1)
        ms64 = time_iterations(ps, torch, pf64, stream, k64) / k64
        block_solve(ps, torch, pf64, h_in, h_out, d_in, d_out)
        torch.cuda.synchronize()
        ref = h_out.numpy()
        fp64_end = ref.copy()
        diff = float(np.linalg.norm(end_state - ref) / np.linalg.norm(ref))
        pert = end_state - st0
        pert_ref = ref - st0
        diff_pert = float(np.linalg.norm(pert - pert_ref) / np.linalg.norm(pert_ref))
        pf64.close()
        fp64 = {"value": world * 1e3 / ms64, "unit": UNIT, "ms_per_step": ms64, "steps": k64,
                "swe_rhs_evals_per_s": rhs_rate("fp64"),
                "speedup_of_value": value / (world * 1e3 / ms64),
                "end_state_rel_l2_vs_fp64": diff, "end_state_change_rel_l2_vs_fp64": diff_pert,
                "what": f"end value of slice {NTS - 1} after predictor + {NPF} iterations: relative L2 difference of "
                        "the state, and of its change from the initial value (bump + jet evolution)"}

    # ---- the same workload with the Coriolis term implicit / the two-substep node solve ----
    variants = None
    if not args.no_variants:
        variants = {}
        for name, kw in (("coriolis_implicit", {"coriolis_implicit": True}), ("implicit_split", {"implicit_split": True}),
                         ("coriolis_implicit+implicit_split", {"coriolis_implicit": True, "implicit_split": True})):
            pv = make(args.prec, **kw)
            ps.pfasst_set_initial(pv, d_st0)
            ps.pfasst_predict(pv)
            kv = max(2, min(10, args.steps))
            prepare_block(ps, pv, kv, 1)
            msv = time_iterations(ps, torch, pv, stream, kv) / kv
            block_solve(ps, torch, pv, h_in, h_out, d_in, d_out)
            torch.cuda.synchronize()
            alt = h_out.numpy()
            pv.close()
            variants[name] = {
                "value": world * 1e3 / msv, "unit": "PFASST iterations/s", "ms_per_step": msv, "steps": kv,
                "end_state_change_rel_l2_vs_headline": float(np.linalg.norm((alt - st0) - (end_state - st0))
                                                             / np.linalg.norm(end_state - st0))}
        # the same workload in the other arithmetic forms of the Legendre contractions
        for prec in ("fp32", "bf16", "bf16x6"):
            if prec == args.prec:
                continue
            pv = make(prec)
            ps.pfasst_set_initial(pv, d_st0)
            ps.pfasst_predict(pv)
            kv = max(2, min(10, args.steps))
            prepare_block(ps, pv, kv, 1)
            msv = time_iterations(ps, torch, pv, stream, kv) / kv
            block_solve(ps, torch, pv, h_in, h_out, d_in, d_out)
            torch.cuda.synchronize()
            alt = h_out.numpy()
            pv.close()
            variants["prec_" + prec] = {
                "value": world * 1e3 / msv, "unit": "PFASST iterations/s", "ms_per_step": msv, "steps": kv,
                "end_state_change_rel_l2_vs_fp64": (float(np.linalg.norm((alt - st0) - (fp64_end - st0))
                                                          / np.linalg.norm(fp64_end - st0))
                                                    if fp64_end is not None else None)}

    # ---- opt-in: the large single instance and the uneven batch ----
    large = large_instance(ps, torch, stream, world, args.prec) if args.config5 else None
    uneven = uneven_batch(ps, torch, stream, world, args.prec) if args.uneven else None

    cpu = cpu_baseline_sample() if (rank == 0 and world == 1 and not args.no_cpu_baseline) else None
    if rank == 0:
        dtype = "f64" if args.prec == "fp64" else \
            f"{args.prec} Legendre GEMMs, f32 FFT/grid, f64 spectral/SDC/FAS"
        line = {
            "metric": METRIC,
            "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "iterations_untimed": warmup_run, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_ts": NTS, "nodes": [NF, NC], "T": [TF, TC],
                       "grid": [list(GRID_F), list(GRID_C)], "dt": DT, "prec": args.prec,
                       "parallelism": f"replicas x{world}", "l2": "working set 1.6 GB > 129 MB L2",
                       "timed": f"one pfasst_iterations block of {args.steps} iterations (one CUDA-graph launch, "
                                "slice groups in a wavefront across iterations)"},
            "swe_rhs_evals_per_s": rhs_per_s,
            "fp64_gpu_path": fp64,
            "variants": variants,
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": state_bytes,
                    "d2h_bytes_per_step": state_bytes,
                    "what": f"per block: H2D initial value, predictor, {NPF} iterations, D2H last slice end value"},
            "gpu_launches": int(launches),
            "clocks": clk,
            "roofline": rooflines[0] if rooflines else None,
            "roofline_selection": "dominant = largest summed device time in a profiled pass of 2 iterations "
                                  "after the timed region, every launch on one stream with an event pair around it",
            "rooflines_top": rooflines[1:],
            "alu_peaks": alu["raw"],
            "kernels_ms_per_iteration": {k: round(v[1] / 2, 4) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])},
            "cpu_baseline": cpu,
            "large_instance": large,
            "uneven_batch": uneven,
            # short keys last, so that they stay in the visible end of the line
            "fp64_gpu_it_s": fp64["value"] if fp64 else None,
            "speedup_vs_fp64": fp64["speedup_of_value"] if fp64 else None,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def large_instance(ps, torch, stream, world, prec):
    """T1279 on 1920 x 3840 / T639 on 960 x 1920, 16 slices x 5 / 3 nodes x 3
    fields, dt = 30 s, 3 PFASST iterations timed after one untimed; balanced
    jet plus seeded n^-3 vorticity and divergence spectra of area-rms 1e-6 1/s
    (seed 5).  Tables streamed from HBM (not recomputed on the fly)."""
    W = Workload(1279, 639, 16, 5, 3)
    st = syn.zonal_jet(W.TF)
    pert = syn.random_spectrum(W.TF, (2,), seed=5, rms=1e-6)
    st[1] += pert[0]
    st[2] += pert[1]
    phibar = st[0, 0].real / math.sqrt(2.0)
    t0 = time.perf_counter()
    pf = ps.pfasst_create(W.NTS, W.NF, W.NC, W.TF, *W.GRID_F, W.TC, *W.GRID_C, 30.0, syn.EARTH_RADIUS, syn.OMEGA,
                          syn.NU, phibar, prec)
    ps.pfasst_set_initial(pf, torch.tensor(st, dtype=torch.complex128, device="cuda"))
    ps.pfasst_predict(pf)
    prepare_block(ps, pf, 3, 1)
    setup_s = time.perf_counter() - t0
    ms = time_iterations(ps, torch, pf, stream, 3) / 3
    ps.pfsh_profiler_enable(True)
    ps.pfasst_iterations(pf, 1, False)
    ps.pfsh_profiler_enable(False)
    prof = ps.pfsh_profiler_report()
    ps.pfsh_sync_status()
    pf.close()
    W.groups = 1 if prec == "fp64" else 2
    roofs = rooflines_of(prof, prec, 1, top=3, W=W)
    rec = legendre_recurrence_vs_stream(ps, W, prec, prof)
    return {"workload": "T1279 (1920x3840, 5 nodes) / T639 (960x1920, 3 nodes), 16 slices, dt=30 s, jet + n^-3 "
                        "vorticity/divergence (seed 5)", "prec": prec, "value": world * 1e3 / ms,
            "unit": "PFASST iterations/s", "ms_per_step": ms, "steps": 3, "setup_s": setup_s,
            "roofline": roofs[0] if roofs else None, "rooflines_top": roofs[1:],
            "legendre_recurrence_vs_stream": rec,
            "kernels_ms_per_iteration": {k: round(v[1], 3) for k, v in
                                         sorted(prof.items(), key=lambda kv: -kv[1][1])}}


def legendre_recurrence_vs_stream(ps, W, prec: str, prof: dict) -> dict:
    """The fine level's P_n^m(mu_j) (n <= T+1, one hemisphere) either come
    from HBM as tensor-core images (what the Legendre launches do) or would be
    generated by the FP64 n-recurrence inside each launch.  Measured: the
    library's FP64 table kernel over every (m, n, j) of the fine level (event
    profiler around an FP64 plan creation; it also evaluates the eps
    coefficients with a square root and a division per step), and the fine
    tensor-core launches of the timed workload.  Derived: the bare recurrence
    (one multiply and one FMA per entry) at the measured FP64 peak, and the
    images' bytes at the measured HBM bandwidth."""
    entries = (W.TF + 2) * (W.TF + 3) // 2 * (W.GRID_F[0] // 2)
    ps.pfsh_profiler_enable(True)
    plan = ps.sht_plan_create(W.TF, *W.GRID_F, 1, "fp64")
    ps.pfsh_profiler_enable(False)
    rep = ps.pfsh_profiler_report()
    plan.close()
    table_ms = rep.get("k_legendre_table", [0, None])[1]
    pk, src = peaks()
    fp64_peak = ALU_PEAKS["fp64"][0]
    part_bytes = {"bf16x6": 6, "bf16x3": 4, "bf16": 2, "fp16": 2}.get(prec)
    out = {"entries_per_direction": entries, "fp64_table_kernel_ms": table_ms,
           "fp64_table_kernel_ns_per_entry": table_ms * 1e6 / entries if table_ms else None,
           "bare_fp64_recurrence_ms_at_peak": 2 * entries / (fp64_peak * 1e12) * 1e3,
           "fp64_peak_tflops": fp64_peak}
    if part_bytes:
        out["image_gb_per_direction"] = entries * part_bytes / 1e9
        out["image_stream_ms_at_hbm_peak"] = entries * part_bytes / (pk["hbm_gbs"] * 1e9) * 1e3
        for name in (f"k_synth_{prec}", f"k_anal_{prec}"):
            if name in prof:
                out[f"{name}_ms_per_launch"] = prof[name][1] / prof[name][0]
    return out


def uneven_batch(ps, torch, stream, world, prec):
    """48 independent instances with T drawn from {63, 127, 170, 255} (seed 4),
    coarse level T/2, 8 slices, 5 / 3 nodes, dt = 120 * 256 / (T + 1) s, advanced
    together (pfasst_ensemble_*): instance-iterations/s over one block of 4
    iterations after an untimed one."""
    rng = np.random.default_rng(4)
    Ts = [int(t) for t in rng.choice([63, 127, 170, 255], size=48)]
    cfgs = []
    for T in Ts:
        gf, gc = syn.gaussian_grid_size(T), syn.gaussian_grid_size(T // 2)
        cfgs.append(ps.pfasst_config(8, 5, 3, T, *gf, T // 2, *gc, 120.0 * 256 / (T + 1), syn.EARTH_RADIUS,
                                     syn.OMEGA, syn.NU, syn.GRAVITY * syn.MEAN_DEPTH, prec))
    t0 = time.perf_counter()
    ens = ps.pfasst_ensemble_create(cfgs)
    for i, T in enumerate(Ts):
        st = syn.zonal_jet(T)
        pert = syn.random_spectrum(T, (2,), seed=100 + i, rms=1e-6)
        st[1] += pert[0]
        st[2] += pert[1]
        ps.pfasst_set_initial(ps.pfasst_ensemble_member(ens, i), torch.tensor(st, dtype=torch.complex128,
                                                                              device="cuda"))
    ps.pfasst_ensemble_predict(ens)
    for _ in range(2):   # eager run, graph capture
        ps.pfasst_ensemble_iterations(ens, 4, False)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ps.pfasst_ensemble_iterations(ens, 4, False)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ps.pfsh_sync_status()
    ens.close()
    return {"workload": "48 instances, T in {63,127,170,255} (seed 4; " +
                        ", ".join(f"{t}: {Ts.count(t)}" for t in (63, 127, 170, 255)) +
                        "), coarse T/2, 8 slices, 5/3 nodes", "prec": prec,
            "value": world * 48 * 4 / (ms / 1e3), "unit": "instance-iterations/s", "ms_per_block": ms,
            "iterations_per_block": 4, "setup_s": setup_s,
            "path": "pfasst_ensemble_iterations: every member on its own stream pair, one CUDA graph"}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# Peaks of the FP64 and FP32 pipes (TFLOP/s) with their source.  run_ours
# replaces the nominal figures with the rates measured on the device at hand
# (measure_alu_peaks) before it computes any roofline.
ALU_PEAKS = {"fp64": (1.25, "nominal GB300 FP64 rate 1.25 TFLOP/s"),
             "fp32": (152 * 128 * 2 * 2.07 / 1e3, "nominal: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz")}


def measure_alu_peaks(ps, torch, dev) -> dict:
    """FP64 and FP32 peaks measured on this GPU with CUDA events: the library's
    FMA-loop probe (independent FMA chains on every SM) and, for FP64, cuBLAS
    DGEMM through torch.matmul at 8192^3 (best of 3); the higher of the two is
    the roofline denominator (a well-fed kernel can reach either)."""
    out = {}
    f64_fma = ps.pfsh_alu_peak("fp64")
    f32_fma = ps.pfsh_alu_peak("fp32")
    a = torch.randn(8192, 8192, dtype=torch.float64, device=dev)
    b = torch.randn(8192, 8192, dtype=torch.float64, device=dev)
    c = a @ b
    best = 1e30
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b, out=c)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    dgemm = 2.0 * 8192 ** 3 / (best / 1e3) / 1e12
    del a, b, c
    props = torch.cuda.get_device_properties(dev)
    out["fp64"] = (max(f64_fma, dgemm), f"measured: FMA loop {f64_fma:.3f}, DGEMM 8192^3 {dgemm:.3f} TFLOP/s "
                                        f"(the higher)")
    out["fp32"] = (f32_fma, f"measured: FMA loop {f32_fma:.1f} TFLOP/s on {props.multi_processor_count} SMs")
    out["raw"] = {"fp64_fma_tflops": f64_fma, "fp64_dgemm_tflops": dgemm, "fp32_fma_tflops": f32_fma,
                  "sms": props.multi_processor_count}
    return out


class Workload:
    """Sizes of a two-level PFASST workload (the default: the headline's)."""

    def __init__(self, TF=TF, TC=TC, NTS=NTS, NF=NF, NC=NC, groups=None):
        self.TF, self.TC, self.NTS, self.NF, self.NC = TF, TC, NTS, NF, NC
        self.GRID_F, self.GRID_C = syn.gaussian_grid_size(TF), syn.gaussian_grid_size(TC)
        self.groups = groups


HEADLINE = Workload()


def rhs_states_per_iteration(W: Workload = HEADLINE):
    """RHS evaluations in one (non-final) iteration of Algorithm 1 over all
    slices: fine = sweep nodes 1..Mf + node 0 after Step D (batched);
    coarse batched = every node in Step B; coarse chain = node 0 of slices
    1.. + sweep nodes 1..Mc, one state per call (small-batch kernels)."""
    fine = W.NTS * (W.NF - 1) + W.NTS
    coarse_batched = W.NTS * W.NC
    coarse_chain = (W.NTS - 1) + W.NTS * (W.NC - 1)
    return fine, coarse_batched, coarse_chain


def kernel_work_per_iteration(name: str, prec: str, W: Workload = HEADLINE):
    """(algorithmic work, unit, bound, note) of all launches of `name` in one
    iteration of the workload W; None if the kernel has no model."""
    TF, TC, NTS, NF, NC, GRID_F, GRID_C = W.TF, W.TC, W.NTS, W.NF, W.NC, W.GRID_F, W.GRID_C
    nfs, ncb, ncs = rhs_states_per_iteration(W)
    (nlat_f, _), (nlat_c, _) = GRID_F, GRID_C
    ncf, ncc = syn.ncoef(TF), syn.ncoef(TC)
    ncf1, ncc1 = syn.ncoef(TF + 1), syn.ncoef(TC + 1)
    elem = 8 if prec == "fp64" else 4
    st_f, st_c = 48 * ncf, 48 * ncc       # bytes of one FP64 state (3 fields, complex)
    tc = prec in ("bf16", "fp16", "bf16x3", "bf16x6")
    simt_bound = ("alu", "FP64 pipe") if prec == "fp64" else ("alu", "FP32 pipe")
    if name.startswith("k_synth") or name.startswith("k_anal"):
        synth = name.startswith("k_synth")
        cols = 4 if synth else 5
        w = nfs * legendre_flops(TF, nlat_f, cols) + ncb * legendre_flops(TC, nlat_c, cols)
        # bytes: per state the activations in and the results out (complex
        # fp32), per launch the Legendre table (bf16 hi/lo images for 3xBF16,
        # bf16 for bf16/fp16, fp32 rows for fp32, fp64 for FP64)
        def per_state(T, nlat):
            spec = syn.ncoef(T + 1) * cols * 8
            four = (T + 1) * nlat * cols * 8
            return spec + four
        tab = {"bf16x6": 6, "bf16x3": 4, "bf16": 2, "fp16": 2, "fp32": 4, "fp64": 8}[prec]
        def table(T, nlat):
            return (T + 2) * (T + 3) // 2 * (nlat // 2) * tab
        groups = W.groups if W.groups else (1 if prec == "fp64" else 2)
        byts = (nfs * per_state(TF, nlat_f) + ncb * per_state(TC, nlat_c) +
                groups * (NF * table(TF, nlat_f) + NC * table(TC, nlat_c)))
        if prec == "fp64":
            byts *= 2   # fp64 complex activations and results
        if tc:
            mult = {"bf16x3": 3, "bf16x6": 6}.get(prec, 1)
            return w, "flop", ("tensor", f"{mult} MMA products per algorithmic flop"), byts
        return w, "flop", simt_bound, byts
    if name.startswith("k_small_synth") or name.startswith("k_small_anal"):
        cols = 4 if "synth" in name else 5
        return ncs * legendre_flops(TC, nlat_c, cols), "flop", simt_bound, None
    if name in ("k_grid_rhs", "k_grid_rhs_long"):
        want = name == "k_grid_rhs_long"
        w = (nfs * grid_rhs_bytes(TF, nlat_f, 1, elem) * (grid_long_rows(GRID_F[1], elem) == want) +
             (ncb + ncs) * grid_rhs_bytes(TC, nlat_c, 1, elem) * (grid_long_rows(GRID_C[1], elem) == want))
        return w, "byte", ("hbm", None), None
    if name == "k_rhs_prep":
        return (nfs * (st_f + 4 * ncf1 * 2 * elem) + ncb * (st_c + 4 * ncc1 * 2 * elem), "byte", ("hbm", None), None)
    if name == "k_rhs_assemble":
        return (nfs * (5 * ncf1 * 2 * elem + 3 * st_f) + ncb * (5 * ncc1 * 2 * elem + 3 * st_c), "byte",
                ("hbm", None), None)
    if name == "k_sdc_old":
        # fine sweeps of every slice: F_E and F_I at every node into M old
        # parts; per real component M(M+1)/2 coefficient pairs take two FMAs
        # and M(M+1)/2 (j = 0 or j > i, equal coefficients) one FMA on the sum
        # F_E + F_I (M+1 additions): (M+1)(3M+1) flops, 2x per complex
        # coefficient; FP64-pipe bound (measured 83% busy)
        mf = NF - 1
        return NTS * 3 * ncf * 2 * (mf + 1) * (3 * mf + 1), "flop", ("alu", "FP64 pipe"), None
    if name == "k_chain_node":
        # every launch but the first of a group analyses one node (5 columns)
        # and synthesises the next (4 columns) of one T127 slice
        n = NTS * (NC - 1)
        return n * (legendre_flops(TC, nlat_c, 5) + legendre_flops(TC, nlat_c, 4)), "flop", simt_bound, None
    if name == "k_sdc_node":
        mf, mc = NF - 1, NC - 1
        return NTS * (mf * (mf + 1) * st_f + mc * (mc + 1) * st_c), "byte", ("hbm", None), None
    if name == "k_interp_inc":
        return 3 * NTS * (2 * NC + 2 * (NF - 1)) * st_c, "byte", ("hbm", None), None
    if name == "k_fas":
        return NTS * (2 * NF + 2 * NC + NC) * st_c, "byte", ("hbm", None), None
    if name == "k_restrict":
        return NTS * (NF + NC) * st_c, "byte", ("hbm", None), None
    if name == "k_node0":
        return (NTS - 1) * (2 * st_f + st_c), "byte", ("hbm", None), None
    return None


# DRAM bytes of one launch (dram__bytes_read.sum + dram__bytes_write.sum) from an ncu capture of
# the kernel as it is built now, on this workload: (bytes, precisions it applies to, summary file).
# Kernels whose launches in the profiled pass differ in shape (two levels, several batch sizes)
# have none.
NCU_TRAFFIC = {
    "k_chain_node": (5.142784e6, ("bf16x3", "bf16", "fp16", "fp32"), "profiles/k_chain_node_T127_bf16x3.md"),
    "k_sdc_old": (353.359616e6, ("bf16x3", "bf16", "fp16", "fp32", "fp64"), "profiles/k_sdc_old_T255_16slices.md"),
}


def roofline_entry(name: str, n: int, tot_ms: float, prec: str, iterations: int, W: Workload = HEADLINE) -> dict:
    tr = NCU_TRAFFIC.get(name) if W is HEADLINE else None
    out = {"kernel": name, "launches": n, "mean_launch_ms": tot_ms / n,
           "traffic": tr[0] if tr and prec in tr[1] else None}
    if out["traffic"] is not None:
        out["traffic_source"] = f"ncu capture of one launch, {tr[2]}"
    model = kernel_work_per_iteration(name, prec, W)
    if model is None:
        out.update({"bound": "unknown", "achieved": None, "peak": None, "unit": None, "frac": None})
        return out
    work, unit, (bound, note), byts = model
    rate = work * iterations / (tot_ms / 1e3)
    pk, src = peaks()
    if bound == "tensor" and byts:
        # per-order GEMMs at this batch: below the bf16 ridge (peak flops /
        # HBM bandwidth) the table and activation traffic bounds them
        mult = int(note.split()[0]) if note and note.split()[0].isdigit() else 1
        intensity = mult * work / byts
        ridge = pk["bf16_tflops_sustained"] * 1e12 / (pk["hbm_gbs"] * 1e9)
        if intensity < ridge:
            brate = byts * iterations / (tot_ms / 1e3)
            out.update({"bound": "hbm", "achieved": brate / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s",
                        "frac": brate / 1e9 / pk["hbm_gbs"], "peak_source": f"{src} copy bandwidth",
                        "note": f"tensor-core GEMM below the ridge: {intensity:.0f} executed flop/B vs "
                                f"{ridge:.0f}; tensor pipe at {rate * mult / 1e12 / pk['bf16_tflops_sustained']:.3f} "
                                f"of the bf16 peak ({note})"})
            return out
    if bound == "tensor":
        peak = pk["bf16_tflops_sustained"]
        out.update({"bound": "tensor", "achieved": rate / 1e12, "peak": peak, "unit": "TFLOP/s",
                    "frac": rate / 1e12 / peak, "peak_source": f"{src} cuBLAS bf16 sustained",
                    "note": f"algorithmic Legendre flops; {note}"})
    elif bound == "alu":
        peak, src_alu = ALU_PEAKS["fp64" if note == "FP64 pipe" else "fp32"]
        out.update({"bound": "alu", "achieved": rate / 1e12, "peak": peak, "unit": "TFLOP/s",
                    "frac": rate / 1e12 / peak, "peak_source": src_alu})
    else:
        out.update({"bound": "hbm", "achieved": rate / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s",
                    "frac": rate / 1e9 / pk["hbm_gbs"], "peak_source": f"{src} copy bandwidth"})
    return out


def rooflines_of(prof: dict, prec: str, iterations: int, top: int = 5, W: Workload = HEADLINE) -> list:
    """Rooflines of the `top` kernels by total time in the profiled pass:
    algorithmic work of their launches / their summed duration (= work per
    launch / mean launch duration).  The first entry is the dominant kernel."""
    if not prof:
        return []
    items = sorted(prof.items(), key=lambda kv: -kv[1][1])[:top]
    return [roofline_entry(name, n, tot, prec, iterations, W) for name, (n, tot) in items]


# ---------------------------------------------------------------------------
# CPU oracle (bounded sample)
# ---------------------------------------------------------------------------
def oracle_problem(n_ts: int):
    from oracle.pfasst import PFASST
    from oracle.sdc import SDCLevel
    from oracle.sht import SHT, unpack
    from oracle.swe import SWEParams

    lam_c, phi_c = syn.bump_center(2)
    sht = SHT(TF, *GRID_F, L=TF + 1)
    lam = 2.0 * math.pi * np.arange(GRID_F[1]) / GRID_F[1]
    bump = syn.GRAVITY * syn.gaussian_bump(sht.mu, lam, amplitude=BUMP_AMPLITUDE, width=BUMP_WIDTH,
                                           lam_c=lam_c, phi_c=phi_c)
    st = unpack(syn.zonal_jet(TF), TF)
    st[0] += sht.analysis(bump, TF + 1)
    phibar = st[0, 0, 0].real / math.sqrt(2.0)
    p = SWEParams(a=syn.EARTH_RADIUS, omega=syn.OMEGA, g=syn.GRAVITY, nu=syn.NU, phibar=phibar)
    pf = PFASST(SDCLevel(TF, *GRID_F, NF, DT, p), SDCLevel(TC, *GRID_C, NC, DT, p), n_ts)
    return pf, st


def proc_cpu_seconds(pids) -> float:
    """User + system CPU seconds of the given processes so far (Linux /proc)."""
    tck = os.sysconf("SC_CLK_TCK")
    tot = 0.0
    for pid in pids:
        try:
            with open(f"/proc/{pid}/stat") as fh:
                f = fh.read().rsplit(")", 1)[1].split()
            tot += (int(f[11]) + int(f[12])) / tck
        except (OSError, IndexError, ValueError):
            pass
    return tot


class OracleRun:
    """The FP64 oracle on ORACLE_SLICES of the 32 slices, its slice-independent
    steps in worker processes on every host core; CPU time is counted over the
    parent and the workers."""

    def __init__(self):
        from oracle.pool import SlicePool
        self.pf, self.st = oracle_problem(ORACLE_SLICES)
        self.pool = SlicePool({"f": self.pf.f.args, "c": self.pf.c.args},
                              workers=min(ORACLE_SLICES, os.cpu_count() or 1))
        self.pf.pool = self.pool
        self.pids = [os.getpid()] + self.pool.pids()

    def iterations(self, k: int):
        """(wall seconds, CPU seconds) of k iterations."""
        c0, t0 = proc_cpu_seconds(self.pids), time.perf_counter()
        for _ in range(k):
            self.pf.iteration(False)
        return time.perf_counter() - t0, proc_cpu_seconds(self.pids) - c0

    def close(self):
        self.pool.close()


def cpu_baseline_sample(steps: int = 1):
    """Oracle: one Algorithm-1 iteration over 16 of the 32 slices (after its
    own predictor) on every host core, scaled x2 to a 32-slice iteration (the
    serial coarse chain is linear in the slices, the parallel steps take two
    rounds of the workers for 32 slices)."""
    o = OracleRun()
    try:
        o.pf.predict(o.st)
        wall, cpu = o.iterations(steps)
        dt = wall / steps
        used = cores_used(cpu, wall)
        # one T255 RHS evaluation (F_E and F_I of one state), best of 2, in this process
        t_rhs = []
        for _ in range(2):
            t0 = time.perf_counter()
            o.pf.f.eval_f(o.st)
            t_rhs.append(time.perf_counter() - t0)
    finally:
        o.close()
    scale = NTS / ORACLE_SLICES
    return {"value": 1.0 / (dt * scale), "unit": UNIT, "cores": used,
            "kind": "oracle", "sample": f"{steps} iteration(s) over {ORACLE_SLICES} of {NTS} slices at T255/T127, "
                                        f"scaled x{scale:g}; {dt:.1f} s each; slice-independent steps in "
                                        f"{o.pool.workers} worker processes; numpy {np.__version__}; "
                                        f"{os.cpu_count()} host cores, {used} busy on average",
            "swe_rhs_evals_per_s": 1.0 / min(t_rhs),
            "swe_rhs_sample": f"one T255 state on one core, best of 2 ({min(t_rhs):.2f} s)"}


def cores_used(cpu_s: float, wall_s: float) -> int:
    """Cores the oracle kept busy on average: CPU time of the parent and its
    worker processes / wall time."""
    return max(1, int(round(cpu_s / max(wall_s, 1e-9))))


def run_reference(args, rank, world):
    if rank != 0:
        return
    o = OracleRun()
    try:
        o.pf.predict(o.st)
        o.iterations(args.warmup)
        el, cpu = o.iterations(args.steps)
    finally:
        o.close()
    used = cores_used(cpu, el)
    scale = NTS / ORACLE_SLICES
    value = args.steps / (el * scale)
    cpu_b = {"value": value, "unit": UNIT, "cores": used, "kind": "oracle",
             "sample": f"each step: one iteration over {ORACLE_SLICES} of {NTS} slices at T255/T127, scaled "
                       f"x{scale:g}; slice-independent steps in {o.pool.workers} worker processes; "
                       f"{os.cpu_count()} host cores, {used} busy on average"}
    print(json.dumps({
        "impl": "reference", "metric": METRIC,
        "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": el / args.steps * 1e3 * scale, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_ts": NTS, "nodes": [NF, NC], "T": [TF, TC], "dt": DT, "prec": "fp64"},
        "cpu_baseline": cpu_b,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--prec", default="bf16x3", choices=["fp64", "fp32", "bf16", "fp16", "bf16x3", "bf16x6"])
    ap.add_argument("--no-fp64-path", action="store_true", help="skip timing the FP64 GPU path")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip timing the Coriolis-implicit and two-substep variants of the workload and the other "
                         "arithmetic forms")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--config5", action="store_true",
                    help="also time the large single instance (T1279/T639, 16 slices, 3 iterations)")
    ap.add_argument("--uneven", action="store_true",
                    help="also time the uneven batch of 48 instances (T from {63,127,170,255})")
    args = ap.parse_args()
    rank, world, local_rank = env_int("RANK", 0), env_int("WORLD_SIZE", 1), env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
