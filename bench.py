"""Throughput of the split pressure-gradient projection on one GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Workload: the 256^3 multimode two-phase problem (density 640/60, 6-cell tanh
layer, 8 seeded interface modes), box 2 pi, periodic x and z, walls in y.  One
step = one whole projection (rho_0, Eq. (34) right-hand side, direct Poisson
solve, Eq. (33) correction) through the C ABI (ppe_project).  The headline form
solves in FP32 inside an FP64-residual iterative refinement to a relative
residual of 1e-10; the plain FP64 form is timed beside it.  Inputs (7 fields,
~0.94 GB) are larger than L2, so no flush is needed between steps.

Prints ONE JSON line (rank 0).  For N > 1 every rank runs an independent replica
of the workload on its own GPU (no collective on the data path); value is the
total solves of all ranks over the slowest rank's time.

--impl reference times the FP64 CPU oracle (the reference arm: a plain,
single-threaded C++ restatement of the paper's method with its own FFT and
Thomas solver) on this host.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "PPE projection solves/s & Gpts/s at 256³ (FP64 vs FP32+refine @1e-10); % HBM roof"
WORKLOAD = "multimode_256: 256x256x256, density 640/60, FP32 solve + FP64 refinement to rel residual 1e-10"
NX = NY = NZ = 256
N_CELLS = NX * NY * NZ
F_BYTES = 8 * N_CELLS


def set_grid(nx: int, ny: int | None = None, nz: int | None = None):
    """Grid of profiling runs of a smaller case (the bench line itself is 256^3)."""
    global NX, NY, NZ, N_CELLS, F_BYTES, WORKLOAD
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    NX, NY, NZ = nx, ny, nz
    N_CELLS = nx * ny * nz
    F_BYTES = 8 * N_CELLS
    if (nx, ny, nz) != (256, 256, 256):
        WORKLOAD = (f"multimode {nx}x{ny}x{nz} (profiling case), density 640/60, FP32 solve + FP64 refinement "
                    f"to rel residual 1e-10")


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# FP64 FMA throughput of a GB300 as measured by an FMA-chain probe on this machine
# (1.19 TFLOP/s; 152 SMs at ~2.0 GHz), used as the ALU roof of FP64-bound kernels.
FP64_TFLOPS_MEASURED = 1.19


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        import tempfile
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# algorithmic bytes per kernel launch (unique bytes a launch must move)
# ---------------------------------------------------------------------------
def p0_fp32() -> bool:
    """ppe_project keeps the first solve's p in FP32 on this grid (nx/2 a power of
    two in 16 .. 256 and (nx/2) nz a power of two; the FP32 form with sweeps)."""
    m = NX // 2
    return 16 <= m <= 256 and (m & (m - 1)) == 0 and ((m * NZ) & (m * NZ - 1)) == 0


def kernel_bytes(kernel: str, fp32: bool) -> float:
    F = float(F_BYTES)
    Fv = F * (NY + 1) / NY
    spec = (NX // 2 + 1) * NY * NZ * (8 if fp32 else 16)
    # the first solve's p and the first sweep's reads of it: FP32 where kept so
    # (the bench workload converges in one sweep), else pairs
    P0 = F / 2 if (fp32 and p0_fp32()) else F
    table = {
        # pass 1 of the minimal-pass count: the 7 FP64 inputs in, f (pairs, kept
        # for the residual) out.  The kernel also writes the split velocities
        # u_pre, v_pre, w_pre, an intermediate of this implementation that the
        # correction reads in place of the 6 inputs it would otherwise re-read;
        # they are not counted here.
        "k_rhs_march": 6 * F + Fv + F,
        "k_xfwd_f": F + spec,
        "k_xfwd_resid": F + P0 + spec,                  # f (pairs), p -> spectrum
        "k_zfft_fwd": 2 * spec,
        "k_ysolve": 2 * spec,
        "k_zfft_inv": 2 * spec,
        "k_xinv": spec + (P0 if fp32 else F),           # -> p (FP64, FP32 or pairs)
        "k_xinv_accum": spec + P0 + F,                  # p (first solve's) + delta -> p (pairs)
        # u_pre + p in, u, v, w out; the refinement form's fused check also reads
        # f (pairs) and writes p as FP64
        "k_correct": (2 * F + Fv) + F + (2 * F + Fv) + (2 * F if fp32 else 0),
        "k_rho_min": F,
    }
    return table.get(kernel, 0.0)


def measured_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` at 256^3 from profiles/traffic.json
    (an ncu capture, scaled by cells when taken on a smaller grid), or None if
    the file is missing or the kernel's source has changed since the capture."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            doc = json.load(fh)
        entry = doc["kernels"][kernel]
        h = hashlib.sha256()
        for src in entry["sources"]:
            with open(os.path.join(ROOT, src), "rb") as fh:
                h.update(fh.read())
        if h.hexdigest() != entry["source_sha256"]:
            return None
        return float(entry["bytes_per_launch_256"])
    except Exception:
        return None


def step_min_bytes(fp32: bool, sweeps: int) -> float:
    """Minimal-pass traffic of one projection: 21F for FP64 (7 inputs read,
    two half-spectrum round trips, 6 fields re-read by the correction, 4
    outputs written); FP32 + refinement (21 + 6k)F for k sweeps."""
    return F_BYTES * (21 + (6 * sweeps if fp32 else 0))


# ---------------------------------------------------------------------------
# Replicas (one independent projection per rank, no data-path collective)
# ---------------------------------------------------------------------------
def replica_seed(rank: int) -> int:
    """Each rank projects its own seeded fields (the replicas share nothing)."""
    return 2 + rank


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """The job's time is the slowest rank's (MAX all-reduce; identity for one rank)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, steps: int, ms_max: float) -> float:
    """Projections per second of the whole job: every rank ran `steps` in at most ms_max."""
    return world * steps / (ms_max * 1e-3)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_gpu(args):
    import numpy as np
    import torch

    from paper_2103_01874_gb300 import fields, ppe

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    if (NX, NY, NZ) == (256, 256, 256):
        fl = fields.multimode_256(seed=replica_seed(rank))
    else:
        fl = fields.make_fields(NX, NY, NZ, seed=replica_seed(rank), recipe="multimode", width=6.0, rho_g=60.0)
    d = {k: torch.from_numpy(v).to(dev) for k, v in fl.arrays().items()}
    c = fl.shape
    out = dict(p=torch.empty(c, dtype=torch.float64, device=dev), u=torch.empty_like(d["u"]),
               v=torch.empty_like(d["v"]), w=torch.empty_like(d["w"]))
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if dist is not None:
            dist.barrier()

    def timed(plan, steps, warmup, profile=False):
        profile = profile or args.host_refine
        for _ in range(warmup):
            plan.project(d["u"], d["v"], d["w"], d["S"], d["rho"], d["p_n"], d["p_nm1"], fl.dt,
                         out["p"], out["u"], out["v"], out["w"])
        torch.cuda.synchronize(dev)
        barrier()
        torch.cuda.synchronize(dev)
        plan.profile(profile)
        if profile:
            plan.profile_read()  # clear
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            plan.project(d["u"], d["v"], d["w"], d["S"], d["rho"], d["p_n"], d["p_nm1"], fl.dt,
                         out["p"], out["u"], out["v"], out["w"])
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        kt = plan.profile_read() if profile else {}
        plan.profile(False)
        return max_over_ranks(ms, dist, dev), kt

    def step_latency(plan, runs=60):
        """Device time of each of `runs` back-to-back projections (one CUDA event
        between consecutive ones on the plan's stream): median, p99 and extremes."""
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(runs + 1)]
        ev[0].record(stream)
        for i in range(runs):
            plan.project(d["u"], d["v"], d["w"], d["S"], d["rho"], d["p_n"], d["p_nm1"], fl.dt,
                         out["p"], out["u"], out["v"], out["w"])
            ev[i + 1].record(stream)
        torch.cuda.synchronize(dev)
        t = sorted(ev[i].elapsed_time(ev[i + 1]) for i in range(runs))
        return {"runs": runs, "median_ms": statistics.median(t), "p99_ms": t[min(runs - 1, math.ceil(0.99 * runs) - 1)],
                "min_ms": t[0], "max_ms": t[-1]}

    steps, warmup = args.steps, args.warmup
    forms = set(args.forms.split(","))
    plan32 = ppe.Plan(NX, NY, NZ, fl.lx, fl.ly, fl.lz, precision=ppe.FP32_REFINE, refine_tol=1e-10,
                      max_sweeps=args.max_sweeps, stream=stream)
    with ClockSampler(dev.index if world > 1 else 0) as clk:
        ms32, _ = timed(plan32, steps, warmup)
    clocks = clk.summary()
    lat32 = step_latency(plan32)
    info32 = plan32.info(allow_not_converged=True)
    # per-kernel event timing over a second timed region of the same steps
    ms32p, kt32 = timed(plan32, steps, 1, profile=True) if args.kernel_times else (0.0, {})

    # the spectral schedules of the same plan, timed back to back (the headline
    # above used the plan's default schedule)
    schedules = {}
    if args.schedules:
        default = plan32.get_tuning()["spectral"]
        for name, sv in (("legacy", ppe.SPECTRAL_LEGACY), ("fused", ppe.SPECTRAL_FUSED),
                         ("pencil", ppe.SPECTRAL_PENCIL)):
            try:
                plan32.set_tuning(spectral=sv)
            except ppe.PPEError:
                continue
            ms_s, _ = timed(plan32, steps, warmup)
            _, kt_s = timed(plan32, max(3, steps // 5), 1, profile=True)
            schedules[name] = {"ms_per_step": ms_s / steps, "default": sv == default,
                               "kernel_avg_us": {k: 1e3 * v[1] / v[0] for k, v in kt_s.items()}}
        plan32.set_tuning(spectral=default)

    steps64 = max(1, steps // 2)
    ms64, kt64 = 0.0, {}
    if "fp64" in forms:
        plan64 = ppe.Plan(NX, NY, NZ, fl.lx, fl.ly, fl.lz, precision=ppe.FP64, stream=stream)
        ms64, _ = timed(plan64, steps64, max(3, warmup // 2))
        if args.kernel_times:
            _, kt64 = timed(plan64, steps64, 1, profile=True)

    # e2e: the same projection from pinned host buffers through the pipelined
    # host API (ppe_project_host_async: each step copies its 7 input fields in
    # and p, u, v, w out; consecutive steps overlap their copies and compute;
    # two output sets so that a step's results are not overwritten in flight)
    hin = {k: torch.from_numpy(v).pin_memory() for k, v in fl.arrays().items()}
    houts = [dict(p=torch.empty(c, dtype=torch.float64).pin_memory(),
                  u=torch.empty(c, dtype=torch.float64).pin_memory(),
                  v=torch.empty(fl.v.shape, dtype=torch.float64).pin_memory(),
                  w=torch.empty(c, dtype=torch.float64).pin_memory()) for _ in range(2)]
    hout = houts[0]

    def host_step(i):
        o = houts[i % 2]
        plan32.project_host_async(hin["u"], hin["v"], hin["w"], hin["S"], hin["rho"], hin["p_n"], hin["p_nm1"],
                                  fl.dt, o["p"], o["u"], o["v"], o["w"])

    e_steps = max(2, steps // 2)
    e2e_s = float("nan")
    if not args.no_e2e:
        for i in range(2):
            host_step(i)
        plan32.host_wait()
        barrier()
        t0 = time.perf_counter()
        for i in range(e_steps):
            host_step(i)
        plan32.host_wait()
        torch.cuda.synchronize(dev)
        e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, dist, dev)
    h2d = sum(v.numel() * 8 for v in hin.values())
    d2h = sum(v.numel() * 8 for v in hout.values())

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return None

    hbm, hbm_src = peaks()
    per_step32 = ms32 / steps
    value = whole_job_rate(world, steps, ms32)
    # dominant kernel of the headline form
    dom = max(kt32.items(), key=lambda kv: kv[1][1]) if kt32 else (None, (0, 0.0))
    dname, (dl, dms) = dom
    avg_ms = dms / dl if dl else float("nan")
    step_total = sum(v[1] for v in kt32.values()) or 1.0
    kernels = {k: {"launches": v[0], "avg_us": 1e3 * v[1] / v[0], "share": v[1] / step_total,
                   "GBps": (kernel_bytes(k, True) / (1e-3 * v[1] / v[0]) / 1e9) if kernel_bytes(k, True) else None}
               for k, v in sorted(kt32.items(), key=lambda kv: -kv[1][1])}
    k64_total = sum(v[1] for v in kt64.values()) or 1.0
    kernels64 = {k: {"launches": v[0], "avg_us": 1e3 * v[1] / v[0], "share": v[1] / k64_total,
                     "GBps": (kernel_bytes(k, False) / (1e-3 * v[1] / v[0]) / 1e9) if kernel_bytes(k, False) else None}
                 for k, v in sorted(kt64.items(), key=lambda kv: -kv[1][1])}
    dbytes = kernel_bytes(dname, True) if dname else 0.0
    achieved = dbytes / (avg_ms * 1e-3) / 1e9 if dbytes and avg_ms > 0 else None
    traffic = measured_traffic(dname) if dname else None
    roof = {"kernel": dname, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": (achieved / hbm) if achieved else None, "traffic": traffic,
            "algorithmic_bytes": dbytes,
            "peak_source": f"{hbm_src} (MEASURED_PEAKS.json hbm_gbs)" if hbm_src == "measured" else hbm_src}
    sweeps = info32.sweeps
    step_bytes = step_min_bytes(True, sweeps)
    res = {
        "metric": METRIC,
        "value": value,
        "unit": "solves/s",
        "n_gpus": world,
        "steps": steps,
        "warmup": warmup,
        "ms_per_step": per_step32,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 solve; f64 I/O; double-float pair (~2^-48) rhs/residual/correction",
        "data": "synthetic (seeded two-phase fields, numpy default_rng)",
        "config": {"workload": WORKLOAD, "grid": [NX, NY, NZ], "precision": "fp32+fp64-refine",
                   "refine_tol": 1e-10, "parallelism": "replicas" if world > 1 else "single",
                   "l2": f"inputs {7 * F_BYTES / 1e9:.2f} GB > L2 (no flush needed)" if 7 * F_BYTES > 135e6
                   else "inputs smaller than L2"},
        "gpts_per_s": value * N_CELLS / 1e9,
        "sweeps": sweeps,
        "rel_residual": info32.rel_residual,
        "step_roofline": {"min_pass_bytes": step_bytes, "achieved_GBps": step_bytes / (per_step32 * 1e-3) / 1e9,
                          "frac_of_hbm": step_bytes / (per_step32 * 1e-3) / 1e9 / hbm,
                          "what": f"(21 + 6k)F minimal-pass bytes of the FP32 + refinement form with k = {sweeps} "
                                  "sweep(s), over the step time, over the measured HBM copy peak",
                          "frac_of_hbm_21F": step_min_bytes(False, 0) / (per_step32 * 1e-3) / 1e9 / hbm,
                          "what_21F": "the plain FP64 problem's 21F minimal-pass bytes over the same step time (the "
                                      "effective fraction, comparable with the FP64 form)",
                          "target": 0.60, "target_met": bool(step_bytes / (per_step32 * 1e-3) / 1e9 / hbm >= 0.60)},
        "fp64": {"solves_per_s": world * steps64 / (ms64 * 1e-3) if ms64 else None,
                 "ms_per_step": ms64 / steps64 if ms64 else None,
                 "gpts_per_s": world * steps64 / (ms64 * 1e-3) * N_CELLS / 1e9 if ms64 else None,
                 "step_min_pass_frac_of_hbm": (step_min_bytes(False, 0) / (ms64 / steps64 * 1e-3) / 1e9 / hbm
                                               if ms64 else None),
                 "kernels": kernels64},
        "roofline": roof,
        "kernels": kernels,
        "clocks": clocks,
        "e2e": {"value": world * e_steps / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(sum(v[0] for v in kt32.values()) * steps // max(1, steps)),
        "gpu_launches_note": "kernels per timed region of the headline form (profiled re-run of the same steps)",
        "profiled_ms_per_step": ms32p / steps,
        "per_step": lat32,
        "spectral_schedules": schedules,
    }
    if args.unsplit:
        res["unsplit"] = run_unsplit(plan32, d, out, fl, per_step32, stream)
        res["divergence_constraint"] = run_div_constraint(plan32, dev, stream, hbm)
        from paper_2103_01874_gb300 import split_study
        res["split_study"] = {
            "what": "max over 40 steps of max|p_split - p_exact| / max|p_exact| when the unsplit pressure is "
                    "P(t) = Q cos(omega t) + R sin(omega t) (phi = omega dt per step); exact_history: p^n, p^{n-1} "
                    "exact; 64^3 multimode, FP64 plan",
            "rows": split_study.sweep(n=64)}
    if args.batched:
        res["batched"] = run_batched(args, dev)
    if args.served:
        res["served"] = run_served(args, dev)
    if not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(args)
        res["precision"] = precision_report(fl, d, dev, stream)
    if dist is not None:
        dist.destroy_process_group()
    return res


def precision_report(fl, d, dev, stream):
    """Error of the FP32 solve + pair refinement against the FP64 oracle on the
    bench workload, per refinement sweep: the projection with exactly k sweeps
    (max_sweeps = k, no tolerance; k = 0 is the FP32 solve and the correction
    alone), max |x - x_oracle| / max |x_oracle| for p, u, v, w, and the
    relative residual the refinement test sees.  Part of the CPU-baseline leg
    (the oracle runs once here, about 2 s on one core)."""
    import torch
    from oracle import ppe_oracle as O
    from paper_2103_01874_gb300 import ppe
    ref = O.project_fields(fl)
    c = fl.shape
    rows = []
    for k in range(4):
        o = dict(p=torch.empty(c, dtype=torch.float64, device=dev), u=torch.empty_like(d["u"]),
                 v=torch.empty_like(d["v"]), w=torch.empty_like(d["w"]))
        with ppe.Plan(fl.nx, fl.ny, fl.nz, fl.lx, fl.ly, fl.lz, precision=ppe.FP32_REFINE, refine_tol=0.0,
                      max_sweeps=k, stream=stream) as plan:
            plan.project(d["u"], d["v"], d["w"], d["S"], d["rho"], d["p_n"], d["p_nm1"], fl.dt,
                         o["p"], o["u"], o["v"], o["w"])
            info = plan.info(allow_not_converged=True)
        row = {"sweeps": int(info.sweeps), "rel_residual": float(info.rel_residual)}
        for key in ("p", "u", "v", "w"):
            g = o[key].cpu().numpy()
            row[f"err_{key}"] = float(abs(g - ref[key]).max() / abs(ref[key]).max())
        rows.append(row)
    return {"what": "FP32 solve + k pair-refinement sweeps (no tolerance) vs the FP64 oracle, 256^3 bench "
                    "workload: max-norm error of p, u, v, w relative to the oracle's max, and the relative "
                    "residual of the refinement test", "rows": rows}


# ---------------------------------------------------------------------------
# the unsplit projection (Eqs. (29)-(30)) on the same fields: the baseline the
# split method replaces
# ---------------------------------------------------------------------------
def run_unsplit(plan, d, out, fl, split_ms, stream, reps=3, tol=1e-10):
    import torch

    def once():
        plan.project_unsplit(d["u"], d["v"], d["w"], d["S"], d["rho"], fl.dt, out["p"], out["u"], out["v"], out["w"],
                             tol=tol, max_iter=1000)
    once()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        once()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    it, rel = plan.unsplit_info(allow_not_converged=True)
    return {"what": "variable-coefficient Eq. (30) by conjugate gradients preconditioned with the FP32 FFT solve "
                    f"(Polak-Ribiere), from p = 0 to max|r| <= {tol:g} max|g|, then Eq. (29); same fields",
            "ms_per_solve": ms, "solves_per_s": 1e3 / ms, "iterations": it, "rel_residual": rel,
            "ms_per_iteration": ms / max(it, 1), "split_speedup": ms / split_ms}


def run_div_constraint(plan, dev, stream, hbm, reps=20):
    """Eq. (31) at the bench grid: 6 FP64 inputs and a byte mask in, S and the
    one-fluid density out (65 B per cell)."""
    import torch
    n = (NZ, NY, NX)
    g = torch.Generator(device=dev).manual_seed(7)
    C = torch.rand(n, generator=g, device=dev, dtype=torch.float64)
    ins = [C] + [torch.randn(n, generator=g, device=dev, dtype=torch.float64) for _ in range(3)]
    ins += [50.0 + 80.0 * torch.rand(n, generator=g, device=dev, dtype=torch.float64),
            600.0 + 100.0 * torch.rand(n, generator=g, device=dev, dtype=torch.float64)]
    mask = (torch.rand(n, generator=g, device=dev) < 0.1).to(torch.uint8)
    S = torch.empty_like(C)
    rho = torch.empty_like(C)
    plan.divergence_constraint(*ins, S, rho=rho, under_resolved=mask)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        plan.divergence_constraint(*ins, S, rho=rho, under_resolved=mask)
    e1.record(stream)
    torch.cuda.synchronize()
    us = 1e3 * e0.elapsed_time(e1) / reps
    nbytes = N_CELLS * (6 * 8 + 1 + 2 * 8)
    del ins, S, rho, mask
    return {"what": "Eq. (31): S and the one-fluid density from C, phase compressibilities, mdot, phase densities "
                    "and an under-resolved mask", "us_per_launch": us, "GBps": nbytes / (us * 1e-6) / 1e9,
            "frac_of_hbm": nbytes / (us * 1e-6) / 1e9 / hbm, "bytes_per_launch": nbytes}


# ---------------------------------------------------------------------------
# batched (64 uneven grids in one graph launch) and served (Poisson arrivals)
# ---------------------------------------------------------------------------
def run_batched(args, dev):
    """64 grids, each dimension from {32, 48, 64, 96, 128, 192}, single-interface
    recipe, FP32 solve + FP64 refinement, captured into one CUDA graph; against
    a loop of plain FP64 projections of the same grids, one after another."""
    import torch

    from paper_2103_01874_gb300 import autotune, fields, ppe
    shapes = fields.batch_shapes(64, seed=3)
    items64, items32 = [], []
    for n, (nx, ny, nz) in enumerate(shapes):
        fl = fields.make_fields(nx, ny, nz, seed=200 + n, recipe="single", width=2.0)
        d = {k: torch.from_numpy(v).to(dev) for k, v in fl.arrays().items()}
        for prec, items in ((ppe.FP32_REFINE, items32), (ppe.FP64, items64)):
            plan = ppe.Plan(nx, ny, nz, fl.lx, fl.ly, fl.lz, precision=prec)
            o = dict(d, p=torch.empty(fl.shape, dtype=torch.float64, device=dev), u_out=torch.empty_like(d["u"]),
                     v_out=torch.empty_like(d["v"]), w_out=torch.empty_like(d["w"]), dt=fl.dt)
            items.append((plan, o))
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5

    def time_batch(**opts):
        try:
            batch = ppe.Batch(items32, stream=stream, **opts)
        except ppe.PPEError:
            return None
        for _ in range(2):
            batch.launch()
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(reps):
            batch.launch()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        st = batch.status()
        batch.close()
        if st["status"] != 0:
            raise RuntimeError(f"persistent batch status {st}")
        return e0.elapsed_time(e1) / reps

    # persistent form (one kernel over a device work queue): default queue
    # order, then the batch tuner's search over queue orders and residency
    ms_pers_default = time_batch(form=ppe.BATCH_PERSISTENT)
    t0 = time.perf_counter()
    pers_best, ms_pers, pers_trials = autotune.tune_batch(lambda o: time_batch(form=ppe.BATCH_PERSISTENT, **o))
    pers_tune_s = time.perf_counter() - t0
    with ppe.Batch(items32, stream=stream, form=ppe.BATCH_PERSISTENT, **pers_best) as b:
        b.launch()
        pers_status = b.status()
    worst_pers = max(pl.info(allow_not_converged=True).rel_residual for pl, _ in items32)
    # graph form: default plans, then per-plan autotuned plans (each distinct
    # grid tuned once: spectral schedule by the whole projection's time, then
    # the x-line tile; the others of its size class take the cached result)
    ms_default = time_batch(form=ppe.BATCH_GRAPH)
    defaults = [pl.get_tuning() for pl, _ in items32]
    tuned = tune_plans(items32, {k: autotune.SEARCH[k] for k in ("spectral", "y_solve", "x_lines")}, stream)
    ms_graph = time_batch(form=ppe.BATCH_GRAPH)
    # the per-plan choices were timed on each grid alone: the batch keeps them
    # only if the whole batch runs faster with them
    tuned["kept"] = ms_graph <= ms_default
    if not tuned["kept"]:
        for (pl, _), t in zip(items32, defaults):
            pl.set_tuning(**t)
        ms_graph = ms_default
    worst = max(pl.info(allow_not_converged=True).rel_residual for pl, _ in items32)
    persistent_wins = ms_pers is not None and ms_pers <= ms_graph
    ms_batch = ms_pers if persistent_wins else ms_graph

    def loop64():
        for pl, o in items64:
            pl.set_stream(stream)
            pl.project(o["u"], o["v"], o["w"], o["S"], o["rho"], o["p_n"], o["p_nm1"], o["dt"], o["p"], o["u_out"],
                       o["v_out"], o["w_out"])
    loop64()
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(reps):
        loop64()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_loop = e0.elapsed_time(e1) / reps
    pts = sum(a * b * c for a, b, c in shapes)
    for pl, _ in items32 + items64:
        pl.close()
    return {"workload": "64 uneven grids (dims from {32,48,64,96,128,192}), FP32 solve + pair refinement to 1e-10; "
                        "the faster of the persistent form (one kernel over a device work queue, tuned queue order) "
                        "and the graph form (one graph launch of per-grid branches, autotuned plans)",
            "form": "persistent" if persistent_wins else "graph",
            "solves_per_s": 64 / (ms_batch * 1e-3), "ms_per_batch": ms_batch, "gpts_per_s": pts / (ms_batch * 1e-3) / 1e9,
            "max_rel_residual": max(worst, worst_pers), "cells": pts,
            "persistent": {"solves_per_s": 64 / (ms_pers * 1e-3) if ms_pers else None, "ms_per_batch": ms_pers,
                           "default_ms_per_batch": ms_pers_default, "options": pers_best,
                           "items": pers_status["items"], "ctas": pers_status["ctas"],
                           "tuner_seconds": pers_tune_s, "trials_ms": pers_trials,
                           "max_rel_residual": worst_pers},
            "graph": {"solves_per_s": 64 / (ms_graph * 1e-3), "ms_per_batch": ms_graph,
                      "untuned_ms_per_batch": ms_default, "autotune": tuned},
            "fp64_loop": {"solves_per_s": 64 / (ms_loop * 1e-3), "ms_per_batch": ms_loop}}


def tune_plans(items, search, stream, path=None):
    """Autotune each (plan, fields) item, once per size class: the first plan of
    a class is searched on its own fields, the others take the cached tuning.
    Returns how often each spectral schedule was chosen and the tuning time."""
    import tempfile

    from paper_2103_01874_gb300 import autotune
    path = path or os.path.join(tempfile.mkdtemp(prefix="ppe_tune_"), "tuning.json")
    t0 = time.perf_counter()
    chosen = {}
    for plan, o in items:
        plan.set_stream(stream)
        if not autotune.apply_cached(plan, path):
            def run(k, plan=plan, o=o):
                for _ in range(k):
                    plan.project(o["u"], o["v"], o["w"], o["S"], o["rho"], o["p_n"], o["p_nm1"], o["dt"], o["p"],
                                 o["u_out"], o["v_out"], o["w_out"])
            autotune.autotune(plan, run, reps=2, path=path, search=search)
        t = plan.get_tuning()
        name = {0: "legacy", 1: "fused", 2: "pencil"}[t["spectral"]]
        if t["spectral"] == 0:
            name += "+" + ("tridiagonal" if t["y_solve"] == 1 else "cosine")
        chosen[name] = chosen.get(name, 0) + 1
    return {"search": list(search), "schedules_chosen": chosen, "seconds": time.perf_counter() - t0,
            "cache": path}


def run_served(args, dev):
    """Poisson arrivals (mean 200 req/s) of grids from 64^3 to 384x256x384,
    admitted under a 150 GB budget: the mixed stream (half FP64, half FP32 +
    refinement) and, on the same arrival trace, an all-FP64 stream.  Every
    request projects its own seeded fields (request seed s uses resident set
    s mod 4 of its shape, drawn before the clock starts)."""
    from paper_2103_01874_gb300 import autotune, ppe, serve
    shapes = [(64, 64, 64), (96, 96, 96), (128, 128, 128), (192, 192, 192), (256, 256, 256), (384, 256, 384)]
    probs = [0.3, 0.2, 0.2, 0.15, 0.1, 0.05]
    import tempfile

    import torch
    pool = 4
    cache = os.path.join(tempfile.mkdtemp(prefix="ppe_tune_"), "tuning.json")
    ex = serve.CudaExecutor(slots=8, device=dev.index, pool=pool, autotune_cache=cache)
    ex.prepare(shapes)   # the seeded input sets, resident before the clock starts
    ex.prealloc(shapes)  # per-slot field buffers
    # every size class tuned before the clock (the executor applies the cache to
    # each plan it creates)
    tune_items = []
    for shp in shapes:
        dd, fl = ex.fields_of(shp, 0)
        for prec in (ppe.FP64, ppe.FP32_REFINE):
            plan = ppe.Plan(*shp, fl.lx, fl.ly, fl.lz, precision=prec, refine_tol=1e-10, max_sweeps=8)
            o = dict(dd, p=torch.empty_like(dd["rho"]), u_out=torch.empty_like(dd["u"]),
                     v_out=torch.empty_like(dd["v"]), w_out=torch.empty_like(dd["w"]), dt=fl.dt)
            tune_items.append((plan, o))
    tuned = tune_plans(tune_items, autotune.SEARCH, torch.cuda.current_stream(dev), path=cache)
    for plan, _ in tune_items:
        plan.close()
    del tune_items
    srv = serve.Server(ex, budget_bytes=150 << 30, slots=8)

    def stream(seed, fp32_share):
        return serve.poisson_requests(args.served_requests, rate=200.0, shapes=shapes, probs=probs, seed=seed,
                                      fp32_share=fp32_share, fp64=ppe.FP64, fp32=ppe.FP32_REFINE)

    # steady state: an untimed replay of an arrival trace of the same law (other
    # seed) lets the plan pool grow to what concurrent requests of each size class
    # need, as a long-running server would have it resident
    warm = stream(12, 0.5)
    for r in warm:
        r.rid = -1 - r.rid
    srv.run(warm)
    # and a resident pool of at least 3 plans per size class and precision
    srv.reserve([(s, p) for s in shapes for p in (ppe.FP64, ppe.FP32_REFINE)], per_class=3)
    created_warm = srv.plans_created
    out = {}
    for name, share in (("mixed", 0.5), ("fp64_only", 0.0)):
        reqs = stream(11, share)  # the same arrival times and shapes; only the precisions differ
        before = srv.plans_created
        stats, _ = srv.run(reqs)
        worst = max((r.rel_residual for r in reqs if r.precision == ppe.FP32_REFINE), default=float("nan"))
        d = stats.as_dict()
        d.update(requests=len(reqs), fp32_requests=sum(r.precision == ppe.FP32_REFINE for r in reqs),
                 max_rel_residual_fp32=worst, plans_created=srv.plans_created - before)
        out[name] = d
    srv.close()
    res = dict(out["mixed"])
    res.update(workload="Poisson 200 req/s, grids 64^3..384x256x384, 50% FP64 / 50% FP32+refine, 150 GB budget, "
                        "8 slots; per-request seeded fields (4 resident sets per shape)",
               plans_created_in_warmup=created_warm, fp64_only=out["fp64_only"], autotune=tuned)
    return res


# ---------------------------------------------------------------------------
# CPU oracle (the reference arm / cpu_baseline)
# ---------------------------------------------------------------------------
# The oracle timed: the C++ FP64 projection (oracle/ppe_oracle.cpp, g++ -O3,
# one thread), on the bench's 256^3 fields.
ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
from oracle import cpp
from paper_2103_01874_gb300 import fields
cpp.lib()
fl = fields.multimode_256()
times = []
for s in range({n}):
    t = time.perf_counter()
    cpp.project_fields(fl)
    times.append(time.perf_counter() - t)
print(json.dumps(times))
"""

ORACLE_KIND = "oracle (C++ FP64, own mixed-radix FFT and Thomas y solve, g++ -O3, 1 thread)"
REF_MAX_SOLVES = 3  # about 20 s each on one core


def oracle_times(n: int):
    from oracle import cpp
    cpp.build()  # compiled once here, before the timed processes start
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-c", ORACLE_SNIPPET.format(root=ROOT, n=n)], capture_output=True,
                       text=True, env=env, timeout=1800)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def oracle_all_cores():
    """Secondary CPU figure: one oracle process per host core, all started at
    once; each times one whole 256^3 solve, and the throughput is the sum of the
    per-process rates (about 2 GB of host memory per process)."""
    k = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    procs = [subprocess.Popen([sys.executable, "-c", ORACLE_SNIPPET.format(root=ROOT, n=1)], stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True, env=env) for _ in range(k)]
    rates = []
    for pr in procs:
        out, err = pr.communicate(timeout=1800)
        if pr.returncode != 0:
            raise RuntimeError(err[-2000:])
        rates.append(1.0 / json.loads(out.strip().splitlines()[-1])[0])
    return {"value": sum(rates), "unit": "solves/s", "cores": k, "kind": ORACLE_KIND,
            "sample": f"{k} concurrent processes (one per host core, 1 thread each), one timed 256^3 solve each; "
                      f"per-process {min(rates):.3f}-{max(rates):.3f} solves/s"}


def cpu_baseline(args):
    n = max(1, args.cpu_solves)
    times = oracle_times(n)
    return {"value": n / sum(times), "unit": "solves/s", "cores": 1, "kind": ORACLE_KIND,
            "sample": f"{n} whole 256^3 projection(s), {sum(times):.1f} s of CPU work on one core; "
                      f"best {min(times):.2f} s/solve",
            "all_cores": oracle_all_cores()}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and rank != 0:
        return None
    # bounded sample: at most REF_MAX_SOLVES timed whole 256^3 solves (about
    # 20 s each on one core; the oracle is compiled before the timed process)
    n_timed = max(1, min(args.steps, REF_MAX_SOLVES))
    timed = oracle_times(n_timed)
    total = sum(timed)
    value = len(timed) / total
    return {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": "solves/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * total / len(timed),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (seeded two-phase fields, numpy default_rng)",
        "config": {"workload": WORKLOAD, "grid": [NX, NY, NZ], "precision": "fp64 (oracle)",
                   "parallelism": "single host core"},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": ORACLE_KIND,
                         "sample": f"{len(timed)} whole 256^3 projections timed (of {args.steps} steps asked; "
                                   f"capped at {REF_MAX_SOLVES} so the run ends in about a minute)"},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    import faulthandler
    faulthandler.enable()  # a fatal signal prints the Python stack of every thread
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)  # ~0.45 s timed: several clock samples
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--max-sweeps", type=int, default=8)
    ap.add_argument("--cpu-solves", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n", type=int, default=256, help="grid edge (profiling runs only; the bench line is 256)")
    ap.add_argument("--shape", default=None,
                    help="NX,NY,NZ of a profiling run (overrides --n; the bench line is 256,256,256)")
    ap.add_argument("--forms", default="fp32,fp64", help="fp32 (always) and/or fp64")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-kernel-times", dest="kernel_times", action="store_false")
    ap.add_argument("--no-batched", dest="batched", action="store_false")
    ap.add_argument("--no-served", dest="served", action="store_false")
    ap.add_argument("--no-unsplit", dest="unsplit", action="store_false")
    ap.add_argument("--no-schedules", dest="schedules", action="store_false",
                    help="skip timing the other spectral schedules of the headline plan")
    ap.add_argument("--served-requests", type=int, default=200)
    ap.add_argument("--host-refine", action="store_true",
                    help="drive every timed step with per-kernel events (refinement loop from the host), so that a "
                         "profiler sees each kernel as its own launch")
    args = ap.parse_args()
    if args.shape:
        set_grid(*[int(v) for v in args.shape.split(",")])
    else:
        set_grid(args.n)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        res = run_reference(args)
    else:
        from paper_2103_01874_gb300 import build
        build.build()
        res = run_gpu(args)
    if res is not None:
        print(json.dumps(res))


if __name__ == "__main__":
    main()
