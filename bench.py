#!/usr/bin/env python3
"""Benchmark of one CheFSI step (Algorithm 1 of arXiv 2302.09708) on GB300.

Workload (default): the 96^3 periodic bulk system, h = 0.4 bohr, 216 atoms on a
jittered simple-cubic lattice, Ns = 1300 orbitals, Chebyshev degree 20, FP64,
seeded synthetic inputs (Gaussian Veff, Gaussian x real-Y_lm KB projectors,
orthonormal random X0).  A "step" is one full CheFSI pass: filter, Yt = H Xt,
projection, subspace eigensolve, rotation, with library-chosen bounds (cached
Lanczos, cut-off = previous largest Ritz value).  The orbital block (9.2 GB)
is far larger than L2, so no flush is needed between steps.

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CheFSI step time & Hpsi GB/s; mixed-FP32/batched vs FP64 speedup at <=1e-6 Ha"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# DRAM bytes (read + write) per orbital of one ring-stencil launch of a filter
# degree on the 96^3 bulk grid, from ncu captures at Ns = 64 scaled by orbitals
# (every orbital is one independent pass over the grid): FP64 (1006.27 +
# 417.48) MB / 64, FP32 (491.28 + 189.31) MB / 64 (the ring-kernel captures),
# each of the thread shape named beside it (the roofline's traffic is null
# when the tuner picked another shape)
RING64_DRAM_BYTES_PER_ORBITAL = (1006.271e6 + 417.475e6) / 64
RING64_CAPTURED_SHAPE = 0
RING32_DRAM_BYTES_PER_ORBITAL = (491.276e6 + 189.307e6) / 64
RING32_CAPTURED_SHAPE = 0
RING_CAPTURED_ND = 96 ** 3  # the grid of both captures
# FLOP per point and orbital of one H application (finite-difference stencil,
# Veff and recurrence), the count the roofline of the FP64 stencil uses
STENCIL_FLOP_PER_POINT = 84
FP64_FLOP_PER_SM_CLK = 4  # 2 FP64 FMA per SM per clock


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="bulk96",
                   help="bulk96 (96^3 bulk, Ns 1300), bulk24 (24^3, Ns 40), member36 (36^3, "
                        "Ns 150: one system of the batched set's size range) or slab64x64x160")
    p.add_argument("--no-mixed", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-batch", action="store_true")
    p.add_argument("--no-slab", action="store_true",
                   help="skip the 64x64x160 slab leg (mixed precision, Ns 4800)")
    p.add_argument("--batch-systems", type=int, default=64)
    p.add_argument("--variants", default="all",
                   help="comma-separated forms to compare with the headline FP64 path, or all")
    p.add_argument("--cpu-seconds", type=float, default=20.0)
    p.add_argument("--ns", type=int, default=0, help="override Ns (profiling on a smaller case)")
    p.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                   help="precision of the timed (headline) run")
    return p.parse_args()


def peaks():
    try:
        return json.load(open(PEAKS_FILE))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, dev):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------------------
# CPU oracle sample (baseline and reference arm)
# --------------------------------------------------------------------------
def oracle_sample(system, ns, degree, budget_s):
    """Time the CPU oracle on a bounded sample of one CheFSI step and
    extrapolate to the full step by each stage's scaling in Ns (filter and
    H Xt ~ Ns, projection and rotation ~ Ns^2, eigensolve ~ Ns^3)."""
    import numpy as np

    import oracle
    from paper_2302_09708_gb300 import synth

    cores = len(os.sched_getaffinity(0))
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    o = oracle.Oracle(system)
    nd = system.nd
    t0 = time.perf_counter()
    a0, b, *_ = o.lanczos(8, 0)
    a = a0 + 0.1 * (b - a0)
    # filter + one H application on `cores` columns (one per thread), scaled by
    # the number of such column batches in Ns
    deg_s = max(1, min(degree, int(budget_s)))  # keep the sample bounded
    nc = cores
    Xs = synth.random_orbitals(nd, nc, seed=1)
    t = time.perf_counter()
    o.cheb_filter(Xs, deg_s, a, b, a0)
    t_deg = (time.perf_counter() - t) / deg_s
    batches = math.ceil(ns / nc)
    t_filter = t_deg * (degree + 1) * batches
    # projection and rotation on a 64-column panel
    p = min(64, ns)
    Xp = np.random.default_rng(2).standard_normal((p, nd))
    t = time.perf_counter()
    oracle.project(Xp, Xp, nd)
    t_proj = (time.perf_counter() - t) * (ns / p) ** 2
    Zp = np.random.default_rng(3).standard_normal((p, p))
    t = time.perf_counter()
    oracle.rotate(Xp, Zp, nd)
    t_rot = (time.perf_counter() - t) * (ns / p) ** 2
    q = min(ns, 200)
    A = np.random.default_rng(4).standard_normal((q, q))
    M = A @ A.T + q * np.eye(q)
    t = time.perf_counter()
    oracle.gen_eig(0.5 * (A + A.T), M)
    t_eig = (time.perf_counter() - t) * (ns / q) ** 3
    total = t_filter + t_proj + t_rot + t_eig
    sample = (f"oracle on {cores} host cores: {deg_s} filter degrees on {nc} of {ns} columns "
              f"(scaled x{degree + 1}/{deg_s} x{batches}), projection and rotation on a {p}-column "
              f"panel (scaled x(Ns/{p})^2), eigensolve at Ns={q} (scaled x(Ns/{q})^3)")
    return {"step_s": total, "cores": cores, "sample": sample,
            "parts_s": {"filter_hx": t_filter, "project": t_proj, "rotate": t_rot,
                        "eig": t_eig}, "wall_s": time.perf_counter() - t0}


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    from paper_2302_09708_gb300 import synth

    cfg = synth.WORKLOADS[args.workload]
    system = synth.make_workload_system(args.workload)
    ns, m = cfg["ns"], cfg["degree"]
    budget = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    times = []
    last = None
    for i in range(args.warmup + args.steps):
        r = oracle_sample(system, ns, m, budget)
        if i >= args.warmup:
            times.append(r["step_s"])
        last = r
    step_s = statistics.mean(times) if times else last["step_s"]
    value = 1.0 / step_s
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": step_s * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": cfg["name"], "precision": "fp64", "l2": "inputs > L2"},
        "cpu_baseline": {"value": value, "unit": "steps/s", "cores": last["cores"],
                         "kind": "oracle", "sample": last["sample"]},
        "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------
def main():
    args = parse()
    world, rank, local = dist_init(args)
    if args.impl == "reference":
        return run_reference(args, world, rank)

    import numpy as np
    import torch

    from paper_2302_09708_gb300 import sparc, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sparc.load()
    cfg = synth.WORKLOADS[args.workload]
    system = synth.make_workload_system(args.workload)
    ns, m = (args.ns or cfg["ns"]), cfg["degree"]
    nd = system.nd
    seed = synth.workload_seed(args.workload) + rank
    t_setup = time.perf_counter()
    X0 = synth.random_orbitals(nd, ns, seed=seed)
    setup_s = time.perf_counter() - t_setup
    stream = torch.cuda.current_stream(dev)

    # ---- headline run (FP64 unless --precision mixed) ------------------
    prec = args.precision
    h = sparc.Handle(system, prec, ns_max=ns, device=local)
    Xd = torch.from_numpy(X0).to(dev, torch.float64 if prec == "fp64" else torch.float32)
    ne = synth.electrons_for(ns)
    lam_d = torch.empty(ns, dtype=torch.float64, device=dev)
    dens_ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def full_step():
        """Algorithm 1 (bounds, filter, H Xt, projection, eigensolve, rotation),
        then Fermi-Dirac occupations and the density of the new orbitals."""
        h.chefsi_step(Xd, m, eig=lam_d)
        dens_ev[0].record(stream)
        occ, _mu = h.occupations(lam_d, ne, 0.01)
        rho = h.density(Xd, occ)
        dens_ev[1].record(stream)
        return rho

    for _ in range(args.warmup):
        full_step()
    torch.cuda.synchronize(dev)
    barrier(world)
    stage = []
    dens_ms = []
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            rho = full_step()
            stage.append(h.timings())
            dens_ev[1].synchronize()
            dens_ms.append(dens_ev[0].elapsed_time(dens_ev[1]))
        e1.record(stream)
        torch.cuda.synchronize(dev)
    rho_electrons = float(rho.sum()) * system.h ** 3
    tuning = h.tuning()
    barrier(world)
    t_loc = e0.elapsed_time(e1) / 1e3
    t_max = max_over_ranks(t_loc, world, dev)
    value = world * args.steps / t_max
    # the step's own launches plus k_fermi and k_density (+ reduce when split)
    launches = int(sum(s["launches"] for s in stage)) + 2 * args.steps

    def med(key):
        return statistics.median(s[key] for s in stage)

    s_bytes = 8 if prec == "fp64" else 4
    st_ms = {k: med(k) for k in ("bounds_ms", "filter_ms", "hx_ms", "project_ms", "eig_ms",
                                 "rotate_ms", "total_ms")}
    # filtering throughput: per degree reads Y_i, Y_{i-1}, writes Y_{i+1}
    # (first degree: read X, write Y_1) -> (2 + 3 (m - 1)) Nd Ns s bytes
    filt_bytes = (2 + 3 * (m - 1)) * nd * ns * s_bytes
    hx_bytes = 2 * nd * ns * s_bytes
    filt_gbs = filt_bytes / (st_ms["filter_ms"] / 1e3) / 1e9
    hx_gbs = hx_bytes / (st_ms["hx_ms"] / 1e3) / 1e9
    proj_flops = 2.0 * nd * ns * ns  # Hs and Ms as symmetric halves
    rot_flops = 2.0 * nd * ns * ns
    stage_rate = {
        "filter": {"ms": st_ms["filter_ms"], "GB/s": filt_gbs},
        "hx": {"ms": st_ms["hx_ms"], "GB/s": hx_gbs},
        "project": {"ms": st_ms["project_ms"],
                    "TFLOP/s": proj_flops / (st_ms["project_ms"] / 1e3) / 1e12},
        "eig": {"ms": st_ms["eig_ms"]},
        "occupations_density": {"ms": statistics.median(dens_ms),
                                "GB/s": nd * ns * s_bytes / (statistics.median(dens_ms) / 1e3)
                                / 1e9, "electrons": rho_electrons, "ne": ne},
        "rotate": {"ms": st_ms["rotate_ms"],
                   "TFLOP/s": rot_flops / (st_ms["rotate_ms"] / 1e3) / 1e12},
    }
    # roofline of the dominant kernel: the ring stencil of the filter (timed per
    # launch by the library's events), against the FP64 pipe (FP64 arithmetic)
    # or HBM (FP32)
    pk = peaks()
    roof = stencil_roofline(stage, nd, ns, prec, pk, dev, tuning)
    roof["filter_stage_share"] = st_ms["filter_ms"] / st_ms["total_ms"]

    clocks = clk.summary()

    # ---- e2e through host buffers ----------------------------------------
    e2e = None
    if not args.no_e2e and prec == "fp64":
        # the headline handle takes a page-locked host block: the call a user
        # makes with data in host memory
        Xh = torch.empty((ns, nd), dtype=torch.float64, pin_memory=True)
        Xn = Xh.numpy()
        Xn[:] = X0
        he = h
        he.chefsi_step(Xn, m)  # warm (staging buffer)
        Xn[:] = X0
        ke = max(1, min(args.steps, 2))
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        for _ in range(ke):
            he.chefsi_step(Xn, m)
        te = time.perf_counter() - t
        te = max_over_ranks(te, world, dev)
        tl = he.timings()
        e2e = {"value": world * ke / te, "unit": "steps/s",
               "h2d_bytes_per_step": nd * ns * 8, "d2h_bytes_per_step": nd * ns * 8 + ns * 8,
               "host_buffer": "torch pinned (cudaHostAlloc)",
               "last_step_ms": {"h2d": round(tl["stage_in_ms"], 1),
                                "device": round(tl["total_ms"] - tl["stage_in_ms"], 1),
                                "d2h": round(tl["stage_out_ms"], 1),
                                "host_wall": round(tl["host_ms"], 1)}}
        del Xh, Xn

    # ---- other forms on the same system (mixed precision first) --------------
    variants = None
    if not args.no_mixed and prec == "fp64":
        try:
            variants = run_variants(system, X0, ns, m, args, dev, stream, h)
        except Exception as exc:  # report, do not hide
            variants = {"error": repr(exc)}
    h.close()
    mixed = variants.get("mixed") if isinstance(variants, dict) else None
    if isinstance(mixed, dict) and "ms_per_step" in mixed:
        mixed["speedup_vs_fp64"] = (t_max / args.steps * 1e3) / mixed["ms_per_step"]

    batched = None
    if not args.no_batch and world == 1 and args.batch_systems > 0:
        try:
            batched = run_batched(args, dev, stream)
        except Exception as exc:  # report, do not hide
            batched = {"error": repr(exc)}

    slab = None
    if not args.no_slab and world == 1 and args.workload == "bulk96":
        try:
            slab = run_slab(args, dev, stream)
        except Exception as exc:  # report, do not hide
            slab = {"error": repr(exc)}

    cpu = None
    if rank == 0 and not args.no_cpu and world == 1:
        r = oracle_sample(system, ns, m, args.cpu_seconds)
        cpu = {"value": 1.0 / r["step_s"], "unit": "steps/s", "cores": r["cores"],
               "kind": "oracle", "sample": r["sample"], "extrapolated_step_s": r["step_s"],
               "parts_s": r["parts_s"]}

    line = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == "fp64" else "f32",
        "data": "synthetic",
        "config": {"workload": cfg["name"] + (f" (Ns overridden to {ns})" if args.ns else ""),
                   "precision": prec, "grid": list(system.shape),
                   "h": system.h, "natoms": system.natoms, "ns": ns, "degree": m,
                   "l2": (f"inputs larger than L2 ({nd * ns * s_bytes / 1e9:.1f} GB block)"
                          if nd * ns * s_bytes > 2 * 129e6 else
                          "inputs fit in L2 (small workload; no flush)"),
                   "bounds": "library: 32-step Lanczos run once per handle before the timed "
                             "steps and cached (outside the timed region); cut-off = previous "
                             "largest Ritz value",
                   "projection_rotation": ("six-digit BF16 tcgen05 split, FP32-pair sums, "
                                           "FP64-accurate to ~2^-45 of sum |x_k y_k|"
                                           if prec == "fp64" else
                                           "four-digit BF16 tcgen05 split (mixed precision)"),
                   "parallelism": f"replicas x{world}"},
        "stages": stage_rate,
        "hpsi_gbs": hx_gbs,
        "roofline": roof,
        "stencil_tuning": tuning,
        "gpu_launches": launches,
        "clocks": clocks,
        "e2e": e2e,
        "mixed": mixed,
        "variants": {k: v for k, v in variants.items() if k != "mixed"} if isinstance(variants, dict) else variants,
        "batched": batched,
        "slab": slab,
        "cpu_baseline": cpu,
        "setup_s": setup_s,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def fp64_peak_tflops(pk, dev):
    """FP64 pipe peak derived from the SM count and the maximum SM clock."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = pk.get("sm_max_mhz", 2070.0)
    return sms * FP64_FLOP_PER_SM_CLK * mhz * 1e6 / 1e12, (
        f"derived: {sms} SMs x {FP64_FLOP_PER_SM_CLK} FP64 FLOP/clk x {mhz:.0f} MHz "
        "(FP64 pipe; no measured FP64 peak exists)")


def stencil_roofline(stage, nd, ns, prec, pk, dev, tuning=None):
    """Roofline object of the ring stencil: achieved = algorithmic work of one
    launch / its average duration (library events over the timed steps).  FP64:
    84 Nd Ns FLOP per launch against the FP64 pipe; FP32: 12 Nd Ns bytes (read
    Y_i and Y_(i-1), write Y_(i+1)) against measured HBM.  traffic: the ncu
    DRAM bytes per orbital x Ns, only for the grid and thread shape they were
    captured on (else null)."""
    runs = [s for s in stage if s.get("stencil_launches", 0) > 0]
    if not runs:
        return {"kernel": "generic stencil (no ring launches)", "achieved": None, "frac": None}
    per_launch_ms = statistics.median(s["stencil_ms"] / s["stencil_launches"] for s in runs)
    nl_ms = statistics.median(s["nonlocal_ms"] / s["stencil_launches"] for s in runs)
    shape = tuning.get("shape") if tuning else None

    def captured(per_orbital, shape_captured):
        return bool(per_orbital) and nd == RING_CAPTURED_ND and shape == shape_captured
    if prec == "fp64":
        flop = STENCIL_FLOP_PER_POINT * nd * ns
        peak, src = fp64_peak_tflops(pk, dev)
        ach = flop / (per_launch_ms / 1e3) / 1e12
        traffic = (RING64_DRAM_BYTES_PER_ORBITAL * ns
                   if captured(RING64_DRAM_BYTES_PER_ORBITAL, RING64_CAPTURED_SHAPE) else None)
        return {"kernel": "k_apply_h_ring<double> (local stencil, one filter degree)",
                "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "peak_source": src, "traffic": traffic,
                "algorithmic_flop": flop, "algorithmic_bytes": 24 * nd * ns,
                "launch_ms": per_launch_ms, "nonlocal_pass_ms": nl_ms,
                "achieved_gbs": 24 * nd * ns / (per_launch_ms / 1e3) / 1e9}
    byts = 12 * nd * ns
    peak = pk.get("hbm_gbs", 6688.8)
    ach = byts / (per_launch_ms / 1e3) / 1e9
    traffic = (RING32_DRAM_BYTES_PER_ORBITAL * ns
               if captured(RING32_DRAM_BYTES_PER_ORBITAL, RING32_CAPTURED_SHAPE) else None)
    return {"kernel": "k_apply_h_ring<float> (local stencil, one filter degree)",
            "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)", "traffic": traffic,
            "algorithmic_bytes": byts, "launch_ms": per_launch_ms, "nonlocal_pass_ms": nl_ms}


def fermi_occupied(lam, ne, kT=0.01):
    """States with Fermi-Dirac occupation above 1e-6 at the electron count ne
    (mu by bisection), the set on which the mixed-precision target is read."""
    import numpy as np
    lo, hi = float(lam.min()) - 1.0, float(lam.max()) + 1.0
    for _ in range(200):
        mu = 0.5 * (lo + hi)
        c = 2.0 * np.sum(1.0 / (1.0 + np.exp(np.clip((lam - mu) / kT, -700, 700))))
        lo, hi = (mu, hi) if c < ne else (lo, mu)
    f = 1.0 / (1.0 + np.exp(np.clip((lam - mu) / kT, -700, 700)))
    return f > 1e-6


VARIANTS = (
    ("mixed", "mixed", 0,
     "FP32 orbitals and filtering, FP64 Yt (double-FP32 stencil), four-digit tensor-core GEMMs"),
    ("fp64_double_fp32_stencil", "fp64", 4,
     "FP64 blocks, H x in double-FP32 arithmetic (options bit 2), six-digit tensor-core GEMMs"),
    ("fp64_simt_gemm", "fp64", 2,
     "FP64 blocks, FP64 arithmetic throughout: FP64 stencil and FP64 SIMT GEMMs (options bit 1)"),
)


def run_variants(system, X0, ns, m, args, dev, stream, h64):
    """Other forms of the step on the same system: Ritz values against the
    headline FP64 path from the same start and bounds (3 steps), then the time
    per step.  The headline path is checked against the oracle by the tests."""
    import numpy as np
    import torch

    from paper_2302_09708_gb300 import sparc, synth

    a0, b = h64.spectrum_bounds(32, 0)
    nsteps = 3
    X64 = torch.from_numpy(X0).to(dev)
    a = a0 + 0.1 * (b - a0)
    ref, cut = [], []
    for _ in range(nsteps):
        cut.append(a)
        lam = h64.chefsi_step(X64, m, bounds=(a, b, a0))
        ref.append(lam)
        a = float(lam[-1])
    ne = synth.electrons_for(ns)
    # density of the FP64 path after the same steps (the reference of the
    # variants' density error at this size, where the CPU oracle is too slow)
    f64, _ = h64.occupations(torch.from_numpy(ref[-1]).to(dev), ne, 0.01)
    rho_ref = h64.density(X64, f64).clone()
    del X64
    torch.cuda.empty_cache()
    occ = fermi_occupied(ref[-1], ne)
    out = {"note": "Ritz-value and density differences vs the headline FP64 GPU path from the "
                   "same start and bounds after 3 steps; occupied = Fermi-Dirac f > 1e-6 at "
                   "kT = 0.01 Ha"}
    for key, prec, flags, what in VARIANTS:
        if args.variants != "all" and key not in args.variants.split(","):
            continue
        try:
            hv = sparc.Handle(system, prec, ns_max=ns, device=dev.index, options_flags=flags)
            Xv = torch.from_numpy(X0).to(dev, torch.float32 if prec == "mixed" else torch.float64)
            errs = []
            for s_ in range(nsteps):
                lam = hv.chefsi_step(Xv, m, bounds=(cut[s_], b, a0))
                errs.append(float(np.max(np.abs(lam - ref[s_]))))
            err_occ = float(np.max(np.abs(lam - ref[-1])[occ]))
            fv, _ = hv.occupations(torch.from_numpy(lam).to(dev), ne, 0.01)
            rho = hv.density(Xv, fv)
            dens_l1 = float((rho - rho_ref).abs().sum()) * system.h ** 3 / ne
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            stage = []
            for _ in range(args.steps):
                hv.chefsi_step(Xv, m)
                stage.append(hv.timings())
            e1.record(stream)
            torch.cuda.synchronize(dev)
            t = e0.elapsed_time(e1) / 1e3 / args.steps
            st = {k: statistics.median(x[k] for x in stage) for k in stage[0] if k != "launches"}
            es = 4 if prec == "mixed" else 8
            filt_bytes = (2 + 3 * (m - 1)) * system.nd * ns * es
            out[key] = {"what": what, "ms_per_step": t * 1e3, "stage_ms": st,
                        "filter_GBps": filt_bytes / (st["filter_ms"] / 1e3) / 1e9,
                        "roofline": stencil_roofline(stage, system.nd, ns, prec, peaks(), dev,
                                                     hv.tuning()),
                        "stencil_tuning": hv.tuning(),
                        "ritz_err_vs_fp64_gpu_per_step": errs, "ritz_err_occupied": err_occ,
                        "density_l1_per_electron_vs_fp64_gpu": dens_l1}
            hv.close()
            del Xv
            torch.cuda.empty_cache()
        except Exception as exc:  # report, do not hide
            out[key] = {"error": repr(exc)}
    return out


def run_slab(args, dev, stream):
    """The 64 x 64 x 160 slab (periodic x, y; Dirichlet z; h = 0.35; 600 atoms
    in the central 60 % of z; Ns = 4800, degree 24) in mixed precision: time per
    step and its stages, from a seeded random start drawn on the device (no
    host orthonormalisation at this size: the step's Rayleigh-Ritz makes the
    block orthonormal), library bounds, one warm-up and two timed steps."""
    import torch

    from paper_2302_09708_gb300 import sparc, synth

    cfg = synth.WORKLOADS["slab64x64x160"]
    t0 = time.perf_counter()
    system = synth.make_workload_system("slab64x64x160")
    ns, m = cfg["ns"], cfg["degree"]
    h = sparc.Handle(system, "mixed", ns_max=ns, device=dev.index)
    g = torch.Generator(device=dev).manual_seed(synth.workload_seed("slab64x64x160"))
    X = torch.randn((ns, system.nd), generator=g, device=dev, dtype=torch.float32)
    X /= system.nd ** 0.5
    setup_s = time.perf_counter() - t0
    h.chefsi_step(X, m)
    stage = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    steps = 2
    for _ in range(steps):
        h.chefsi_step(X, m)
        stage.append(h.timings())
    e1.record(stream)
    torch.cuda.synchronize(dev)
    t = e0.elapsed_time(e1) / steps
    st = {k: statistics.median(x[k] for x in stage) for k in stage[0]
          if k not in ("launches", "stencil_launches")}
    filt_bytes = (2 + 3 * (m - 1)) * system.nd * ns * 4
    out = {"workload": cfg["name"], "ms_per_step": t, "steps": steps, "stage_ms": st,
           "filter_GBps": filt_bytes / (st["filter_ms"] / 1e3) / 1e9,
           "roofline": stencil_roofline(stage, system.nd, ns, "mixed", peaks(), dev,
                                        h.tuning()),
           "stencil_tuning": h.tuning(), "setup_s": setup_s,
           "start": "seeded torch.randn on the device / sqrt(Nd)"}
    h.close()
    del X
    torch.cuda.empty_cache()
    return out


def run_batched(args, dev, stream):
    """Batched form on 64 uneven small systems (N^3 grids, N in 24..48, 4-40
    atoms, Ns 40-300, degree 16-24, fixed bounds per member): time per batched step (member
    chains on concurrent streams and one batched eigensolve, replayed CUDA graph) against the same
    members stepped one after another through sparc_chefsi_step, in FP64 and
    mixed precision, with the largest Ritz-value difference between the two."""
    import numpy as np
    import torch

    from paper_2302_09708_gb300 import sparc, synth

    members = synth.batch_members(args.batch_systems)
    t0 = time.perf_counter()
    systems = [synth.random_system(mb["shape"], mb["h"], mb["bc"], mb["natoms"], seed=mb["seed"])
               for mb in members]
    X0 = [synth.random_orbitals(s.nd, mb["ns"], seed=mb["seed"] + 7)
          for s, mb in zip(systems, members)]
    setup_s = time.perf_counter() - t0
    degrees = [mb["degree"] for mb in members]
    out = {"systems": len(members), "setup_s": setup_s,
           "nd_range": [min(s.nd for s in systems), max(s.nd for s in systems)],
           "ns_range": [min(mb["ns"] for mb in members), max(mb["ns"] for mb in members)]}
    steps = max(2, args.steps)
    for prec, dt in (("fp64", torch.float64), ("mixed", torch.float32)):
        handles = [sparc.Handle(s, prec, ns_max=mb["ns"], device=dev.index)
                   for s, mb in zip(systems, members)]
        bounds = []  # fixed (a, b, a0) per member, the same for both forms
        for hh in handles:
            a0, b = hh.spectrum_bounds(32, 0)
            bounds.append((a0 + 0.1 * (b - a0), b, a0))
        Xb = [torch.from_numpy(x).to(dev, dt) for x in X0]
        Xs = [x.clone() for x in Xb]
        batch = sparc.Batch(handles)
        for _ in range(2):  # capture, then replay
            lam_b = batch.chefsi_step(Xb, degrees, bounds=bounds)
        for hh, x, d, bd in zip(handles, Xs, degrees, bounds):
            hh.chefsi_step(x, d, bounds=bd)
            hh.chefsi_step(x, d, bounds=bd)
        torch.cuda.synchronize(dev)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e[0].record(stream)
        for _ in range(steps):
            lam_b = batch.chefsi_step(Xb, degrees, bounds=bounds)
        e[1].record(stream)
        e[2].record(stream)
        for _ in range(steps):
            lam_s = [hh.chefsi_step(x, d, bounds=bd)
                     for hh, x, d, bd in zip(handles, Xs, degrees, bounds)]
        e[3].record(stream)
        torch.cuda.synchronize(dev)
        tb = e[0].elapsed_time(e[1]) / steps
        ts = e[2].elapsed_time(e[3]) / steps
        diff = max(float(np.max(np.abs(a - b))) for a, b in zip(lam_b, lam_s))
        seq_launches = sum(hh.timings()["launches"] for hh in handles)
        out[prec] = {"batched_ms_per_step": tb, "sequential_ms_per_step": ts,
                     "speedup": ts / tb, "launches_batched": batch.launches(),
                     "launches_sequential": int(seq_launches),
                     "max_ritz_diff_batched_vs_sequential": diff}
        batch.close()
        for hh in handles:
            hh.close()
        del Xb, Xs
        torch.cuda.empty_cache()
    out["mixed_vs_fp64_batched_speedup"] = (out["fp64"]["batched_ms_per_step"]
                                            / out["mixed"]["batched_ms_per_step"])
    return out


if __name__ == "__main__":
    sys.exit(main())
