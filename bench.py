#!/usr/bin/env python
"""Benchmark of the level-by-level multigrid Poisson solve (cuRAMSES,
arXiv 2604.06035) on one GB300 per rank.

Workload (default "two_level_128"): periodic 128^3 base level (lognormal
density, sigma_ln rho = 1.5, P(k) ~ k^-2, seed 2) plus one refined level on
the cells above 8 rho_bar (face-dilated, ~1.4 M fine cells).  A step solves
both levels, base then fine (Dirichlet ghosts from the base phi), each from
phi = 0 to relative residual 1e-10, through libcmg.so.  Inputs (keys,
densities) are resident in HBM when the timed region starts; L2 is flushed
(512 MiB write) before every timed step, outside its CUDA-event interval.

metric: cell-updates per second (a cell visited by one full red-black sweep,
summed over all multigrid levels), whole job over all ranks.  With --gpus N
each rank solves its own replica (the level solve is not sharded): "weak".

--impl reference times the CPU FP64 oracle (test infrastructure, single
thread) on a bounded sample of the same workload: one V-cycle of each level.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

FP64_PEAK_TFLOPS = 1.25  # GB300 nominal FP64 (profiling recipe); FMA = 2 flops
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="two_level_128", choices=["two_level_128"])
    ap.add_argument("--quick", action="store_true", help="timed steps only (profiling runs)")
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--learned-traj", type=int, default=128,
                    help="trajectories of 8 steps for the learned warm start (1/16 held out)")
    ap.add_argument("--train-seconds", type=float, default=60.0, help="U-Net training budget")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned warm-start block")
    ap.add_argument("--no-amr3", action="store_true", help="skip the 256^3 + 3-level mixed-precision block")
    ap.add_argument("--block", choices=["smoother", "learned", "forward", "fft", "pcg", "amr3", "batched"], default=None,
                    help="run one sub-benchmark alone and print its JSON (profiling runs)")
    ap.add_argument("--smoother-level", type=int, default=9, help="level of the full periodic grid (9 = 512^3)")
    ap.add_argument("--fft-level", type=int, default=9, help="level of the fft block's full periodic grid")
    ap.add_argument("--fwd-batches", default="1,8", help="batch sizes of --block forward")
    ap.add_argument("--fwd-paths", default="tcgen05,mma_sync", help="kernel paths of --block forward")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers

def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")), int(
        os.environ.get("WORLD_SIZE", "1"))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons every 200 ms while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for name, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def traffic_for(kernel):
    """ncu DRAM bytes per launch recorded in profiles/traffic.json for the
    current kernel source (null when the source changed since the capture)."""
    try:
        rec = json.load(open(PROFILE_TRAFFIC))
    except (OSError, ValueError):
        return None
    e = rec.get(kernel)
    if not e:
        return None
    from paper_2604_06035_gb300 import build as _b
    if e.get("source_sha") != _b.source_digest(tuple(e.get("sources", ())) or None):
        return None
    return e.get("dram_bytes_per_launch")


def aggregate_ranks(dev_ms, updates, world, device=None):
    """Whole-job figures of N replicas (one per rank, each timing its own
    steps): the slowest rank's device time and the cell updates of all ranks,
    by torch.distributed collectives (any backend; one rank: unchanged)."""
    if world <= 1:
        return dev_ms, updates
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(dev_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(updates)], dtype=torch.float64, device=device)
    dist.all_reduce(u)
    return float(t.item()), float(u.item())


def read_peaks():
    """HBM GB/s and dense BF16 TFLOP/s (burst) from MEASURED_PEAKS.json, else
    the profiling recipe's fallback figures."""
    out = {"hbm": 6800.0, "hbm_src": "fallback", "bf16": 1900.0, "bf16_src": "fallback"}
    try:
        rec = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return out
    if "hbm_gbs" in rec:
        out["hbm"], out["hbm_src"] = float(rec["hbm_gbs"]), "measured"
    if "bf16_tflops" in rec:
        out["bf16"], out["bf16_src"] = float(rec["bf16_tflops"]), "measured (burst)"
    return out


def cycle_updates(n_octs_per_mg, n_pre=2, n_post=2, coarse_sweeps=4, exact_coarse=True):
    u = sum((n_pre + n_post) * 8 * n for n in n_octs_per_mg[:-1])
    if not exact_coarse:
        u += coarse_sweeps * 8 * n_octs_per_mg[-1]
    return u


# ------------------------------------------------------------- reference

def two_level_workload(n_fine_octs, tol):
    """The `config.workload` text of the two-level benchmark (both arms)."""
    return ("two_level_128: 128^3 periodic lognormal base (sigma 1.5, k^-2) + 1 refined level "
            "(rho > 8 rho_bar, %d fine octs); FP64 V(2,2) to rel. residual %g per level" % (n_fine_octs, tol))


def run_reference(args, rank, world):
    import numpy as np  # noqa: F401
    import oracle as O
    from paper_2604_06035_gb300 import inputs
    if rank != 0:
        return
    cfg = inputs.two_level_amr(base_level=7, seed=2)
    B = O.Level(7, O.morton_encode(cfg["coords"][0]))
    F = O.Level(8, O.morton_encode(cfg["coords"][1]), parent=B)
    B.set_density(cfg["rho"][0], 1.0)
    F.set_density(cfg["rho"][1], 1.0)
    ub = cycle_updates([B.mg_n_octs(m) for m in range(B.mg_depth)], exact_coarse=True)
    uf = cycle_updates([F.mg_n_octs(m) for m in range(F.mg_depth)], exact_coarse=False)

    def step():
        B.solve(fixed_cycles=1)
        F.solve(fixed_cycles=1)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    value = (ub + uf) / dt / 1e6
    sample = "one FP64 V(2,2) cycle on the 128^3 base and one on the refined level per step"
    print(json.dumps({
        "metric": "poisson_cell_updates_per_s", "value": value, "unit": "Mcell-updates/s", "impl": "reference",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": two_level_workload(F.n, args.tol), "l2": "not applicable (CPU oracle)",
                   "parallelism": "single"},
        "cpu_baseline": {"value": value, "unit": "Mcell-updates/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "Mcell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def cpu_baseline_sample():
    """The oracle as it stands on a bounded sample: two V-cycles of each level
    of the same workload, single thread."""
    import oracle as O
    from paper_2604_06035_gb300 import inputs
    cfg = inputs.two_level_amr(base_level=7, seed=2)
    B = O.Level(7, O.morton_encode(cfg["coords"][0]))
    F = O.Level(8, O.morton_encode(cfg["coords"][1]), parent=B)
    B.set_density(cfg["rho"][0], 1.0)
    F.set_density(cfg["rho"][1], 1.0)
    ub = cycle_updates([B.mg_n_octs(m) for m in range(B.mg_depth)], exact_coarse=True)
    uf = cycle_updates([F.mg_n_octs(m) for m in range(F.mg_depth)], exact_coarse=False)
    t0 = time.perf_counter()
    B.solve(fixed_cycles=2)
    F.solve(fixed_cycles=2)
    dt = time.perf_counter() - t0
    return {"value": 2 * (ub + uf) / dt / 1e6, "unit": "Mcell-updates/s", "cores": 1, "kind": "oracle",
            "sample": "two FP64 V(2,2) cycles on the 128^3 base and two on the refined level (%.1f s)" % dt}


# ------------------------------------------------------------------- ours

def bench_batched(cmg, ctx, dev, stream, args):
    """512 independent refined patches (log-uniform 64..200000 octs, level 11,
    Dirichlet values from a smooth coarse field): one persistent cooperative
    kernel per solve.  Autotunes the schedule, then times mixed-precision and
    FP64 solves from phi = 0 to rel. residual tol on every patch, as V-cycle
    iterations and as per-patch CG preconditioned by them."""
    import torch
    from paper_2604_06035_gb300 import inputs
    t0 = time.perf_counter()
    b = inputs.batched_patches(n_patches=512, seed=4)
    gen_s = time.perf_counter() - t0
    lev = b["level"]
    P = cmg.cmg_level_build(ctx, lev - 1, cmg.cmg_morton_encode(ctx, torch.from_numpy(b["parent_coords"]).to(dev)))
    cmg.cmg_level_set_phi(P, torch.from_numpy(b["parent_phi"]).to(dev))
    keys = cmg.cmg_morton_encode(ctx, torch.from_numpy(b["coords"]).to(dev))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    F = cmg.cmg_level_build(ctx, lev, keys, parent=P)
    B = cmg.cmg_batch_create(F, b["offsets"])
    torch.cuda.synchronize()
    build_ms = (time.perf_counter() - t0) * 1e3
    cmg.cmg_level_set_density(F, torch.from_numpy(b["rho"]).to(dev), 1.0)
    zeros = torch.zeros((len(b["coords"]), 8), dtype=torch.float64, device=dev)
    cmg.cmg_level_set_phi(F, zeros)
    t0 = time.perf_counter()
    best, best_ms = cmg.cmg_batch_autotune(B, tol=args.tol, precision=cmg.CMG_PREC_MIXED)
    tune_s = time.perf_counter() - t0
    res = {"patches": 512, "octs": int(len(b["coords"])), "cells": int(8 * len(b["coords"])),
           "level": lev, "schedule": best, "autotune_s": tune_s, "build_ms": build_ms, "generate_s": gen_s}
    reps = max(3, min(args.steps, 5))
    for name, prec, kr in (("mixed", cmg.CMG_PREC_MIXED, 0), ("fp64", cmg.CMG_PREC_FP64, 0),
                           ("mixed_pcg", cmg.CMG_PREC_MIXED, 1), ("fp64_pcg", cmg.CMG_PREC_FP64, 1)):
        cmg.cmg_level_set_phi(F, zeros)
        cmg.cmg_batch_solve(B, tol=args.tol, precision=prec, krylov=kr)  # records the graph
        ms, upd = [], 0
        for _ in range(reps):
            cmg.cmg_level_set_phi(F, zeros)
            torch.cuda.synchronize()
            rc, st = cmg.cmg_batch_solve(B, tol=args.tol, precision=prec, krylov=kr)
            ms.append(st["ms"])
            upd += st["cell_updates"]
        res[name] = {"ms_per_solve": statistics.median(ms), "Mcell_updates_per_s": upd / (sum(ms) / 1e3) / 1e6,
                     "cycles": st["cycles"], "rel_max": st["rel_max"], "n_converged": st["n_converged"],
                     "grid_barriers": st["grid_barriers"], "status": rc}
    cmg.cmg_batch_destroy(B)
    cmg.cmg_level_destroy(F)
    cmg.cmg_level_destroy(P)
    del zeros
    torch.cuda.empty_cache()
    return res


def bench_smoother(cmg, ctx, dev, peaks, lev=9, sweeps=10):
    """The smoother and residual kernels alone on a full periodic 512^3 level
    (16.8 M octs; every field far larger than L2): per-launch CUDA events on
    the library stream, algorithmic bytes per launch (FP32: 3 x 4 cells x 4 B
    per oct and colour; the neighbour indices are not counted) against the
    measured HBM copy rate."""
    import torch
    from paper_2604_06035_gb300 import inputs
    coords = torch.from_numpy(inputs.uniform_oct_coords(lev)).to(dev)
    L = cmg.cmg_level_build(ctx, lev, cmg.cmg_morton_encode(ctx, coords))
    del coords
    n = cmg.cmg_level_n_octs(L)
    g = torch.Generator(device=dev)
    g.manual_seed(7)
    rho = torch.rand((n, 8), dtype=torch.float64, device=dev, generator=g) + 0.5
    cmg.cmg_level_set_density(L, rho, float(rho.mean().item()))
    del rho
    cmg.cmg_level_set_phi(L, torch.zeros((n, 8), dtype=torch.float64, device=dev))
    res = {"grid": "%d^3 periodic (%d octs)" % (1 << lev, n), "sweeps": sweeps}
    for name, prec in (("fp32", cmg.CMG_PREC_MIXED), ("fp64", cmg.CMG_PREC_FP64)):
        cmg.cmg_level_mg_step(L, 0, cmg.CMG_OP_SWEEP, prec, 2)
        cmg.cmg_ctx_reset_profile(ctx)
        cmg.cmg_ctx_set_profiling(ctx, True)
        cmg.cmg_level_mg_step(L, 0, cmg.CMG_OP_SWEEP, prec, sweeps)
        cmg.cmg_level_mg_step(L, 0, cmg.CMG_OP_RESIDUAL, prec)
        cmg.cmg_ctx_set_profiling(ctx, False)
        prof = cmg.cmg_ctx_get_profile(ctx)
        for fam in ("rbgs_" + name, "residual_" + name):
            d = prof[fam]
            gbs = d["bytes"] / (d["ms"] / 1e3) / 1e9
            res[fam] = {"launches": d["launches"], "ms_per_launch": d["ms"] / d["launches"],
                        "bytes_per_launch": d["bytes"] / d["launches"], "achieved_GBs": gbs,
                        "frac_of_hbm": gbs / peaks["hbm"], "hbm_source": peaks["hbm_src"],
                        "TFLOPs": d["flops"] / (d["ms"] / 1e3) / 1e12, "traffic": traffic_for(fam + "_512")}
    cmg.cmg_level_destroy(L)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return res


def bench_fft(cmg, ctx, dev, B, rho_b, args, peaks):
    """Time to rel. residual tol of full periodic levels by the FFT solve
    (FP32 FFT inside FP64 refinement) against FP64 and mixed multigrid: the
    two-level workload's 128^3 base, and a 512^3 level (rho uniform in
    [0.5, 1.5), seed 7)."""
    import torch
    from paper_2604_06035_gb300 import inputs

    def time_level(L, rho, reps=5):
        out = {}
        n = cmg.cmg_level_n_octs(L)
        z = torch.zeros((n, 8), dtype=torch.float64, device=dev)
        cmg.cmg_level_set_density(L, rho, float(rho.mean().item()))
        for name, prec in (("fp64", cmg.CMG_PREC_FP64), ("mixed", cmg.CMG_PREC_MIXED), ("fft", cmg.CMG_PREC_FFT)):
            ms, st = [], None
            for _ in range(reps + 1):
                cmg.cmg_level_set_phi(L, z)
                rc, st = cmg.cmg_level_solve(L, tol=args.tol, precision=prec)
                ms.append(st["ms"])
            out[name] = {"ms_to_tol": statistics.median(ms[1:]), "steps": st["cycles"], "rel_final": st["rel_final"]}
        cmg.cmg_ctx_reset_profile(ctx)
        cmg.cmg_ctx_set_profiling(ctx, True)
        cmg.cmg_level_set_phi(L, z)
        cmg.cmg_level_solve(L, tol=args.tol, precision=cmg.CMG_PREC_FFT)
        cmg.cmg_ctx_set_profiling(ctx, False)
        f = cmg.cmg_ctx_get_profile(ctx)["fft_fp32"]
        gbs = f["bytes"] / (f["ms"] / 1e3) / 1e9
        n = cmg.cmg_level_n_octs(L)
        out["fft_kernels"] = {"launches": f["launches"], "ms": f["ms"], "achieved_GBs": gbs,
                              "frac_of_hbm": gbs / peaks["hbm"], "hbm_source": peaks["hbm_src"],
                              "bytes_per_launch": f["bytes"] / f["launches"],
                              "traffic": traffic_for("fft_fp32_%d" % round((8 * n) ** (1 / 3)))}
        out["speedup_fft_vs_fp64"] = out["fp64"]["ms_to_tol"] / out["fft"]["ms_to_tol"]
        return out

    res = {"base_128": time_level(B, rho_b)}
    lev = getattr(args, "fft_level", 9)
    coords = torch.from_numpy(inputs.uniform_oct_coords(lev)).to(dev)
    L = cmg.cmg_level_build(ctx, lev, cmg.cmg_morton_encode(ctx, coords))
    del coords
    g = torch.Generator(device=dev)
    g.manual_seed(7)
    rho = torch.rand((cmg.cmg_level_n_octs(L), 8), dtype=torch.float64, device=dev, generator=g) + 0.5
    res["periodic_%d" % (1 << lev)] = time_level(L, rho, reps=3)
    del rho
    cmg.cmg_level_destroy(L)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return res


def bench_pcg(cmg, ctx, dev, levels, args):
    """Time to rel. residual tol of the two-level workload's levels from
    phi = 0: the stationary V-cycle iteration against V-cycle-preconditioned
    CG, in FP64 and in mixed precision (FP32 V-cycles), each one CUDA graph
    with the stop test on the device."""
    import torch
    out = {}
    for name, L, rho in levels:
        z = torch.zeros_like(rho)
        cmg.cmg_level_set_density(L, rho, 1.0)
        r = {}
        for kind, kr, prec in (("vcycle", 0, cmg.CMG_PREC_FP64), ("pcg", 1, cmg.CMG_PREC_FP64),
                               ("mixed", 0, cmg.CMG_PREC_MIXED), ("pcg_mixed", 1, cmg.CMG_PREC_MIXED)):
            ms = []
            for _ in range(6):
                cmg.cmg_level_set_phi(L, z)
                rc, st = cmg.cmg_level_solve(L, tol=args.tol, krylov=kr, precision=prec)
                ms.append(st["ms"])
            r[kind] = {"ms_to_tol": statistics.median(ms[1:]), "iterations": st["cycles"],
                       "rel_final": st["rel_final"]}
            # the same solve launch by launch, for the per-kernel-family split
            cmg.cmg_level_set_phi(L, z)
            cmg.cmg_ctx_reset_profile(ctx)
            cmg.cmg_ctx_set_profiling(ctx, True)
            cmg.cmg_level_solve(L, tol=args.tol, krylov=kr, precision=prec)
            cmg.cmg_ctx_set_profiling(ctx, False)
            r[kind]["kernel_ms"] = {k: round(v["ms"], 4) for k, v in cmg.cmg_ctx_get_profile(ctx).items()
                                    if v["launches"]}
        out[name] = r
    return out


def bench_amr3(cmg, ctx, dev, args):
    """The 256^3 mixed-precision workload: periodic lognormal base (sigma 2)
    plus three levels refined where rho > 8 rho_bar, solved level by level
    (each after its parent, whose phi gives the coarse-fine values) from phi = 0
    to rel. residual tol: FP64 V-cycles, FP32 V-cycles inside FP64 refinement,
    and the FFT solve of the base under mixed fine levels; phi of the mixed
    chain against the FP64 one."""
    import torch
    from paper_2604_06035_gb300 import inputs
    t0 = time.perf_counter()
    cfg = inputs.mixed_amr()
    gen_s = time.perf_counter() - t0
    levels, parent = [], None
    for lev, c, r in zip(cfg["levels"], cfg["coords"], cfg["rho"]):
        L = cmg.cmg_level_build(ctx, lev, cmg.cmg_morton_encode(ctx, torch.from_numpy(c).to(dev)), parent=parent)
        rho = torch.from_numpy(r).to(dev)
        cmg.cmg_level_set_density(L, rho, cfg["rho_bar"])
        levels.append((lev, L, rho))
        parent = L
    out = {"workload": "256^3 periodic lognormal base (sigma 2, k^-2) + 3 levels refined at rho > 8 rho_bar",
           "levels": cfg["levels"], "octs": [len(c) for c in cfg["coords"]],
           "cells": int(sum(8 * len(c) for c in cfg["coords"])), "generate_s": gen_s, "tol": args.tol}

    def chain(precs, reps=5):
        per = [[] for _ in levels]
        stats = [None] * len(levels)
        for _ in range(reps):
            for k, (lev, L, rho) in enumerate(levels):
                cmg.cmg_level_set_phi(L, torch.zeros_like(rho))
                rc, st = cmg.cmg_level_solve(L, tol=args.tol, precision=precs[k])
                per[k].append(st["ms"])
                stats[k] = st
        ms = [statistics.median(p[1:]) for p in per]
        upd = sum(st["cell_updates"] for st in stats)
        return {"ms_to_tol_per_level": ms, "ms_total": sum(ms),
                "iterations": [st["cycles"] for st in stats], "rel_final": [st["rel_final"] for st in stats],
                "Mcell_updates_per_s": upd / (sum(ms) / 1e3) / 1e6}

    F64, MIX, FFT = cmg.CMG_PREC_FP64, cmg.CMG_PREC_MIXED, cmg.CMG_PREC_FFT
    out["fp64"] = chain([F64] * len(levels))
    phi64 = [cmg.cmg_level_get_phi(L, device=True).clone() for _, L, _ in levels]
    out["mixed"] = chain([MIX] * len(levels))
    err = []
    for (lev, L, rho), p64 in zip(levels, phi64):
        p = cmg.cmg_level_get_phi(L, device=True)
        err.append(float((p - p64).abs().max() / p64.abs().max()))
    out["mixed"]["phi_rel_err_vs_fp64"] = err
    # the precision effect alone: both chains refined to 1e-12 (untimed)
    tight = []
    for precs in ([F64] * len(levels), [MIX] * len(levels)):
        got = []
        for k, (lev, L, rho) in enumerate(levels):
            cmg.cmg_level_set_phi(L, torch.zeros_like(rho))
            cmg.cmg_level_solve(L, tol=1e-12, precision=precs[k])
            got.append(cmg.cmg_level_get_phi(L, device=True).clone())
        tight.append(got)
    out["mixed"]["phi_rel_err_vs_fp64_both_at_1e-12"] = [
        float((b - a).abs().max() / a.abs().max()) for a, b in zip(*tight)]
    out["fft_base_mixed_fine"] = chain([FFT] + [MIX] * (len(levels) - 1))
    out["speedup_mixed_vs_fp64"] = out["fp64"]["ms_total"] / out["mixed"]["ms_total"]
    out["speedup_fft_mixed_vs_fp64"] = out["fp64"]["ms_total"] / out["fft_base_mixed_fine"]["ms_total"]
    for _, L, _ in reversed(levels):
        cmg.cmg_level_destroy(L)
    return out


def bench_forward(cmg, ctx, dev, peaks, D=64, batches=(1, 8), reps=20, paths=("tcgen05", "mma_sync")):
    """The U-Net forward alone on random inputs (untrained He-normal weights):
    device time per call and the convolutions' tensor-core rate."""
    import torch
    from paper_2604_06035_gb300 import warmstart as W
    g = torch.Generator(device=dev)
    g.manual_seed(3)
    net = cmg.cmg_unet_create(ctx, D, max(batches))
    cmg.cmg_unet_set_params(net, W.init_params(5, zero_head=False))
    res = {"grid": "%d^3" % D}
    for B in batches:
        rho = torch.rand((B, D, D, D), device=dev, generator=g) + 0.5
        field = torch.randn((B, D, D, D), device=dev, generator=g)
        for path, name in ((1, "tcgen05"), (0, "mma_sync")):
            if name not in paths:
                continue
            cmg.cmg_unet_set_kernels(net, path)
            for _ in range(3):
                cmg.cmg_unet_forward(net, rho, field)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            for _ in range(reps):
                cmg.cmg_unet_forward(net, rho, field)
            b.record()
            torch.cuda.synchronize()
            cmg.cmg_ctx_reset_profile(ctx)
            cmg.cmg_ctx_set_profiling(ctx, True)
            for _ in range(reps):
                cmg.cmg_unet_forward(net, rho, field)
            torch.cuda.synchronize()
            cmg.cmg_ctx_set_profiling(ctx, False)
            conv = cmg.cmg_ctx_get_profile(ctx)["conv_fwd"]
            tf = conv["flops"] / (conv["ms"] / 1e3) / 1e12
            target = field + 0.01 * torch.randn((B, D, D, D), device=dev, generator=g)
            for _ in range(2):
                cmg.cmg_unet_gradients(net, rho, field, target, grads=False)
            torch.cuda.synchronize()
            a2, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a2.record()
            for _ in range(5):
                cmg.cmg_unet_gradients(net, rho, field, target, grads=False)
            b2.record()
            torch.cuda.synchronize()
            res["b%d_%s" % (B, name)] = {"ms_per_forward": a.elapsed_time(b) / reps,
                                         "conv_ms_per_forward": conv["ms"] / reps, "conv_TFLOPs": tf,
                                         "conv_frac_of_bf16": tf / peaks["bf16"],
                                         "ms_per_training_step": a2.elapsed_time(b2) / 5}
    cmg.cmg_unet_set_kernels(net, 1)
    cmg.cmg_unet_destroy(net)
    return res


def bench_learned(cmg, ctx, dev, args, peaks):
    """Learned warm start on 64^3 periodic blocks: dataset from the FP64
    solver (lognormal trajectories), U-Net training with the library's BF16
    kernels for a fixed wall-clock budget, then on held-out trajectories the
    V-cycles and device time to rel. residual tol from phi_prev and from the
    network's prediction (FP64 and mixed precision), the warm start's own
    cost, and the forward convolutions' tensor-core rate."""
    import numpy as np
    import torch
    from paper_2604_06035_gb300 import warmstart as W
    D, n_steps = 64, 8
    n_traj = args.learned_traj
    n_test = max(2, n_traj // 16)
    t0 = time.perf_counter()
    data = W.build_dataset(ctx, n_traj=n_traj, n_steps=n_steps, D=D, seed=5)
    gen_s = time.perf_counter() - t0
    net = cmg.cmg_unet_create(ctx, D, 8)
    # delta = 0 at the start: the untrained network returns phi_prev
    cmg.cmg_unet_set_params(net, W.init_params(12))
    train_trajs = list(range(n_traj - n_test))
    test_trajs = list(range(n_traj - n_test, n_traj))
    t0 = time.perf_counter()
    losses = W.train(net, data, train_trajs, batch=4, lr=2e-3, seconds=args.train_seconds)
    train_s = time.perf_counter() - t0
    res = {"grid": "%d^3 periodic" % D, "pairs_train": len(train_trajs) * n_steps,
           "pairs_test": len(test_trajs) * n_steps, "dataset_s": gen_s, "train_s": train_s,
           "epochs": len(losses), "loss_first_epoch": losses[0], "loss_last_epoch": losses[-1],
           "output_scale": cmg.cmg_unet_get_output_scale(net)}
    for name, prec in (("fp64", cmg.CMG_PREC_FP64), ("mixed", cmg.CMG_PREC_MIXED)):
        W.evaluate(ctx, net, data, test_trajs[:1], tol=args.tol, precision=prec)  # warm the graphs
        m, _ = W.evaluate(ctx, net, data, test_trajs, tol=args.tol, precision=prec)
        res[name] = {k: m[k] for k in ("cycles_prev", "cycles_net", "cycles_zero", "ms_prev", "ms_net", "ms_zero",
                                       "rel_final_net", "err_prev", "err_net")}
    # the warm start's cost: residual of phi_prev + forward (batch 1), and the
    # forward alone, on device inputs
    S = W.PeriodicSolver(ctx, D)
    k, t = test_trajs[0], 0
    rho, prev = data["rho"][k, t + 1], data["phi"][k, t]
    r = data["res"][k, t][None].contiguous()
    rho1, prev1 = rho[None].contiguous(), prev[None].contiguous()

    def ev_time(fn, reps=20):
        for _ in range(3):
            fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    res["ms_warm_start_b1_python"] = ev_time(lambda: W.predict(S, net, rho, prev))
    res["ms_forward_b1"] = ev_time(lambda: cmg.cmg_unet_forward(net, rho1, r, base=prev1))
    rho8 = data["rho"][k, 1:9].contiguous()
    r8 = data["res"][k, 0:8].contiguous()
    prev8 = data["phi"][k, 0:8].contiguous()
    res["ms_forward_per_block_b8"] = ev_time(lambda: cmg.cmg_unet_forward(net, rho8, r8, base=prev8)) / 8
    # the residual of phi_prev on the level (density and phi are set for the
    # solve anyway): the residual kernel and the oct -> dense copy
    S._load(rho, prev)
    dense = torch.empty((D, D, D), dtype=torch.float64, device=dev)

    def residual_only():
        cmg.cmg_level_get_residual(S.level, device=True, out=S.octs)
        cmg.cmg_dense_octs(ctx, S.octs, D, dense, 0)
    res["ms_residual_per_block"] = ev_time(residual_only)
    res["ms_warm_start_per_block_b8"] = res["ms_forward_per_block_b8"] + res["ms_residual_per_block"]
    cmg.cmg_ctx_reset_profile(ctx)
    cmg.cmg_ctx_set_profiling(ctx, True)
    for _ in range(5):
        cmg.cmg_unet_forward(net, rho8, r8, base=prev8)
    torch.cuda.synchronize()
    cmg.cmg_ctx_set_profiling(ctx, False)
    conv = cmg.cmg_ctx_get_profile(ctx)["conv_fwd"]
    tf = conv["flops"] / (conv["ms"] / 1e3) / 1e12
    res["roofline_conv_fwd"] = {"bound": "tensor", "achieved": tf, "peak": peaks["bf16"], "unit": "TFLOP/s",
                                "frac": tf / peaks["bf16"], "peak_source": peaks["bf16_src"],
                                "launches": conv["launches"], "ms": conv["ms"],
                                "flops_per_block": conv["flops"] / (5 * 8),
                                "traffic": traffic_for("conv_fwd_b8"), "traffic_unit": "DRAM bytes per launch"}
    f, m = res["fp64"], res["mixed"]
    ws = res["ms_warm_start_per_block_b8"]
    res["summary"] = {
        "warm_start_ms_per_block": ws, "fp64_ms_zero": f["ms_zero"], "fp64_ms_prev": f["ms_prev"],
        "fp64_ms_net_plus_warm_start": f["ms_net"] + ws,
        "mixed_ms_prev": m["ms_prev"], "mixed_ms_net_plus_warm_start": m["ms_net"] + ws,
        "cycles_saved_fp64": f["cycles_prev"] - f["cycles_net"]}
    del S, net
    del data
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return res


def run_ours(args, rank, local, world):
    import numpy as np
    import torch

    import __graft_entry__ as ge
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if local == 0:
        ge.build()
    if world > 1:
        dist.barrier()
    from paper_2604_06035_gb300 import cmg, inputs

    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    ctx = cmg.cmg_ctx_create(local, stream=stream.cuda_stream)
    cfg = inputs.two_level_amr(base_level=7, seed=2)
    coords = [torch.from_numpy(c).to(dev) for c in cfg["coords"]]
    rho = [torch.from_numpy(r).to(dev) for r in cfg["rho"]]
    zeros = [torch.zeros_like(r) for r in rho]

    # setup: keys (a1), hash + neighbour cache + hierarchy (a2, a3), ghost stencils
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    keys = [cmg.cmg_morton_encode(ctx, c) for c in coords]
    B = cmg.cmg_level_build(ctx, 7, keys[0])
    F = cmg.cmg_level_build(ctx, 8, keys[1], parent=B)
    torch.cuda.synchronize()
    build_ms = (time.perf_counter() - t0) * 1e3

    def step(precision=cmg.CMG_PREC_FP64):
        # both levels' inputs, both solves queued (the fine level's coarse-fine
        # values read the base phi in stream order), then both reports
        for L, r, z in ((B, rho[0], zeros[0]), (F, rho[1], zeros[1])):
            cmg.cmg_level_set_phi(L, z)
            cmg.cmg_level_set_density(L, r, 1.0)
        for L in (B, F):
            cmg.cmg_level_solve_async(L, tol=args.tol, precision=precision)
        return [cmg.cmg_level_solve_wait(L)[1] for L in (B, F)]

    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        step()

    def timed(profile):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        cmg.cmg_ctx_reset_profile(ctx)
        cmg.cmg_ctx_set_profiling(ctx, profile)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        stats = []
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            ev[k][0].record(stream)
            stats.append(step())
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        cmg.cmg_ctx_set_profiling(ctx, False)
        return stats, sum(a.elapsed_time(b) for a, b in ev), cmg.cmg_ctx_launch_count(ctx)

    # timed region: the solve graphs as a user runs them (no per-launch events)
    sampler = ClockSampler(local)
    sampler.start()
    all_stats, dev_ms, launches = timed(False)
    clocks = sampler.stop()
    # the same steps again, kernel by kernel with CUDA events on the library's
    # stream, for the per-kernel-family rates of the roofline
    _, prof_ms, _ = timed(True)
    prof = cmg.cmg_ctx_get_profile(ctx)
    updates = sum(s["cell_updates"] for st in all_stats for s in st)
    t_max, upd_total = aggregate_ranks(dev_ms, updates, world, dev)
    value = upd_total / (t_max / 1e3) / 1e6
    st_b, st_f = all_stats[-1]

    # dominant kernel family of the timed region and its roofline
    dom = max(prof.items(), key=lambda kv: kv[1]["ms"])
    dname, d = dom
    achieved_tflops = d["flops"] / (d["ms"] / 1e3) / 1e12
    achieved_gbs = d["bytes"] / (d["ms"] / 1e3) / 1e9
    peaks = read_peaks()
    hbm, hbm_src = peaks["hbm"], peaks["hbm_src"]
    fp64 = dname.endswith("fp64")
    if fp64:
        # the sweep issues 6 FP64-pipe instructions (5 DADD + 1 DFMA = 7 flop)
        # per cell update against 2 per SM per clock: 7/12 of the nominal
        # flop rate is the pipe's ceiling for this instruction mix
        pipe_ops = achieved_tflops * 1e12 * 6.0 / 7.0
        roofline = {"bound": "alu", "achieved": achieved_tflops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved_tflops / FP64_PEAK_TFLOPS, "kernel": dname,
                    "peak_source": "GB300 nominal FP64 1.25 TFLOP/s (FMA = 2)",
                    "fp64_pipe_frac": pipe_ops / (FP64_PEAK_TFLOPS * 1e12 / 2.0),
                    "fp64_pipe_note": "6 FP64 instructions per cell update vs 2 per SM per clock (nominal)",
                    "hbm_equivalent_gbs": achieved_gbs, "hbm_frac_of_%s" % hbm_src: achieved_gbs / hbm}
    else:
        roofline = {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm, "unit": "GB/s",
                    "frac": achieved_gbs / hbm, "kernel": dname, "peak_source": hbm_src}
    roofline["traffic"] = traffic_for(dname)
    roofline["launches"] = d["launches"]
    roofline["share_of_kernel_ms"] = d["ms"] / sum(v["ms"] for v in prof.values())
    roofline["timing"] = ("per-launch CUDA events on the library stream over a repeat of the timed steps "
                          "launched kernel by kernel (%.2f ms/step there)" % (prof_ms / args.steps))

    out = {
        "metric": "poisson_cell_updates_per_s", "value": value, "unit": "Mcell-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": two_level_workload(cmg.cmg_level_n_octs(F), args.tol),
                   "l2": "flushed before each timed step (512 MiB write)", "parallelism": "replicas" if world > 1
                   else "single"},
        "time_to_tol_ms": {"base": st_b["ms"], "fine": st_f["ms"]},
        "cycles": {"base": st_b["cycles"], "fine": st_f["cycles"]},
        "rel_residual": {"base": st_b["rel_final"], "fine": st_f["rel_final"]},
        "setup_ms": build_ms,
        "roofline": roofline,
        "kernels": {k: {"launches": v["launches"], "ms": v["ms"], "GB/s": v["bytes"] / v["ms"] / 1e6,
                        "TFLOP/s": v["flops"] / v["ms"] / 1e9} for k, v in prof.items()},
        "gpu_launches": launches,
        "clocks": clocks,
    }

    if not args.quick:
        # mixed precision on the same workload (FP32 V-cycles, FP64 refinement)
        for _ in range(2):
            step(cmg.CMG_PREC_MIXED)
        mixed_ms, mixed_upd = 0.0, 0
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sm = step(cmg.CMG_PREC_MIXED)
            b.record(stream)
            torch.cuda.synchronize()
            mixed_ms += a.elapsed_time(b)
            mixed_upd += sum(s["cell_updates"] for s in sm)
        phi_mixed_f = cmg.cmg_level_get_phi(F)
        cmg.cmg_ctx_reset_profile(ctx)
        cmg.cmg_ctx_set_profiling(ctx, True)
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            step(cmg.CMG_PREC_MIXED)
        torch.cuda.synchronize()
        cmg.cmg_ctx_set_profiling(ctx, False)
        mprof = cmg.cmg_ctx_get_profile(ctx)
        sw = mprof.get("rbgs_fp32")
        mixed_roof = None
        if sw and sw["ms"] > 0:
            gbs = sw["bytes"] / (sw["ms"] / 1e3) / 1e9
            mixed_roof = {"bound": "hbm", "kernel": "rbgs_fp32", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                          "frac": gbs / hbm, "peak_source": hbm_src, "launches": sw["launches"],
                          "share_of_kernel_ms": sw["ms"] / sum(v["ms"] for v in mprof.values()),
                          "traffic": traffic_for("rbgs_fp32")}
        step()
        phi_fp64_f = cmg.cmg_level_get_phi(F)
        out["mixed"] = {"ms_per_step": mixed_ms / args.steps,
                        "Mcell_updates_per_s": mixed_upd / (mixed_ms / 1e3) / 1e6,
                        "time_to_tol_ms": {"base": sm[0]["ms"], "fine": sm[1]["ms"]},
                        "refinement_steps": {"base": sm[0]["cycles"], "fine": sm[1]["cycles"]},
                        "phi_rel_diff_vs_fp64_gpu": float(np.max(np.abs(phi_mixed_f - phi_fp64_f)) /
                                                          np.max(np.abs(phi_fp64_f))),
                        "roofline_smoother": mixed_roof,
                        "kernels": {k: {"launches": v["launches"], "ms": v["ms"],
                                        "GB/s": v["bytes"] / v["ms"] / 1e6 if v["ms"] else None}
                                    for k, v in mprof.items()}}

        # end to end through the C ABI with host buffers (pinned): H2D densities,
        # both solves, D2H of both phi arrays
        pin_rho = [torch.from_numpy(r).pin_memory().numpy() for r in cfg["rho"]]
        pin_phi = [torch.empty((cmg.cmg_level_n_octs(L), 8), dtype=torch.float64).pin_memory().numpy()
                   for L in (B, F)]
        e2e_ms, e2e_upd = 0.0, 0
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            # per level: upload (overlapping the parent's queued solve), solve,
            # queued read-back (overlapping the next level's solve)
            for L, r, z, o in zip((B, F), pin_rho, zeros, pin_phi):
                cmg.cmg_level_set_phi(L, z)  # zero initial guess, already on the device
                cmg.cmg_level_set_density(L, r, 1.0)
                cmg.cmg_level_solve_async(L, tol=args.tol)
                cmg.cmg_level_get_phi_async(L, out=o)
            for L in (B, F):
                rc, st = cmg.cmg_level_solve_wait(L)
                e2e_upd += st["cell_updates"]
            cmg.cmg_ctx_synchronize(ctx)
            e2e_ms += (time.perf_counter() - t0) * 1e3
        h2d = sum(r.nbytes for r in pin_rho)
        d2h = sum(o.nbytes for o in pin_phi)
        out["e2e"] = {"value": e2e_upd * world / (e2e_ms / 1e3) / 1e6, "unit": "Mcell-updates/s",
                      "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms / args.steps}
        out["batched"] = bench_batched(cmg, ctx, dev, stream, args)
        out["smoother_512"] = bench_smoother(cmg, ctx, dev, peaks)
        out["fft"] = bench_fft(cmg, ctx, dev, B, rho[0], args, peaks)
        out["pcg"] = bench_pcg(cmg, ctx, dev, (("base", B, rho[0]), ("fine", F, rho[1])), args)
        if not args.no_amr3:
            out["amr3_256"] = bench_amr3(cmg, ctx, dev, args)
        if not args.no_learned:
            out["learned"] = bench_learned(cmg, ctx, dev, args, peaks)
        if rank == 0 and world == 1:
            out["cpu_baseline"] = cpu_baseline_sample()
    else:
        out["e2e"] = None
    if rank == 0:
        print(json.dumps(out), flush=True)
    torch.cuda.synchronize()
    cmg.cmg_level_destroy(F)
    cmg.cmg_level_destroy(B)
    cmg.cmg_ctx_destroy(ctx)
    if world > 1:
        dist.destroy_process_group()


def run_block(args):
    """One sub-benchmark alone on cuda:0 (for profiler captures)."""
    import torch

    import __graft_entry__ as ge
    ge.build()
    from paper_2604_06035_gb300 import cmg
    dev = torch.device("cuda", 0)
    ctx = cmg.cmg_ctx_create(0, stream=torch.cuda.current_stream(dev).cuda_stream)
    peaks = read_peaks()
    if args.block == "smoother":
        out = bench_smoother(cmg, ctx, dev, peaks, lev=args.smoother_level)
    elif args.block == "fft":
        from paper_2604_06035_gb300 import inputs
        cfg = inputs.two_level_amr(base_level=7, seed=2)
        B = cmg.cmg_level_build(ctx, 7, cmg.cmg_morton_encode(ctx, torch.from_numpy(cfg["coords"][0]).to(dev)))
        out = bench_fft(cmg, ctx, dev, B, torch.from_numpy(cfg["rho"][0]).to(dev), args, peaks)
        cmg.cmg_level_destroy(B)
    elif args.block == "batched":
        out = bench_batched(cmg, ctx, dev, torch.cuda.current_stream(dev), args)
    elif args.block == "amr3":
        out = bench_amr3(cmg, ctx, dev, args)
    elif args.block == "pcg":
        from paper_2604_06035_gb300 import inputs
        cfg = inputs.two_level_amr(base_level=7, seed=2)
        cs = [torch.from_numpy(c).to(dev) for c in cfg["coords"]]
        rs = [torch.from_numpy(r).to(dev) for r in cfg["rho"]]
        B = cmg.cmg_level_build(ctx, 7, cmg.cmg_morton_encode(ctx, cs[0]))
        F = cmg.cmg_level_build(ctx, 8, cmg.cmg_morton_encode(ctx, cs[1]), parent=B)
        out = bench_pcg(cmg, ctx, dev, (("base", B, rs[0]), ("fine", F, rs[1])), args)
        cmg.cmg_level_destroy(F)
        cmg.cmg_level_destroy(B)
    elif args.block == "forward":
        out = bench_forward(cmg, ctx, dev, peaks, batches=[int(b) for b in args.fwd_batches.split(",")],
                            paths=args.fwd_paths.split(","))
    else:
        out = bench_learned(cmg, ctx, dev, args, peaks)
    print(json.dumps({"block": args.block, **out}), flush=True)
    torch.cuda.synchronize()
    cmg.cmg_ctx_destroy(ctx)


def main():
    args = parse()
    rank, local, world = dist_env()
    if args.block is not None and args.impl == "ours":
        run_block(args)
    elif args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, local, world)


if __name__ == "__main__":
    main()
