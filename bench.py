#!/usr/bin/env python
"""Benchmark of the level-by-level multigrid Poisson solve (cuRAMSES,
arXiv 2604.06035) on one GB300 per rank.

Workload (default "amr3_256"): the periodic 256^3 base level (lognormal
density, sigma_ln rho = 2, P(k) ~ k^-2, seed 3) plus three levels refined
where rho > 8 rho_bar (face-dilated, properly nested): 2.10 M, 1.75 M,
0.94 M and 1.64 M octs, 51.5 M cells.  A step solves the four levels in FP64,
level by level (each after its parent, whose phi gives the coarse-fine
Dirichlet values), each from phi = 0 to relative residual 1e-10, through
libcmg.so.  Inputs (keys, densities) are resident in HBM when the timed
region starts; every level's fields are far larger than L2, and L2 is also
flushed (512 MiB write) before every timed step, outside its event interval.

metric: cell-updates per second (a cell visited by one full red-black sweep,
summed over all multigrid levels), whole job over all ranks.  With --gpus N
each rank solves its own replica (the level solve is not sharded): "weak".

Extra blocks: the same workload in mixed precision and with the FFT base
solve, the 128^3 two-level workload, the 32^3 periodic workload, 512 batched
patches, the smoother alone on 512^3, FFT and CG comparisons, the learned warm
start, and phi against the FP64 oracle for every workload (outside the timed
region).

cpu_baseline / --impl reference: the CPU FP64 oracle (test infrastructure)
as it stands, on the host cores (OpenMP over its per-oct loops, bit-identical
to one thread), on bounded samples of the same workload.
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

PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="amr3_256", choices=["amr3_256"])
    ap.add_argument("--quick", action="store_true", help="timed steps only: no e2e, extra blocks or CPU baseline "
                                                          "(profiling runs)")
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--learned-traj", type=int, default=256,
                    help="trajectories of 8 steps for the learned warm start (1/16 held out)")
    ap.add_argument("--train-seconds", type=float, default=60.0, help="U-Net training budget")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned warm-start block")
    ap.add_argument("--no-extra", action="store_true", help="headline, e2e and cpu_baseline only")
    ap.add_argument("--no-oracle-errors", action="store_true", help="skip the phi-vs-oracle block")
    ap.add_argument("--block", choices=["smoother", "learned", "forward", "fft", "pcg", "amr3", "batched", "two_level",
                                        "periodic32", "oracle_errors"], default=None,
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


def vcycle_bytes(mg_octs, elem, n_sweeps, coarse_sweeps=None):
    """Algorithmic HBM bytes of one V-cycle over a hierarchy of mg_octs octs
    per level, with perfect reuse: a sweep reads the other colour and g and
    writes its own colour (3 values) plus 3 B of neighbour index per cell; the
    residual + restriction reads phi and g, 3 B of index, writes 1/8 of a
    value; the prolongation reads 1/8 of a value and rewrites phi (2 values).
    The coarsest level gets coarse_sweeps sweeps (default n_sweeps)."""
    total = 0.0
    last = len(mg_octs) - 1
    for m, nm in enumerate(mg_octs):
        cells = 8.0 * nm
        sw = n_sweeps if m < last or coarse_sweeps is None else coarse_sweeps
        total += sw * cells * (3 * elem + 3)
        if m < last:
            total += cells * (2 * elem + 3 + elem / 8.0) + cells * (2 * elem + elem / 8.0)
    return total


def cycle_updates(n_octs_per_mg, n_pre=2, n_post=2, coarse_sweeps=4, exact_coarse=True):
    u = sum((n_pre + n_post) * 8 * n for n in n_octs_per_mg[:-1])
    if not exact_coarse:
        u += coarse_sweeps * 8 * n_octs_per_mg[-1]
    return u


# ------------------------------------------------------------- reference

def host_cores():
    """Cores this process may run on (the CPU baseline's thread count)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def amr3_workload(octs, tol):
    """The `config.workload` text of the headline benchmark (both arms)."""
    return ("amr3_256: 256^3 periodic lognormal base (sigma 2, k^-2, seed 3) + 3 levels refined at rho > 8 rho_bar "
            "(%s octs, %d cells); FP64 V(2,2) from phi = 0 to rel. residual %g per level, level by level"
            % ("/".join(str(int(o)) for o in octs), 8 * int(sum(octs)), tol))


def oracle_levels(cfg, n=None):
    """Oracle levels of a workload (each with its parent), densities set."""
    import oracle as O
    levels, parent = [], None
    for lev, c, r in list(zip(cfg["levels"], cfg["coords"], cfg["rho"]))[:n]:
        L = O.Level(lev, O.morton_encode(c), parent=parent)
        L.set_density(r, cfg.get("rho_bar", 1.0))
        levels.append(L)
        parent = L
    return levels


def oracle_updates(L, k):
    """Cell updates of one oracle V(2,2) cycle on the k-th level of a chain
    (the base level's coarsest 2^3 level is solved exactly, a refined level's
    coarsest gets its red-black sweeps), as the library counts them."""
    return cycle_updates([L.mg_n_octs(m) for m in range(L.mg_depth)], exact_coarse=(k == 0))


def run_reference(args, rank, world):
    """The oracle as it stands on the headline workload, on all host cores:
    each step is one FP64 V(2,2) cycle of one level of the chain, the levels
    taken in turn (level 8, 9, 10, 11, 8, ...), so that K steps sample every
    level of the workload about equally.  Builds and the ghost values from
    the parent's phi are outside the timed region."""
    import oracle as O
    from paper_2604_06035_gb300 import inputs
    if rank != 0:
        return
    cores = host_cores()
    threads = O.set_threads(cores)
    cfg = inputs.mixed_amr()
    levels = oracle_levels(cfg)
    upd = [oracle_updates(L, k) for k, L in enumerate(levels)]

    def step(k):
        levels[k % len(levels)].solve(fixed_cycles=1)

    for k in range(args.warmup):
        step(k)
    t0 = time.perf_counter()
    total = 0
    for k in range(args.steps):
        step(k)
        total += upd[k % len(levels)]
    dt = (time.perf_counter() - t0) / args.steps
    value = total / args.steps / dt / 1e6
    sample = ("one FP64 V(2,2) cycle per step, of levels 8, 9, 10, 11 in turn (%d threads on %d host cores)"
              % (threads, cores))
    print(json.dumps({
        "metric": "poisson_cell_updates_per_s", "value": value, "unit": "Mcell-updates/s", "impl": "reference",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": amr3_workload([len(c) for c in cfg["coords"]], args.tol),
                   "l2": "not applicable (CPU oracle)", "parallelism": "single"},
        "cpu_baseline": {"value": value, "unit": "Mcell-updates/s", "cores": threads, "host_cores": cores,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "Mcell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)
    O.set_threads(1)


def cpu_baseline_sample(cfg_amr3):
    """The oracle as it stands, timed on the host cores on bounded samples:
    one FP64 V(2,2) cycle of the headline workload's 256^3 base level on all
    host cores (OpenMP; bit-identical to one thread) and on one thread, and,
    labelled separately, one FP64 V(2,2) cycle of a 32-patch subset of the
    512-patch batched workload on all cores."""
    import oracle as O
    from paper_2604_06035_gb300 import inputs
    cores = host_cores()
    threads = O.set_threads(cores)
    t0 = time.perf_counter()
    base = oracle_levels(cfg_amr3, n=1)[0]
    build_s = time.perf_counter() - t0
    u = oracle_updates(base, 0)
    t0 = time.perf_counter()
    base.solve(fixed_cycles=1)
    dt_all = time.perf_counter() - t0
    O.set_threads(1)
    t0 = time.perf_counter()
    base.solve(fixed_cycles=1)
    dt_one = time.perf_counter() - t0
    del base
    out = {"value": u / dt_all / 1e6, "unit": "Mcell-updates/s", "cores": threads, "host_cores": cores,
           "kind": "oracle",
           "sample": "one FP64 V(2,2) cycle of the 256^3 base level (%d cell updates) on %d threads: %.2f s; "
                     "oracle build %.1f s untimed" % (u, threads, dt_all, build_s),
           "single_thread": {"value": u / dt_one / 1e6, "unit": "Mcell-updates/s", "cores": 1,
                             "sample": "the same cycle on one thread: %.2f s" % dt_one}}
    # 32-patch subset of the batched workload (every 16th patch by size rank)
    O.set_threads(cores)
    b = inputs.batched_patches(n_patches=512, seed=4)
    sub = batched_subset(b, 32)
    P = O.Level(b["level"] - 1, O.morton_encode(b["parent_coords"]))
    P.set_phi(b["parent_phi"])
    F = O.Level(b["level"], O.morton_encode(sub["coords"]), parent=P)
    F.set_density(sub["rho"], 1.0)
    uf = oracle_updates(F, 1)
    t0 = time.perf_counter()
    F.solve(fixed_cycles=1)
    dt_p = time.perf_counter() - t0
    out["batched_subset"] = {"value": uf / dt_p / 1e6, "unit": "Mcell-updates/s", "cores": threads,
                             "sample": "one FP64 V(2,2) cycle of 32 of the 512 patches (%d octs, every 16th by size); "
                                       "the batched block's GPU figure covers all 512" % len(sub["coords"])}
    O.set_threads(1)
    return out


def batched_subset(b, k):
    """k patches of a batched workload, every (n/k)-th by size rank: their
    octs (in patch order), densities and offsets."""
    import numpy as np
    off = np.asarray(b["offsets"])
    sizes = np.diff(off)
    order = np.argsort(sizes, kind="stable")
    pick = np.sort(order[::max(1, len(sizes) // k)][:k])
    idx = np.concatenate([np.arange(off[p], off[p + 1]) for p in pick])
    new_off = np.concatenate([[0], np.cumsum(sizes[pick])])
    return {"coords": b["coords"][idx], "rho": b["rho"][idx], "offsets": new_off, "patches": pick, "index": idx}


# ------------------------------------------------------------------- ours

def bench_batched(cmg, ctx, dev, stream, args):
    """512 independent refined patches (log-uniform 64..200000 octs, level 11,
    Dirichlet values from a smooth coarse field): one persistent cooperative
    kernel per solve.  Times mixed-precision and FP64 solves from phi = 0 to
    rel. residual tol on every patch, as V-cycle iterations and as per-patch
    CG preconditioned by them, each with the schedule the library's autotuner
    picks for it."""
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
    res = {"patches": 512, "octs": int(len(b["coords"])), "cells": int(8 * len(b["coords"])),
           "level": lev, "autotune_s": 0.0, "build_ms": build_ms, "generate_s": gen_s}
    reps = max(3, min(args.steps, 5))
    for name, prec, kr in (("mixed", cmg.CMG_PREC_MIXED, 0), ("fp64", cmg.CMG_PREC_FP64, 0),
                           ("mixed_pcg", cmg.CMG_PREC_MIXED, 1), ("fp64_pcg", cmg.CMG_PREC_FP64, 1)):
        cmg.cmg_level_set_phi(F, zeros)
        t0 = time.perf_counter()
        best, _ = cmg.cmg_batch_autotune(B, tol=args.tol, precision=prec, krylov=kr)
        res["autotune_s"] += time.perf_counter() - t0
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
                     "grid_barriers": st["grid_barriers"], "status": rc, "schedule": best}
        if kr == 0:
            # algorithmic bytes of the solve: per outer step, the V-cycles
            # (FP32 inner cycles in mixed precision) plus, per step, the FP64
            # residual with its norm (phi, g, index: 19 B per fine cell) and in
            # mixed precision the FP32 right-hand side (4 B) and phi += S e
            # (20 B)
            sch = cmg.cmg_batch_get_schedule(B)
            nsw = sch["n_pre"] + sch["n_post"]
            mg = [cmg.cmg_level_mg_info(F, m)[0] for m in range(cmg.cmg_level_mg_depth(F))]
            cells0 = 8.0 * mg[0]
            if prec == cmg.CMG_PREC_MIXED:
                per_step = sch["inner_cycles"] * vcycle_bytes(mg, 4, nsw) + cells0 * (19 + 4 + 20)
            else:
                per_step = vcycle_bytes(mg, 8, nsw) + cells0 * 19
            nbytes = per_step * st["cycles"]
            gbs = nbytes / (res[name]["ms_per_solve"] / 1e3) / 1e9
            res[name]["roofline"] = {"bound": "hbm", "achieved": gbs, "peak": read_peaks()["hbm"], "unit": "GB/s",
                                     "frac": gbs / read_peaks()["hbm"], "bytes_per_solve": nbytes,
                                     "bytes_per_fine_cell_per_step": per_step / cells0,
                                     "kernel": "k_batch (one persistent launch per solve)"}
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


def load_chain(cmg, ctx, dev, cfg):
    """Build a workload's levels on the device, each with its parent; returns
    (levels, rho device tensors, zero tensors)."""
    import torch
    levels, parent = [], None
    for lev, c in zip(cfg["levels"], cfg["coords"]):
        keys = cmg.cmg_morton_encode(ctx, torch.from_numpy(c).to(dev))
        L = cmg.cmg_level_build(ctx, lev, keys, parent=parent)
        levels.append(L)
        parent = L
    rho = [torch.from_numpy(r).to(dev) for r in cfg["rho"]]
    return levels, rho, [torch.zeros_like(r) for r in rho]


def chain_step(cmg, levels, rho, zeros, rho_bar, tol, precs):
    """One step of a chain: every level's phi = 0 and density, every solve
    queued level by level (a level's coarse-fine values read its parent's phi
    in stream order), then every report."""
    for L, r, z in zip(levels, rho, zeros):
        cmg.cmg_level_set_phi(L, z)
        cmg.cmg_level_set_density(L, r, rho_bar)
    for L, p in zip(levels, precs):
        cmg.cmg_level_solve_async(L, tol=tol, precision=p)
    return [cmg.cmg_level_solve_wait(L)[1] for L in levels]


def time_chain(cmg, levels, rho, zeros, rho_bar, tol, precs, reps=5, flush=None):
    """Median per-level time to tol over reps steps (after one untimed)."""
    per = [[] for _ in levels]
    stats = None
    for k in range(reps + 1):
        if flush is not None:
            flush.fill_(k & 0xFF)
        stats = chain_step(cmg, levels, rho, zeros, rho_bar, tol, precs)
        if k:
            for j, st in enumerate(stats):
                per[j].append(st["ms"])
    ms = [statistics.median(p) for p in per]
    upd = sum(st["cell_updates"] for st in stats)
    return {"ms_to_tol_per_level": ms, "ms_total": sum(ms), "iterations": [st["cycles"] for st in stats],
            "rel_final": [st["rel_final"] for st in stats], "Mcell_updates_per_s": upd / (sum(ms) / 1e3) / 1e6}


def rel_err(a, b):
    """max |a - b| / max |b| (torch or numpy)."""
    import numpy as np
    a = a.detach().cpu().numpy() if hasattr(a, "detach") else np.asarray(a)
    b = b.detach().cpu().numpy() if hasattr(b, "detach") else np.asarray(b)
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def bench_amr3(cmg, ctx, dev, args, chain, phi64, flush=None):
    """The headline workload in mixed precision (FP32 V-cycles inside FP64
    refinement) and with the FFT solve of the base under mixed fine levels,
    time to rel. residual tol level by level; phi of each chain against the
    FP64 chain at the benchmark tolerance and with both refined to 1e-12; the
    mixed chain's FP32 smoother rate."""
    levels, rho, zeros, rho_bar = chain
    F64, MIX, FFT = cmg.CMG_PREC_FP64, cmg.CMG_PREC_MIXED, cmg.CMG_PREC_FFT
    n = len(levels)
    out = {"tol": args.tol}
    out["mixed"] = time_chain(cmg, levels, rho, zeros, rho_bar, args.tol, [MIX] * n, flush=flush)
    out["mixed"]["phi_rel_err_vs_fp64_gpu"] = [rel_err(cmg.cmg_level_get_phi(L, device=True), p)
                                               for L, p in zip(levels, phi64)]
    out["fft_base_mixed_fine"] = time_chain(cmg, levels, rho, zeros, rho_bar, args.tol, [FFT] + [MIX] * (n - 1),
                                            flush=flush)
    out["fft_base_mixed_fine"]["phi_rel_err_vs_fp64_gpu"] = [
        rel_err(cmg.cmg_level_get_phi(L, device=True), p) for L, p in zip(levels, phi64)]
    # the precision effect alone: both chains refined to 1e-12 (untimed)
    tight = []
    for precs in ([F64] * n, [MIX] * n):
        chain_step(cmg, levels, rho, zeros, rho_bar, 1e-12, precs)
        tight.append([cmg.cmg_level_get_phi(L, device=True).clone() for L in levels])
    out["mixed"]["phi_rel_err_vs_fp64_gpu_both_at_1e-12"] = [rel_err(b, a) for a, b in zip(*tight)]
    # the FP32 smoother of the mixed chain, launch by launch
    cmg.cmg_ctx_reset_profile(ctx)
    cmg.cmg_ctx_set_profiling(ctx, True)
    chain_step(cmg, levels, rho, zeros, rho_bar, args.tol, [MIX] * n)
    cmg.cmg_ctx_set_profiling(ctx, False)
    prof = cmg.cmg_ctx_get_profile(ctx)
    peaks = read_peaks()
    sw = prof.get("rbgs_fp32")
    if sw and sw["ms"] > 0:
        gbs = sw["bytes"] / (sw["ms"] / 1e3) / 1e9
        out["mixed"]["roofline_smoother"] = {
            "bound": "hbm", "kernel": "rbgs_fp32", "achieved": gbs, "peak": peaks["hbm"], "unit": "GB/s",
            "frac": gbs / peaks["hbm"], "peak_source": peaks["hbm_src"], "launches": sw["launches"],
            "share_of_kernel_ms": sw["ms"] / sum(v["ms"] for v in prof.values())}
    out["mixed"]["kernels"] = {k: {"launches": v["launches"], "ms": round(v["ms"], 4)} for k, v in prof.items()
                               if v["launches"]}
    return out


def bench_small_chain(cmg, ctx, dev, args, cfg, name):
    """Time to rel. residual tol, FP64 and mixed, of a smaller workload (the
    128^3 two-level and the 32^3 periodic ones)."""
    levels, rho, zeros = load_chain(cmg, ctx, dev, cfg)
    n = len(levels)
    res = {"workload": name, "octs": [cmg.cmg_level_n_octs(L) for L in levels]}
    for pname, prec in (("fp64", cmg.CMG_PREC_FP64), ("mixed", cmg.CMG_PREC_MIXED)):
        res[pname] = time_chain(cmg, levels, rho, zeros, cfg["rho_bar"], args.tol, [prec] * n, reps=10)
    return res, (levels, rho, zeros)


def bench_oracle_errors(cmg, ctx, dev, args):
    """phi of the GPU solves against the FP64 oracle converged to 1e-12, per
    workload and level, outside any timed region: the GPU chain at the
    benchmark tolerance and at 1e-12, FP64 and mixed precision.  Workloads:
    32^3 periodic (full), 128^3 two-level (full), the 256^3 + 3-level
    hierarchy on a 64^3 base (the full one needs minutes of oracle time), and
    a 32-patch subset of the batched workload.  The learned warm start's
    error is in its own block."""
    import numpy as np
    import torch
    import oracle as O
    from paper_2604_06035_gb300 import inputs
    threads = O.set_threads(host_cores())
    F64, MIX = cmg.CMG_PREC_FP64, cmg.CMG_PREC_MIXED
    res = {"oracle_tol": 1e-12, "oracle_threads": threads,
           "measure": "max |phi_gpu - phi_oracle| / max |phi_oracle| per level"}

    def chain(cfg):
        t0 = time.perf_counter()
        ol = oracle_levels(cfg)
        for L in ol:
            L.solve(tol=1e-12, max_cycles=200)
        ref = [L.get_phi() for L in ol]
        out = {"oracle_s": time.perf_counter() - t0}
        levels, rho, zeros = load_chain(cmg, ctx, dev, cfg)
        for pname, prec in (("fp64", F64), ("mixed", MIX)):
            for tol in (args.tol, 1e-12):
                st = chain_step(cmg, levels, rho, zeros, cfg["rho_bar"], tol, [prec] * len(levels))
                out["%s_tol_%g" % (pname, tol)] = [rel_err(cmg.cmg_level_get_phi(L), r) for L, r in zip(levels, ref)]
                out["%s_tol_%g_cycles" % (pname, tol)] = [x["cycles"] for x in st]
        for L in reversed(levels):
            cmg.cmg_level_destroy(L)
        return out

    res["periodic_32"] = chain(inputs.periodic_grf_level(5, seed=1))
    res["two_level_128"] = chain(inputs.two_level_amr(base_level=7, seed=2))
    res["amr3_64_base"] = chain(inputs.mixed_amr(base_level=6))
    # batched: 32 patches (every 16th by size) of the 512-patch workload
    b = inputs.batched_patches(n_patches=512, seed=4)
    sub = batched_subset(b, 32)
    t0 = time.perf_counter()
    P = O.Level(b["level"] - 1, O.morton_encode(b["parent_coords"]))
    P.set_phi(b["parent_phi"])
    F = O.Level(b["level"], O.morton_encode(sub["coords"]), parent=P)
    F.set_density(sub["rho"], 1.0)
    F.solve(tol=1e-12, max_cycles=200)
    ref = F.get_phi()
    out = {"patches": 32, "octs": int(len(sub["coords"])), "oracle_s": time.perf_counter() - t0}
    Pg = cmg.cmg_level_build(ctx, b["level"] - 1,
                             cmg.cmg_morton_encode(ctx, torch.from_numpy(b["parent_coords"]).to(dev)))
    cmg.cmg_level_set_phi(Pg, torch.from_numpy(b["parent_phi"]).to(dev))
    Fg = cmg.cmg_level_build(ctx, b["level"], cmg.cmg_morton_encode(ctx, torch.from_numpy(sub["coords"]).to(dev)),
                             parent=Pg)
    Bg = cmg.cmg_batch_create(Fg, sub["offsets"])
    rho = torch.from_numpy(sub["rho"]).to(dev)
    zeros = torch.zeros_like(rho)
    cmg.cmg_level_set_density(Fg, rho, 1.0)
    for pname, prec in (("fp64", F64), ("mixed", MIX)):
        for tol in (args.tol, 1e-12):
            cmg.cmg_level_set_phi(Fg, zeros)
            rc, st = cmg.cmg_batch_solve(Bg, tol=tol, precision=prec)
            out["%s_tol_%g" % (pname, tol)] = rel_err(cmg.cmg_level_get_phi(Fg), ref)
            out["%s_tol_%g_cycles" % (pname, tol)] = st["cycles"]
    cmg.cmg_batch_destroy(Bg)
    cmg.cmg_level_destroy(Fg)
    cmg.cmg_level_destroy(Pg)
    res["batched_subset"] = out
    O.set_threads(1)
    return res


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
           "output_scale": cmg.cmg_unet_get_output_scale(net), "grad_clip": cmg.cmg_unet_grad_clip_stats(net)}
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
    # phi from the network's start at tol against the FP64 oracle converged to
    # 1e-12 on the same held-out density (64^3 periodic level)
    import oracle as O
    from paper_2604_06035_gb300 import inputs
    O.set_threads(host_cores())
    lev = int(round(np.log2(D)))
    coords = inputs.uniform_oct_coords(lev)
    ol = O.Level(lev, O.morton_encode(coords))
    rho_np = rho.double().cpu().numpy().transpose(2, 1, 0)  # (z, y, x) -> [x, y, z]
    ol.set_density(inputs.dense_to_octs(rho_np, coords), float(rho_np.mean()))
    ol.solve(tol=1e-12, max_cycles=200)
    ref = inputs.octs_to_dense(ol.get_phi(), coords, D).transpose(2, 1, 0)
    O.set_threads(1)
    pred = W.predict(S, net, rho, prev)
    errs = {}
    for name, prec in (("fp64", cmg.CMG_PREC_FP64), ("mixed", cmg.CMG_PREC_MIXED)):
        for tol in (args.tol, 1e-12):
            phi, _ = S.solve(rho, pred, tol, prec)
            errs["%s_tol_%g" % (name, tol)] = rel_err(phi, ref)
    res["phi_vs_oracle"] = {"pair": "trajectory %d, step %d" % (k, t + 1), "start": "network prediction",
                            "oracle_tol": 1e-12, **errs}
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


def headline_roofline(prof, peaks, sm_mhz):
    """Roofline of the dominant kernel family of the timed steps: algorithmic
    bytes per launch (field values plus the neighbour cache, 27 B per FP64
    cell update in a colour pass) over its per-launch CUDA-event time, against
    the measured HBM copy rate.  The FP64 colour pass also gets its FP64-pipe
    fraction: 2 FP64 instructions per cell update (1 DADD + 1 DFMA; the other
    neighbour additions run as an integer fixed-point sum on the ALU pipe)
    against 2 lanes per SM per clock, 152 SMs at the sampled SM clock."""
    dname, d = max(prof.items(), key=lambda kv: kv[1]["ms"])
    gbs = d["bytes"] / (d["ms"] / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm"], "unit": "GB/s", "frac": gbs / peaks["hbm"],
            "kernel": dname, "peak_source": peaks["hbm_src"] + " copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}
    if dname.startswith("rbgs_") and dname.endswith("fp64"):
        clk = (sm_mhz or 2070.0) * 1e6
        cells_per_s = d["bytes"] / 27.0 / (d["ms"] / 1e3)
        instr = 2.0 * cells_per_s
        peak_instr = 2.0 * 152 * clk
        roof["fp64_issue_frac"] = instr / peak_instr
        roof["fp64_issue_note"] = ("FP64 lane-instructions/s (2 per cell update: 1 DADD + 1 DFMA; five of the six "
                                   "neighbours are summed on the integer pipe) against 2 per SM per clock x 152 SMs "
                                   "at %.0f MHz" % (clk / 1e6))
    roof["launches"] = d["launches"]
    roof["ms_per_launch"] = d["ms"] / d["launches"]
    roof["bytes_per_launch"] = d["bytes"] / d["launches"]
    roof["share_of_kernel_ms"] = d["ms"] / sum(v["ms"] for v in prof.values())
    roof["traffic"] = traffic_for(dname + "_amr3")
    return roof


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
    t0 = time.perf_counter()
    cfg = inputs.mixed_amr()
    gen_s = time.perf_counter() - t0
    rho_bar = cfg["rho_bar"]
    coords = [torch.from_numpy(c).to(dev) for c in cfg["coords"]]
    rho = [torch.from_numpy(r).to(dev) for r in cfg["rho"]]
    zeros = [torch.zeros_like(r) for r in rho]

    # setup: keys (a1), hash + neighbour cache + hierarchy (a2, a3), ghost stencils
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    levels, parent = [], None
    for lev, c in zip(cfg["levels"], coords):
        L = cmg.cmg_level_build(ctx, lev, cmg.cmg_morton_encode(ctx, c), parent=parent)
        levels.append(L)
        parent = L
    torch.cuda.synchronize()
    build_ms = (time.perf_counter() - t0) * 1e3
    del coords
    n = len(levels)
    octs = [cmg.cmg_level_n_octs(L) for L in levels]
    F64 = cmg.CMG_PREC_FP64

    def step(precision=F64):
        return chain_step(cmg, levels, rho, zeros, rho_bar, args.tol, [precision] * n)

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
    last = all_stats[-1]
    peaks = read_peaks()
    roofline = headline_roofline(prof, peaks, clocks.get("sm_mhz"))
    roofline["timing"] = ("per-launch CUDA events on the library stream over a repeat of the timed steps "
                          "launched kernel by kernel (%.2f ms/step there)" % (prof_ms / args.steps))
    phi64 = [cmg.cmg_level_get_phi(L, device=True).clone() for L in levels]

    out = {
        "metric": "poisson_cell_updates_per_s", "value": value, "unit": "Mcell-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": amr3_workload(octs, args.tol),
                   "l2": "inputs larger than L2 (every level's phi + g > 129 MB), and flushed before each timed "
                         "step (512 MiB write)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "time_to_tol_ms": {"level_%d" % lv: st["ms"] for lv, st in zip(cfg["levels"], last)},
        "cycles": {"level_%d" % lv: st["cycles"] for lv, st in zip(cfg["levels"], last)},
        "rel_residual": {"level_%d" % lv: st["rel_final"] for lv, st in zip(cfg["levels"], last)},
        "setup_ms": build_ms, "generate_s": gen_s,
        "roofline": roofline,
        "kernels": {k: {"launches": v["launches"], "ms": v["ms"], "GB/s": v["bytes"] / v["ms"] / 1e6,
                        "TFLOP/s": v["flops"] / v["ms"] / 1e9} for k, v in prof.items() if v["launches"]},
        "gpu_launches": launches,
        "clocks": clocks,
    }

    if args.quick:
        # profiling runs: the timed steps only
        out["e2e"] = None
        if rank == 0:
            print(json.dumps(out), flush=True)
        torch.cuda.synchronize()
        for L in reversed(levels):
            cmg.cmg_level_destroy(L)
        cmg.cmg_ctx_destroy(ctx)
        if world > 1:
            dist.destroy_process_group()
        return

    # end to end through the C ABI with host buffers (pinned): H2D densities
    # of the four levels, the four solves, D2H of the four phi arrays
    pin_rho = [torch.from_numpy(r).pin_memory().numpy() for r in cfg["rho"]]
    pin_phi = [torch.empty((o, 8), dtype=torch.float64).pin_memory().numpy() for o in octs]
    e2e_ms, e2e_upd = 0.0, 0
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        # per level: upload (overlapping the parent's queued solve), solve,
        # queued read-back (overlapping the next level's solve)
        for L, r, z, o in zip(levels, pin_rho, zeros, pin_phi):
            cmg.cmg_level_set_phi(L, z)  # zero initial guess, already on the device
            cmg.cmg_level_set_density(L, r, rho_bar)
            cmg.cmg_level_solve_async(L, tol=args.tol)
            cmg.cmg_level_get_phi_async(L, out=o)
        for L in levels:
            rc, st = cmg.cmg_level_solve_wait(L)
            e2e_upd += st["cell_updates"]
        cmg.cmg_ctx_synchronize(ctx)
        e2e_ms += (time.perf_counter() - t0) * 1e3
    h2d = sum(r.nbytes for r in pin_rho)
    d2h = sum(o.nbytes for o in pin_phi)
    e2e_max, e2e_upd_total = aggregate_ranks(e2e_ms, e2e_upd, world, dev)
    out["e2e"] = {"value": e2e_upd_total / (e2e_max / 1e3) / 1e6, "unit": "Mcell-updates/s",
                  "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_max / args.steps}
    del pin_rho, pin_phi

    if not args.no_extra:
        chain = (levels, rho, zeros, rho_bar)
        out["amr3_mixed"] = bench_amr3(cmg, ctx, dev, args, chain, phi64, flush=flush)
        fp64_ms = sum(st["ms"] for st in last)
        out["amr3_mixed"]["fp64_ms_total"] = fp64_ms
        out["amr3_mixed"]["speedup_mixed_vs_fp64"] = fp64_ms / out["amr3_mixed"]["mixed"]["ms_total"]
        out["amr3_mixed"]["speedup_fft_mixed_vs_fp64"] = fp64_ms / out["amr3_mixed"]["fft_base_mixed_fine"]["ms_total"]
        del phi64
        out["two_level_128"], (tl_levels, tl_rho, _) = bench_small_chain(
            cmg, ctx, dev, args, inputs.two_level_amr(base_level=7, seed=2), "128^3 lognormal (sigma 1.5) + 1 level")
        out["periodic_32"], (p32, _, _) = bench_small_chain(
            cmg, ctx, dev, args, inputs.periodic_grf_level(5, seed=1), "32^3 periodic, rho = 1 + GRF (rms 0.5)")
        cmg.cmg_level_destroy(p32[0])
        out["batched"] = bench_batched(cmg, ctx, dev, stream, args)
        out["smoother_512"] = bench_smoother(cmg, ctx, dev, peaks)
        out["fft"] = bench_fft(cmg, ctx, dev, tl_levels[0], tl_rho[0], args, peaks)
        out["pcg"] = bench_pcg(cmg, ctx, dev, (("base", tl_levels[0], tl_rho[0]), ("fine", tl_levels[1], tl_rho[1])),
                               args)
        for L in reversed(tl_levels):
            cmg.cmg_level_destroy(L)
        if not args.no_learned:
            out["learned"] = bench_learned(cmg, ctx, dev, args, peaks)
        if not args.no_oracle_errors and rank == 0:
            out["phi_vs_oracle"] = bench_oracle_errors(cmg, ctx, dev, args)
    if rank == 0 and world == 1:
        out["cpu_baseline"] = cpu_baseline_sample(cfg)
    if rank == 0:
        print(json.dumps(out), flush=True)
    torch.cuda.synchronize()
    for L in reversed(levels):
        cmg.cmg_level_destroy(L)
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
        # the headline chain once in FP64 (its phi is the reference), then the
        # mixed and FFT chains
        from paper_2604_06035_gb300 import inputs
        cfg = inputs.mixed_amr()
        levels, rho, zeros = load_chain(cmg, ctx, dev, cfg)
        chain_step(cmg, levels, rho, zeros, cfg["rho_bar"], args.tol, [cmg.CMG_PREC_FP64] * len(levels))
        phi64 = [cmg.cmg_level_get_phi(L, device=True).clone() for L in levels]
        out = bench_amr3(cmg, ctx, dev, args, (levels, rho, zeros, cfg["rho_bar"]), phi64)
        for L in reversed(levels):
            cmg.cmg_level_destroy(L)
    elif args.block in ("two_level", "periodic32"):
        from paper_2604_06035_gb300 import inputs
        cfg = (inputs.two_level_amr(base_level=7, seed=2) if args.block == "two_level"
               else inputs.periodic_grf_level(5, seed=1))
        out, (levels, _, _) = bench_small_chain(cmg, ctx, dev, args, cfg, args.block)
        for L in reversed(levels):
            cmg.cmg_level_destroy(L)
    elif args.block == "oracle_errors":
        out = bench_oracle_errors(cmg, ctx, dev, args)
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
