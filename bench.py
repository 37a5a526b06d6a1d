"""Benchmark: cell-updates/s of the dimension-split wave-propagation step.

Workload (default): 2D shallow water, Roe + Harten-Hyman, radial dam break on
[-1,1]^2 at 4096 x 4096 cells, minmod, outflow boundaries, CFL 0.9, FP32
chosen form (the FP64 plain path is timed beside it).  A step is one full
time step: x sweep, y sweep and the device-side CFL control, over the whole
grid.  Inputs are synthetic (seeded) and resident in HBM; each FP32 state
version is 201 MB (> 129 MB L2), so every sweep streams from HBM.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle instead (the reference arm).
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import platform
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_DEFAULT = 4096
METRIC = "cell-updates/s"
# Algorithmic flops of one shallow-water cell per sweep: the paper's Nsight
# count of 313 flop per cell-step over its two sweeps (Tables 1-2 give the
# per-sweep MFlop at 1024^2).  Our FP32 sweep executes 158.7 per cell; the
# FP64 x sweep executes 197.1 (2 per DFMA, 1 per DADD / DMUL: the double
# reciprocal square roots and the Newton reciprocals expand into FMA
# sequences) -- both counted with ncu, see profiles/.
SW_FLOP_PER_CELL_SWEEP = 313.0 / 2.0
FP64_EXECUTED_DFLOP = 197.1


# Files the FP32 shallow-water sweep kernels are compiled from (the unit
# that instantiates them and every header it includes) and the build flags.
SWEEP_SOURCES = ("sweep_shallow_water_f32.cu", "sweep_dispatch.cuh", "launch.h", "sweep.cuh",
                 "claw_types.cuh", "riemann.cuh", "pair.cuh", "tma.cuh", "../build.py")


def kernel_source_digest(files=SWEEP_SOURCES):
    """Digest of the sources the profiled kernels are built from: a traffic
    record taken with ncu is valid only for the kernels it was taken on."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1805_08846_gb300", "csrc")
    for f in files:
        h.update(f.encode())
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_record(kernel, workload):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu
    summaries (a line `traffic-record: kernel=... workload=... sources=...
    dram_bytes=...`), or None when no record matches the current sources."""
    digest = kernel_source_digest()
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        with open(path) as f:
            for line in f:
                line = line.strip().strip("`")
                if not line.startswith("traffic-record:"):
                    continue
                kv = dict(t.split("=", 1) for t in line.split()[1:] if "=" in t)
                if kv.get("kernel") == kernel and kv.get("workload") == workload \
                        and kv.get("sources") == digest:
                    return float(kv["dram_bytes"]), os.path.relpath(path, ROOT)
    return None, None


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if parts[5 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_oracle_rate(prob, seconds_budget=20.0, max_steps=50):
    """Time the FP64 oracle (all host threads) on full steps of the workload;
    returns (cell-updates/s, steps, threads)."""
    import oracle
    o = oracle.Oracle(prob)
    q = prob.q0
    t0 = time.perf_counter()
    r = o.run_steps(q, 1)
    one = time.perf_counter() - t0
    steps = max(1, min(max_steps, int(seconds_budget / max(one, 1e-3))))
    t0 = time.perf_counter()
    o.run_steps(r["q"], steps, dt=r["dt"])
    el = time.perf_counter() - t0
    return prob.ncells * steps / el, steps, oracle.threads(), el


def graph_ms_per_step(s, prob, steps, warm=3):
    """Milliseconds per step of one claw_run_steps call of `steps` steps (one
    graph replay), timed with CUDA events on torch's current stream (the
    solver's stream).  The graph is captured in an untimed call first; the
    state then starts over from prob.q0."""
    import torch
    s.run_steps(steps)
    s.set_q(prob.q0)
    s.set_time(0.0, 0.0, 0)
    s.run_steps(warm)
    st = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    s.run_steps(steps)
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def extra_acoustics3d(args, peak_gbs):
    """3D variable-coefficient acoustics, two layers, 512^3, walls, MC: FP32
    and FP64 cell-updates/s, per-sweep times and the HBM fraction of the
    dominant FP32 sweep (6 values of 4 B per cell and sweep: p, u_d read and
    written, Z, c read)."""
    from paper_1805_08846_gb300 import Solver, inputs
    prob = inputs.acoustics_3d_layers(args.n3)
    out = {"workload": f"3D two-layer acoustics {args.n3}^3, MC, walls, CFL 0.9"}
    for prec, steps in ((32, args.steps3), (64, max(2, args.steps3 // 10))):
        s = Solver.from_problem(prob, precision=prec, stream="torch")
        seg = s.autotune(2)
        s.run_steps(3)
        ms, tot, nl = s.profile_steps(steps)          # per-sweep breakdown
        step_ms = graph_ms_per_step(s, prob, steps)
        s.close()
        r = {"value": prob.ncells / (step_ms * 1e-3), "ms_per_step": step_ms,
             "sweep_ms": ms[:3], "steps": steps, "segments": seg}
        if prec == 32:
            dom = int(np.argmax(ms[:3]))
            ach = 24 * prob.ncells / (ms[dom] * 1e-3) / 1e9
            r["roofline"] = {"bound": "hbm", "achieved": ach, "peak": peak_gbs, "unit": "GB/s",
                             "frac": ach / peak_gbs, "kernel": f"sweep dir={'xyz'[dom]}"}
        out[f"f{prec}"] = r
    return out


def extra_bathymetry(args, peak_gbs):
    """Shallow water over a seamount (source term as f-waves, well-balanced),
    4096^2, minmod, outflow: FP32 and FP64 cell-updates/s and the HBM
    fraction of the dominant FP32 sweep (7 values of 4 B per cell and sweep:
    h, hu, hv read and written, B read)."""
    from paper_1805_08846_gb300 import Solver, inputs
    prob = inputs.sw_bathymetry(args.n)
    out = {"workload": f"2D shallow water over a seamount {args.n}^2 (f-wave source), minmod, "
                       f"outflow, CFL 0.9"}
    for prec, steps in ((32, 100), (64, 5)):
        s = Solver.from_problem(prob, precision=prec, stream="torch")
        seg = s.autotune(2)
        s.run_steps(3)
        ms, tot, nl = s.profile_steps(steps)          # per-sweep breakdown
        step_ms = graph_ms_per_step(s, prob, steps)
        s.close()
        r = {"value": prob.ncells / (step_ms * 1e-3), "ms_per_step": step_ms,
             "sweep_ms": ms[:2], "steps": steps, "segments": seg[:2]}
        if prec == 32:
            dom = int(np.argmax(ms[:2]))
            ach = 28 * prob.ncells / (ms[dom] * 1e-3) / 1e9
            r["roofline"] = {"bound": "hbm", "achieved": ach, "peak": peak_gbs, "unit": "GB/s",
                             "frac": ach / peak_gbs, "kernel": f"sweep dir={'xy'[dom]}"}
        out[f"f{prec}"] = r
    return out


def extra_dry(args, peak_gbs):
    """Shallow water with wetting and drying (hydrostatic reconstruction
    around HLLE) on a 4096^2 lake around an emerged island, a surface hump
    running up its shore, walls: FP32 and FP64 cell-updates/s and the HBM
    fraction of the dominant FP32 sweep (7 values of 4 B per cell and sweep:
    h, hu, hv read and written, B read)."""
    from paper_1805_08846_gb300 import Solver, inputs
    prob = inputs.sw_island(args.n)
    out = {"workload": f"2D shallow water with wetting and drying, {args.n}^2 lake around an "
                       f"emerged island, hump running up its shore, minmod, walls, CFL 0.9"}
    for prec, steps in ((32, 100), (64, 5)):
        s = Solver.from_problem(prob, precision=prec, stream="torch")
        seg = s.autotune(2)
        s.run_steps(3)
        ms, tot, nl = s.profile_steps(steps)          # per-sweep breakdown
        step_ms = graph_ms_per_step(s, prob, steps)
        s.close()
        r = {"value": prob.ncells / (step_ms * 1e-3), "ms_per_step": step_ms,
             "sweep_ms": ms[:2], "steps": steps, "segments": seg[:2]}
        if prec == 32:
            dom = int(np.argmax(ms[:2]))
            ach = 28 * prob.ncells / (ms[dom] * 1e-3) / 1e9
            r["roofline"] = {"bound": "hbm", "achieved": ach, "peak": peak_gbs, "unit": "GB/s",
                             "frac": ach / peak_gbs, "kernel": f"sweep dir={'xy'[dom]}"}
        out[f"f{prec}"] = r
    return out


def extra_unsplit(args, peak_gbs):
    """The unsplit update with transverse waves on the 4096^2 radial dam
    break (minmod, outflow): FP32 and FP64 cell-updates/s of the one kernel
    per step and its HBM fraction (6 values per cell and step: h, hu, hv
    read once and written once; 24 B in FP32)."""
    from paper_1805_08846_gb300 import Solver, inputs
    prob = inputs.sw_radial_dam_break(args.n).with_(splitting="unsplit")
    out = {"workload": f"2D shallow water radial dam break {args.n}^2, unsplit update with "
                       f"transverse waves, minmod, outflow, CFL 0.9"}
    for prec, steps in ((32, 100), (64, 5)):
        s = Solver.from_problem(prob, precision=prec, stream="torch")
        seg = s.autotune(2)
        s.run_steps(3)
        ms, tot, nl = s.profile_steps(steps)          # kernel breakdown
        step_ms = graph_ms_per_step(s, prob, steps)
        s.close()
        ach = (6 * prec // 8) * prob.ncells / (ms[0] * 1e-3) / 1e9
        out[f"f{prec}"] = {"value": prob.ncells / (step_ms * 1e-3), "ms_per_step": step_ms,
                           "kernel_ms": ms[0], "control_ms": ms[3], "steps": steps,
                           "rows_per_tile": seg[1],
                           "roofline": {"bound": "hbm", "achieved": ach, "peak": peak_gbs,
                                        "unit": "GB/s", "frac": ach / peak_gbs,
                                        "kernel": f"unsplit_kernel<ShallowWater<{'float' if prec == 32 else 'double'}>,minmod>"}}
    return out


# Sec. 7.1 (Tables 1-6): the paper's kernel-analysis problems.  Values a
# sweep reads and writes per cell (fields it leaves unchanged are neither):
# 2D acoustics p, u_d (2 + 2); shallow water h, hu, hv (3 + 3); 3D
# variable-coefficient acoustics p, u_d (2 + 2) and Z, c (2 read).
PAPER_PROBLEMS = (
    ("acoustics_2d_1024", "mc", 4, "acoustics_2d_pulse", 1024),
    ("shallow_water_1024", "minmod", 6, "sw_radial_dam_break", 1024),
    ("acoustics_3d_96", "mc", 6, "acoustics_3d_layers", 96),
)


def paper_tables(args):
    """Per-sweep times at the sizes of Sec. 7.1 Tables 1-6, for the full
    method and for its first-order form (the Riemann solution and the
    fluctuation update alone: the "Riemann solver" kernels of Tables 4-6),
    FP32 and FP64.  DRAM bytes and flops per kernel come from ncu on the
    same command (profiles/)."""
    from paper_1805_08846_gb300 import Solver, inputs
    rows = []
    for name, lim, vals, gen, n in PAPER_PROBLEMS:
        for method in (lim, "first_order"):
            prob = getattr(inputs, gen)(n, limiter=method)
            for prec in (32, 64):
                s = Solver.from_problem(prob, precision=prec)
                if args.fixed_segments:
                    for d in range(prob.ndim):
                        s.set_segment(d, 64)
                    seg = [64] * prob.ndim
                else:
                    seg = s.autotune(2)[:prob.ndim]
                s.run_steps(args.warmup)
                best = None
                for _ in range(3 if not args.fixed_segments else 1):
                    ms, tot, _nl = s.profile_steps(args.steps)
                    if best is None or tot < best[1]:
                        best = (ms, tot)
                s.close()
                ms, tot = best
                es = prec // 8
                alg = vals * es * prob.ncells
                rows.append({
                    "problem": name, "method": method, "precision": prec,
                    "sweep_us": [round(1e3 * m, 2) for m in ms[:prob.ndim]],
                    "step_us": round(1e3 * tot / args.steps, 2),
                    "alg_bytes_per_sweep": alg,
                    "achieved_gbs": [round(alg / (m * 1e-3) / 1e9, 1) for m in ms[:prob.ndim]],
                    "cell_updates_per_s": prob.ncells * args.steps / (tot * 1e-3),
                    "segments": seg})
    print(json.dumps({"mode": "paper_tables", "steps": args.steps, "rows": rows}), flush=True)
    return 0


def size_scaling(args):
    """Cell-updates/s against grid size, 256^2 .. 16384^2 (the paper's
    problem-size scaling figures), both 2D systems, FP32 and FP64."""
    from paper_1805_08846_gb300 import Solver, inputs
    rows = []
    for name, gen in (("shallow_water", lambda n: inputs.sw_radial_dam_break(n)),
                      ("acoustics_2d", lambda n: inputs.acoustics_2d_pulse(n))):
        for n in (256, 512, 1024, 2048, 4096, 8192, 16384):
            prob = gen(n)
            for prec in (32, 64):
                s = Solver.from_problem(prob, precision=prec)
                seg = s.autotune(1 if n >= 8192 else 2)[:2]
                cost = (1.0 if prec == 32 else 25.0) * prob.ncells   # ~cells x relative step cost
                steps = int(max(3, min(200, 4e9 / cost)))
                s.run_steps(3)
                ms, tot, _nl = s.profile_steps(steps)
                s.close()
                rows.append({"system": name, "n": n, "precision": prec, "steps": steps,
                             "ms_per_step": tot / steps,
                             "cell_updates_per_s": prob.ncells * steps / (tot * 1e-3),
                             "sweep_ms": ms[:2], "segments": seg})
                print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    print(json.dumps({"mode": "size_scaling", "rows": rows}), flush=True)
    return 0


def accuracy(args):
    """Errors of the GPU paths on the five workloads, against the FP64 oracle
    (or, for the 3D acoustics ensemble and 100 steps of the 512^3 problem,
    against the FP64 GPU path pinned to it), with the time of each path:
    relative L-inf per field (worst field) for FP64, relative L1 on h and on
    h - 1 for FP32 shallow water, relative L2 (worst field) for FP32
    acoustics.  The oracle runs on all host cores."""
    import oracle as orc
    from oracle import Oracle
    from paper_1805_08846_gb300 import Ensemble, Solver, inputs

    def linf(a, b):
        return max(orc.rel_linf(a[f], b[f]) for f in range(a.shape[0]))

    def l2(a, b):
        return max(orc.rel_l2(a[f], b[f]) for f in range(a.shape[0]) if np.abs(b[f]).max() > 0)

    def gpu(prob, steps, prec):
        with Solver.from_problem(prob, precision=prec) as s:
            s.autotune(2)
            t0 = time.perf_counter()
            s.run_steps(steps)
            q = s.get_q()
            el = time.perf_counter() - t0
            t = s.time()[0]
        return q, el, t

    def oracle_run(prob, steps):
        t0 = time.perf_counter()
        r = Oracle(prob).run_steps(prob.q0, steps)
        return r, time.perf_counter() - t0

    out = {"mode": "accuracy", "host_threads": orc.threads(), "rows": []}
    add = out["rows"].append
    # C1: 2D acoustics 128^2, 100 steps
    prob = inputs.acoustics_2d_pulse(128)
    ref, el_o = oracle_run(prob, 100)
    q64, el64, _ = gpu(prob, 100, 64)
    q32, el32, _ = gpu(prob, 100, 32)
    add({"config": "C1 acoustics 128^2, 100 steps", "cells_x_steps": prob.ncells * 100,
         "oracle_s": el_o, "fp64_s": el64, "fp32_s": el32,
         "fp64_rel_linf": linf(q64, ref["q"]), "fp32_rel_l2": l2(q32, ref["q"])})
    # C2: 4096^2 dam break, 200 steps
    prob = inputs.sw_radial_dam_break(4096)
    ref, el_o = oracle_run(prob, 200)
    q64, el64, _ = gpu(prob, 200, 64)
    q32, el32, _ = gpu(prob, 200, 32)
    add({"config": "C2 shallow water 4096^2, 200 steps", "cells_x_steps": prob.ncells * 200,
         "oracle_s": el_o, "fp64_s": el64, "fp32_s": el32,
         "fp64_rel_linf": linf(q64, ref["q"]),
         "fp32_rel_l1_h": orc.rel_l1(q32[0], ref["q"][0]),
         "fp32_rel_l1_h_minus_1": orc.rel_l1(q32[0] - 1.0, ref["q"][0] - 1.0),
         "fp32_rel_l1_hu": orc.rel_l1(q32[1], ref["q"][1]),
         "fp32_rel_l1_hv": orc.rel_l1(q32[2], ref["q"][2])})
    # shallow water with wetting and drying: the 4096^2 island run-up, 20 steps
    prob = inputs.sw_island(4096)
    ref, el_o = oracle_run(prob, 20)
    q64, el64, _ = gpu(prob, 20, 64)
    q32, el32, _ = gpu(prob, 20, 32)
    add({"config": "wetting and drying, 4096^2 island run-up, 20 steps", "cells_x_steps": prob.ncells * 20,
         "oracle_s": el_o, "fp64_s": el64, "fp32_s": el32,
         "fp64_rel_linf": linf(q64, ref["q"]),
         "fp32_rel_l1": [orc.rel_l1(q32[f], ref["q"][f]) for f in range(3)],
         "min_h_fp64": float(q64[0].min()), "min_h_fp32": float(q32[0].min()),
         "mass_change_fp64": float(q64[0].sum() / prob.q0[0].sum() - 1.0)})
    # C3: 512^3 two-layer acoustics: 2 steps against the oracle, 100 steps
    # FP32 against FP64
    prob = inputs.acoustics_3d_layers(512)
    ref, el_o = oracle_run(prob, 2)
    q64, _, _ = gpu(prob, 2, 64)
    q32, _, _ = gpu(prob, 2, 32)
    q64b, el64, _ = gpu(prob, 100, 64)
    q32b, el32, _ = gpu(prob, 100, 32)
    add({"config": "C3 3D acoustics 512^3", "oracle_s_2_steps": el_o,
         "fp64_s_100_steps": el64, "fp32_s_100_steps": el32,
         "fp64_rel_linf_2_steps_vs_oracle": linf(q64, ref["q"]),
         "fp32_rel_l2_2_steps_vs_oracle": l2(q32, ref["q"]),
         "fp32_rel_l2_100_steps_vs_fp64_gpu": l2(q32b, q64b)})
    # C4: 256-grid SW ensemble, 50 steps; 12 instances against the oracle
    probs = inputs.sw_ensemble()
    sizes = [p.n[0] for p in probs]
    sample = sorted(set([0, 1, 2, 3, 64, 128, 200, 255, int(np.argmin(sizes)), int(np.argmax(sizes))]))
    res = {}
    for prec in (32, 64):
        e = Ensemble.from_problems(probs, precision=prec)
        e.autotune(1)
        e.run_steps(50)
        res[prec] = {i: e.get_q(i) for i in sample}
        e.close()
    e64, e32, e32p = 0.0, 0.0, 0.0
    for i in sample:
        ref = Oracle(probs[i]).run_steps(probs[i].q0, 50)["q"]
        e64 = max(e64, linf(res[64][i], ref))
        e32 = max(e32, orc.rel_l1(res[32][i][0], ref[0]))
        e32p = max(e32p, orc.rel_l1(res[32][i][0] - 1.0, ref[0] - 1.0))
    add({"config": "C4 SW ensemble, 256 grids, 50 steps", "instances_checked": len(sample),
         "fp64_rel_linf_max": e64, "fp32_rel_l1_h_max": e32, "fp32_rel_l1_h_minus_1_max": e32p})
    # C5: 64-cube acoustics ensemble, 100 steps, FP32 batched against FP64
    # per instance (every instance)
    probs = inputs.acoustics3d_ensemble()
    e = Ensemble.from_problems(probs, precision=32)
    e.autotune(1)
    e.run_steps(100)
    worst = 0.0
    for i, p in enumerate(probs):
        with Solver.from_problem(p, precision=64) as s:
            s.run_steps(100)
            worst = max(worst, l2(e.get_q(i), s.get_q()))
    e.close()
    add({"config": "C5 3D acoustics ensemble, 64 cubes, 100 steps", "instances_checked": len(probs),
         "fp32_rel_l2_vs_fp64_gpu_max": worst})
    print(json.dumps(out), flush=True)
    return 0


def extra_ensembles(args, peak_gbs):
    """Batched FP32 ensembles (one launch per sweep for all instances) against
    the plain FP64 path run instance by instance on the same instances; the
    batched sweeps' times and the HBM fraction of the dominant one (24 B per
    cell and sweep in both: shallow water h, hu, hv read and written; 3D
    acoustics p, u_d read and written, Z, c read)."""
    from paper_1805_08846_gb300 import Ensemble, Solver, inputs
    res = {}
    for name, gen, steps32, steps64 in (
            ("sw_256", lambda: inputs.sw_ensemble(), 50, 5),
            ("acoustics3d_64", lambda: inputs.acoustics3d_ensemble(), 100, 3)):
        probs = gen()
        cells = sum(p.ncells for p in probs)
        ndim = probs[0].ndim
        e = Ensemble.from_problems(probs, precision=32)
        seg = e.autotune(1)
        shapes = [e.tile_shape(d) for d in range(ndim)]
        e.run_steps(3)
        ms, tot, nl = e.profile_steps(steps32)
        e.close()
        v32 = cells * steps32 / (tot * 1e-3)
        dom = int(np.argmax(ms[:ndim]))
        ach = 24 * cells / (ms[dom] * 1e-3) / 1e9
        t64 = 0.0
        for p in probs:
            s = Solver.from_problem(p, precision=64)
            s.run_steps(1)
            ms64, tot64, _ = s.profile_steps(steps64)
            s.close()
            t64 += tot64
        v64 = cells * steps64 / (t64 * 1e-3)
        res[name] = {"instances": len(probs), "cells": cells, "fp32_batched": v32,
                     "fp32_steps": steps32, "fp64_per_instance": v64, "fp64_steps": steps64,
                     "ratio": v32 / v64, "segments": seg, "unit": METRIC,
                     "tile_shapes": [{"lines": l_, "segment": s_, "order": ["largest_first", "list"][o_]}
                                     for (l_, s_, o_) in shapes],
                     "sweep_ms": ms[:ndim],
                     "roofline": {"bound": "hbm", "achieved": ach, "peak": peak_gbs, "unit": "GB/s",
                                  "frac": ach / peak_gbs, "kernel": f"batched sweep dir={'xyz'[dom]}"},
                     "step_hbm_frac": 24 * ndim * v32 / 1e9 / peak_gbs}
        del probs
    return res


def slab_bench(args):
    """One 2D grid split along y across the ranks (strong scaling): each rank
    a Solver over its slab with a halo of 2K rows, K steps per halo refresh
    (all-gather over NCCL), one step size agreed per period (all-reduce).
    value = cells of the whole grid x steps / the slowest rank's time."""
    import torch
    from paper_1805_08846_gb300 import Solver, inputs
    from paper_1805_08846_gb300 import slab as S
    rank, world, local_rank = dist_env()
    torch.cuda.set_device(local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    prob = inputs.sw_radial_dam_break(args.n)
    k = args.period
    layout = S.SlabLayout(prob.n[1], world, 2 * k, False)
    lp = S.local_problem(prob, layout, rank)
    solver = Solver.from_problem(lp, precision=32)
    seg = solver.autotune(2)
    steppers = {rank: S.solver_stepper(solver)}
    comm = S.DistComm() if world > 1 else S.LocalComm()
    S.run_steps(steppers, layout, comm, args.warmup, k)
    S.run_steps(steppers, layout, comm, args.steps, k)   # captures the graphs of the period lengths
    solver.set_q(lp.q0)
    S.run_steps(steppers, layout, comm, args.warmup, k)
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    info = S.run_steps(steppers, layout, comm, args.steps, k)
    torch.cuda.synchronize()
    barrier(world)
    el = max_over_ranks(time.perf_counter() - t0, world)
    solver.close()
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": prob.ncells * args.steps / el, "unit": METRIC,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"2D shallow water radial dam break {args.n}x{args.n} split into "
                                   f"{world} slabs along y, halo {2 * k} rows, {k} steps per refresh",
                       "parallelism": f"slab{world}", "segments": seg[:2],
                       "timing": "wall clock of the decomposed run: per period a halo refresh, a "
                                 "state snapshot and one graph of fixed steps (a speed pass before "
                                 "the first period only)"},
            "periods": info.periods, "redone": info.redone, "cfl_max_seen": info.cfl_max_seen}),
            flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def reference_arm(args):
    """The oracle as the reference arm: each step is the full step of the
    workload on a bounded subset of its lines (the x sweep on the first L rows
    and the y sweep on the first L columns), so K + W steps stay within a
    few minutes."""
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_1805_08846_gb300 import inputs
    prob = inputs.sw_radial_dam_break(args.n)
    o = oracle.Oracle(prob)
    q = prob.q0
    dt = 0.9 / o.max_speed_over_dx(q)
    N = args.n
    # calibrate L: one full-size sweep pair's cost per line
    t0 = time.perf_counter()
    qa, _ = o.sweep(0, q, dt, 0, 64)
    o.sweep(1, qa, dt, 0, 64)
    per_line = (time.perf_counter() - t0) / 64
    total_budget = 150.0
    steps_all = args.steps + args.warmup
    L = int(max(8, min(N, total_budget / max(steps_all * per_line, 1e-9))))
    for _ in range(args.warmup):
        qa, _ = o.sweep(0, q, dt, 0, L)
        o.sweep(1, qa, dt, 0, L)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        qa, _ = o.sweep(0, q, dt, 0, L)
        o.sweep(1, qa, dt, 0, L)
    el = time.perf_counter() - t0
    value = L * N * args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": METRIC,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"2D shallow water radial dam break {N}x{N}, Roe+HH, minmod, "
                               f"outflow, CFL 0.9", "global_batch": 1, "seq_len": N * N},
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": oracle.threads(),
                         "kind": "oracle",
                         "sample": f"x sweep on rows [0,{L}) and y sweep on columns [0,{L}) of "
                                   f"the {N}^2 grid per step, FP64 oracle"},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 plain-path timing")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the 3D acoustics and ensemble measurements")
    ap.add_argument("--n3", type=int, default=512)
    ap.add_argument("--steps3", type=int, default=20)
    ap.add_argument("--segments", default=None,
                    help="fixed FP32 segment lengths 'x,y' instead of the autotuner's")
    ap.add_argument("--paper-tables", action="store_true",
                    help="per-sweep times at the sizes of the paper's kernel tables (one JSON line)")
    ap.add_argument("--size-scaling", action="store_true",
                    help="cell-updates/s from 256^2 to 16384^2 (one JSON line)")
    ap.add_argument("--accuracy", action="store_true",
                    help="errors of every workload against the oracle, with times (one JSON line)")
    ap.add_argument("--decomp", default="replicas", choices=["replicas", "slab"],
                    help="replicas: every rank its own grid (weak scaling, the default); "
                         "slab: one grid split along y across the ranks (strong scaling)")
    ap.add_argument("--period", type=int, default=8, help="with --decomp slab: steps per halo refresh")
    ap.add_argument("--only-extra", default=None,
                    choices=["acoustics3d", "sw_bathymetry", "sw_dry", "sw_unsplit", "ensembles"],
                    help="run one extra measurement alone and print it")
    ap.add_argument("--fixed-segments", action="store_true",
                    help="with --paper-tables: 64-cell segments, no autotuning (for ncu)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return reference_arm(args)
    if args.decomp == "slab":
        return slab_bench(args)
    if args.only_extra:
        import torch
        torch.cuda.set_device(0)
        peak_gbs, _ = load_peaks()
        fn = {"acoustics3d": extra_acoustics3d, "sw_bathymetry": extra_bathymetry, "sw_dry": extra_dry,
              "sw_unsplit": extra_unsplit, "ensembles": extra_ensembles}[args.only_extra]
        print(json.dumps({args.only_extra: fn(args, peak_gbs)}), flush=True)
        return 0
    if args.paper_tables or args.size_scaling or args.accuracy:
        import torch
        torch.cuda.set_device(0)
        if args.paper_tables:
            if "--steps" not in sys.argv:
                args.steps = 20
            paper_tables(args)
        if args.size_scaling:
            size_scaling(args)
        if args.accuracy:
            accuracy(args)
        return 0

    rank, world, local = dist_env()
    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1805_08846_gb300 import Solver, inputs
    import paper_1805_08846_gb300._lib as L

    N = args.n
    prob = inputs.sw_radial_dam_break(N)
    ncell = prob.ncells
    peak_gbs, peak_kind = load_peaks()

    segs = {}

    def timed(precision):
        s = Solver.from_problem(prob, precision=precision, stream="torch")
        if precision == 32 and args.segments:
            segs[precision] = [int(v) for v in args.segments.split(",")][:2]
            for d, L_ in enumerate(segs[precision]):
                s.set_segment(d, L_)
        else:
            segs[precision] = s.autotune(4)           # tile shapes (state restored)
        # Untimed set-up: the CUDA graph of the timed call length is captured
        # once (like compilation), then the state and clock start over.
        s.run_steps(args.steps)
        s.set_q(prob.q0)
        s.set_time(0.0, 0.0, 0)
        s.run_steps(args.warmup)                      # warm-up steps: caches, clocks
        stream = torch.cuda.current_stream()
        rej0 = s.rejections()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        barrier(world)
        torch.cuda.synchronize()
        e0.record(stream)
        s.run_steps(args.steps)                       # the timed call: one graph replay
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        total_ms = max_over_ranks(e0.elapsed_time(e1), world)
        rej = s.rejections() - rej0
        # Per-kernel durations: a separate graph of the same steps with CUDA
        # events around every kernel (the events slow the graph a little, so
        # this pass gives the kernel breakdown, not the step rate).
        ms, prof_ms, _ = s.profile_steps(args.steps)
        s.close()
        # kernels of the timed call: the arming kernel, then per attempt
        # (kept steps and redone ones) two sweeps and the step control
        launches = 1 + (args.steps + rej) * 3
        return ms, total_ms, launches, prof_ms, rej

    clocks = ClockSampler(local)
    clocks.start()
    ms32, tot32, launches, prof32, rej32 = timed(32)
    clk = clocks.stop()
    value = world * ncell * args.steps / (tot32 * 1e-3)

    # Roofline of the dominant kernel: algorithmic bytes per launch =
    # 3 fields read + 3 written, 4 B each, per cell of the grid.
    bytes_per_launch = 6 * 4 * ncell
    dom = 0 if ms32[0] >= ms32[1] else 1
    achieved = bytes_per_launch / (ms32[dom] * 1e-3) / 1e9
    dom_kernel = f"sweep_kernel<ShallowWater<float>,minmod,dir={'xy'[dom]}>"
    traffic, traffic_src = traffic_record(dom_kernel, f"sw_dam_break_{N}")

    # End to end through the public API with pinned host buffers.
    q_host = torch.from_numpy(prob.q0).pin_memory()
    out_host = torch.empty_like(q_host).pin_memory()
    s = Solver.from_problem(prob, precision=32, stream="torch")
    for d, L_ in enumerate(segs[32][:2]):
        s.set_segment(d, L_)
    # untimed pass of the same calls (captures the graph of the timed call length)
    s.set_q(q_host)
    s.run_steps(args.steps)
    s.get_q(out_host)
    s.set_q(q_host)
    s.run_steps(args.warmup)
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    s.set_q(q_host)
    s.run_steps(args.steps)
    s.get_q(out_host)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    s.close()
    e2e_value = world * ncell * args.steps / e2e_s
    state_bytes = int(q_host.numel() * 8)

    fp64 = None
    if not args.no_fp64:
        ms64, tot64, _, _, _ = timed(64)
        fma64 = L.claw_probe_fma(64)
        dom64 = 0 if ms64[0] >= ms64[1] else 1
        ach64 = SW_FLOP_PER_CELL_SWEEP * ncell / (ms64[dom64] * 1e-3)
        fp64 = {"value": world * ncell * args.steps / (tot64 * 1e-3), "unit": METRIC,
                "ms_per_step": tot64 / args.steps,
                "sweep_ms": {"x": ms64[0], "y": ms64[1]},
                "roofline": {"bound": "alu", "achieved": ach64 / 1e12, "peak": fma64 / 1e12,
                             "unit": "TFLOP/s", "frac": ach64 / fma64,
                             "peak_kind": "measured FP64 FMA probe (claw_probe_fma)",
                             "flop_per_cell_sweep": SW_FLOP_PER_CELL_SWEEP,
                             "executed_dflop_per_cell_sweep": FP64_EXECUTED_DFLOP,
                             "executed_frac": FP64_EXECUTED_DFLOP * ncell / (ms64[dom64] * 1e-3) / fma64}}

    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()      # the rest is rank 0's single-GPU work
    extras = {}
    if not args.no_extras and rank == 0:
        for key, fn in (("acoustics3d", lambda: extra_acoustics3d(args, peak_gbs)),
                        ("sw_bathymetry", lambda: extra_bathymetry(args, peak_gbs)),
                        ("sw_dry", lambda: extra_dry(args, peak_gbs)),
                        ("sw_unsplit", lambda: extra_unsplit(args, peak_gbs)),
                        ("ensembles", lambda: extra_ensembles(args, peak_gbs))):
            try:
                extras[key] = fn()
            except Exception as exc:    # recorded, the main line still prints
                extras[key] = {"error": repr(exc)[:300]}

    if rank != 0:
        return 0
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot32 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"2D shallow water radial dam break {N}x{N}, Roe+HH, minmod, "
                               f"outflow, CFL 0.9, FP32 state (FP64 dt/time)",
                   "global_batch": world, "seq_len": ncell,
                   "parallelism": f"replicas{world}" if world > 1 else "single",
                   "l2": "inputs larger than L2 (201 MB per FP32 state version vs 129 MB L2)",
                   "timing": "CUDA events around one claw_run_steps call (one graph replay of all "
                             "steps; its graph captured in an untimed run first); per-kernel times "
                             "from a separate claw_profile_steps graph with events around each kernel",
                   "segments": {"f32": segs.get(32, [])[:2], "f64": segs.get(64, [])[:2]}},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak_gbs, "unit": "GB/s",
                     "frac": achieved / peak_gbs, "traffic": traffic,
                     "traffic_source": traffic_src, "algorithmic_bytes": bytes_per_launch,
                     "kernel": dom_kernel,
                     "peak_kind": f"{peak_kind} (copy)",
                     "sweep_ms": {"x": ms32[0], "y": ms32[1], "control": ms32[3]}},
        "e2e": {"value": e2e_value, "unit": METRIC, "h2d_bytes_per_step": state_bytes / args.steps,
                "d2h_bytes_per_step": state_bytes / args.steps},
        "gpu_launches": launches,
        "rejected_attempts": rej32,
        "kernel_breakdown_ms_per_step": prof32 / args.steps,
        "clocks": clk,
        "fp64_plain": fp64,
    }
    line.update(extras)
    if not args.no_cpu:
        rate, steps, threads, el = cpu_oracle_rate(prob)
        line["cpu_baseline"] = {"value": rate, "unit": METRIC, "cores": threads, "kind": "oracle",
                                "sample": f"{steps} full FP64 oracle steps of the {N}^2 grid "
                                          f"({el:.1f} s), {platform.machine()}"}
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
