#!/usr/bin/env python3
"""Benchmark: HFDIB steady-RANS SIMPLE sweep on one GB300 (sm_103a).

Workload: 2D immersed backward-facing step, h = 1, expansion 9/8, uniform
1024 x 256 grid over 30h x 9h, inlet plug U = 1 with I = 5 %, Re_h = 36000,
k-omega SST with immersed-boundary wall functions (synthetic lambda field
from the analytic step geometry).

A step is one extended SIMPLE sweep (Fig. simplehfdibrans: imposed fields,
momentum predictor, pressure corrector with multigrid-preconditioned CG,
flux/velocity update, omega and k transport), issued as one CUDA graph.
`value` = cell-updates/s = cells x timed sweeps / device time, with L2
flushed (a 512 MB write) between timed steps because the working set fits
in L2.  Also reported: converged solves/s to max scaled residual 1e-6, the
end-to-end rate through the public API from host arrays, the roofline of the
dominant kernel class, and the CPU oracle on the host cores.

Two more legs (rank 0): `batch` -- 16 NACA 0012 lambda fields (angles of
attack 0-15 deg, 2048 x 1024 each, k-omega SST, mixed precision) advanced
together by the batched persistent pressure launch, against the same designs
one at a time; `adjoint` -- channel designs with random smooth obstacles
(k-epsilon, 256 x 128 and 264 x 132) solved together to 1e-10, then the
frozen-turbulence adjoint gradient of the pressure drop per design.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--no-solve] [--no-cpu] [--no-batch] [--no-adjoint]
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SIMPLE cell-updates/s & solves/s to residual 1e-6 (% HBM roofline), mixed vs FP64"
WORKLOAD = "bfs_1024x256_sst"
NX, NY = 1024, 256
TOL = 1e-6
FREEZE = 300           # one-way y+ switch from sweep 300 (limit cycles otherwise)
P_RELTOL = 0.2         # per-sweep pressure tolerance on this workload (time to 1e-6:
                       # 0.1 -> 19.7 s, 0.2 -> 17.2 s mixed; 0.3 diverged); both legs use it
MAX_SOLVE_SWEEPS = 20000


def max_over_ranks(x, dist, device):
    """The job's time is its slowest rank's: the largest of a per-rank time
    over the process group (x itself on one rank)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(units_per_rank, world, seconds):
    """Whole-job throughput of `world` replicas that each process
    units_per_rank in `seconds` (the slowest rank's time)."""
    return world * units_per_rank / seconds


# Algorithmic bytes per cell for one launch group of each kernel class
# (2D, FP64 words of 8 B, minimum traffic with perfect neighbour reuse,
# face arrays counted as one word per cell and direction, flags 2 B).
def PCG_ITERS_FACTOR(piters):
    """The 'pcg' class is one launch of the whole pressure solve."""
    return max(float(piters.mean()), 1.0)


# DRAM bytes of one launch of the dominant kernel, from an ncu capture of this
# workload (dram__bytes_read.sum + dram__bytes_write.sum; mixed: the FP32
# V-cycle variant).  At 262k cells the pressure hierarchy stays in L2, so
# this is far below the algorithmic count.
TRAFFIC = {("pcg", "mixed"): 10.674176e6 + 1.420288e6, ("pcg", "fp64"): 12.108800e6 + 0.996608e6}

# FP64 flops of one launch of the FP64 assembly kernels on this workload
# (ncu: 2 x DFMA + DADD + DMUL thread instructions).  These kernels are bound
# by FP64 arithmetic, so their roofline is the FP64 rate.  Only the profiling
# classes that time exactly one kernel are listed.
FP64_FLOPS = {"mom_asm": 4.7356e7, "turb_final": 3.1783e7, "scal_asm": 1.5748e7}
FP64_PEAK_GFLOPS = 1250.0   # nominal GB300 FP64 rate (no measured FP64 peak is available)

BYTES_PER_CELL = {
    # u, v, p, nut, phi_x, phi_y, 4 gradient comps read; bm x2, u* x2 written
    "mom_asm": 8 * (10 + 4) + 2,
    # one colour: bm x2 (half the cells), u* x2, phi x2, nut read; u* x2 (half) written
    "mom_smooth": 8 * (1 + 2 + 2 + 1 + 1) + 2,
    # u*, bm x2, p, phi x2, nut read; HbyA x2, rAU, phiH x2 written
    "hbya": 8 * (7 + 5) + 2,
    "vcycle0": int(8 * 26 * 4 / 3),
    # phiH x2, pn, p, HbyA x2, rAU, cf x2 read; phi x2, u x2, p written
    "update": 8 * (9 + 5) + 2,
    "grad_u": 8 * (2 + 4) + 2,
    "turb_prep": 8 * (4 + 4 + 2 + 1 + 6) + 2,
    "scal_asm": 8 * (2 + 1 + 2 + 2 + 2) + 2,
    "scal_smooth": 8 * (1 + 1 + 2 + 1 + 1) + 2,
    "imposed": 8 * 8 + 2,
    "p_coef": 8 * (1 + 3),
    "turb_final": 8 * (5 + 4) + 2,
    "sweep_end": 0,
}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while timing."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- CPU oracle
def oracle_rate(seconds=15.0, min_sweeps=1, max_sweeps=1000):
    """Time the FP64 oracle sweeping the same workload on this host (one
    thread).  Run in a child process so the thread-count variables apply."""
    code = r"""
import json, sys, time
sys.path.insert(0, %r)
from paper_2606_06135_gb300 import geometry as G
from oracle import hfdib_oracle as O
case = G.case_bfs(%d, %d)
o = O.Oracle(case, dict(freeze_switch=%d))
n = 0; t0 = time.perf_counter()
while True:
    o.sweep(); n += 1
    el = time.perf_counter() - t0
    if (el >= %f and n >= %d) or n >= %d:
        break
print(json.dumps({"sweeps": n, "seconds": el, "cells": %d}))
""" % (ROOT, NX, NY, FREEZE, seconds, min_sweeps, max_sweeps, NX * NY)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if out.returncode != 0:
        raise RuntimeError("oracle run failed: " + out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def run_reference(args, rank):
    """Reference arm: the CPU oracle as it stands, on this host's cores; each
    step is one full-size oracle sweep of the same workload."""
    if rank != 0:
        return 0
    code = r"""
import json, sys, time
sys.path.insert(0, %r)
from paper_2606_06135_gb300 import geometry as G
from oracle import hfdib_oracle as O
case = G.case_bfs(%d, %d)
o = O.Oracle(case, dict(freeze_switch=%d))
for _ in range(%d):
    o.sweep()
t0 = time.perf_counter()
for _ in range(%d):
    o.sweep()
print(json.dumps({"seconds": time.perf_counter() - t0}))
""" % (ROOT, NX, NY, FREEZE, args.warmup, args.steps)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if out.returncode != 0:
        print(json.dumps({"impl": "reference", "unavailable": "oracle failed: " + out.stderr[-300:].replace("\n", " ")}))
        return 0
    sec = json.loads(out.stdout.strip().splitlines()[-1])["seconds"]
    value = NX * NY * args.steps / sec
    line = {"metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "grid": [NX, NY], "model": "komega_sst", "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
                             "sample": "%d full-size FP64 oracle sweeps after %d warm-up sweeps" % (args.steps, args.warmup)},
            "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- extra legs
NACA_NX, NACA_NY, NACA_AOAS = 2048, 1024, 16   # batched multi-lambda workload (16 angles of attack)
ADJ_DESIGNS = 2                                # random-obstacle designs for the adjoint leg


def _naca_case(aoa):
    """Geometry of one angle of attack (runs in a spawned worker)."""
    sys.path.insert(0, ROOT)
    from paper_2606_06135_gb300 import geometry as G
    return G.case_naca(NACA_NX, NACA_NY, aoa_deg=float(aoa))


def _grf_case(b):
    sys.path.insert(0, ROOT)
    from paper_2606_06135_gb300 import geometry as G
    nx, ny = G.grf_design_size(b)
    return G.case_grf(nx, ny, seed=b)


def batch_leg(hfdib, torch, cases, dev, steps, warmup):
    """B lambda fields advanced together (one batched persistent pressure
    launch per sweep) against the same designs solved one at a time."""
    N = sum(c["grid"]["nx"] * c["grid"]["ny"] for c in cases)
    bs = hfdib.BatchSolver(cases, device=str(dev), precision=1)
    bs.sweep(warmup, read=False)
    tune = bs.autotune(2)
    bs.sweep(2, read=False)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    bs.stream.synchronize()
    e0.record(bs.stream)
    bs.sweep(steps, read=False)
    e1.record(bs.stream)
    bs.stream.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    res = bs.sweep(1)
    bs.close()
    one = 0.0
    n1 = 0
    for c in cases[:2]:
        s = hfdib.Solver(c, device=str(dev), precision=1)
        s.sweep(warmup, read=False)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.stream.synchronize()
        a.record(s.stream)
        s.sweep(steps, read=False)
        b.record(s.stream)
        s.stream.synchronize()
        one += a.elapsed_time(b) / 1e3
        n1 += c["grid"]["nx"] * c["grid"]["ny"]
        s.close()
    return {"workload": "naca0012_%daoa_%dx%d_sst" % (len(cases), NACA_NX, NACA_NY), "designs": len(cases),
            "cells": N, "sweeps": steps, "value": N * steps / t, "unit": "cell-updates/s",
            "ms_per_batched_sweep": 1e3 * t / steps, "precision": "mixed",
            "one_by_one": {"designs": 2, "value": n1 * steps / one, "unit": "cell-updates/s"},
            "autotune": tune, "max_residual_after": float(max(res[:, :6].max(), 0.0)),
            "l2": "working set %.0f MB per field set > L2" % (N * 8 / 1e6)}


def adjoint_leg(hfdib, torch, cases, dev):
    """Designs solved together to 1e-10 (FP64), then one frozen-turbulence
    adjoint gradient dJ/dlambda (pressure drop) per design."""
    import time as _t
    N = sum(c["grid"]["nx"] * c["grid"]["ny"] for c in cases)
    bs = hfdib.BatchSolver(cases, device=str(dev), precision=0)
    t0 = _t.perf_counter()
    rc, its, res = bs.solve(tol=1e-10, max_iter=40000, check_every=100)
    torch.cuda.synchronize(dev)
    t_solve = _t.perf_counter() - t0
    per = []
    t_adj = 0.0
    for i in range(len(cases)):
        p = bs.problem(i)
        t0 = _t.perf_counter()
        J, g, passes, ch, arc = p.adjoint_grad(tol=1e-9, max_iter=40000)
        dt = _t.perf_counter() - t0
        t_adj += dt
        per.append({"grid": [cases[i]["grid"]["nx"], cases[i]["grid"]["ny"]], "J": J, "status": arc,
                    "transposed_sweeps": passes, "seconds": dt, "ms_per_transposed_sweep": 1e3 * dt / max(passes, 1),
                    "forward_sweeps": int(its[i])})
    bs.close()
    return {"workload": "grf_channel_keps_designs_%d" % len(cases), "cells": N, "solve_status": rc,
            "solve_tol": 1e-10, "adjoint_tol": 1e-9, "solve_seconds": t_solve, "adjoint_seconds": t_adj,
            "gradients_per_s": len(cases) / (t_solve + t_adj), "designs": per}


# ---------------------------------------------------------------- GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-solve", action="store_true", help="skip the converged-solve and e2e legs")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle leg")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched multi-lambda leg")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint leg")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank)

    # geometry of the extra legs, generated by spawned workers while the
    # GPU legs run (the pool starts before the first CUDA call)
    pool, fut_naca, fut_grf = None, [], []
    if rank == 0 and (not args.no_batch or not args.no_adjoint):
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        pool = ProcessPoolExecutor(max_workers=min(16, os.cpu_count() or 1), mp_context=mp.get_context("spawn"))
        if not args.no_batch:
            fut_naca = [pool.submit(_naca_case, a) for a in range(NACA_AOAS)]
        if not args.no_adjoint:
            fut_grf = [pool.submit(_grf_case, b) for b in range(ADJ_DESIGNS)]

    import numpy as np
    import torch
    from paper_2606_06135_gb300 import build as B
    from paper_2606_06135_gb300 import geometry as G
    from paper_2606_06135_gb300 import hfdib

    if not os.path.exists(hfdib.LIBPATH):
        B.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if dist is not None:
            dist.barrier()

    case = G.case_bfs(NX, NY)
    N = NX * NY
    peak, peak_kind = measured_peaks()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(dev)

    def timed_sweeps(precision):
        """W warm-up + K timed sweeps; L2 flushed between timed sweeps."""
        opts = dict(freeze_switch=FREEZE, p_reltol=P_RELTOL, precision=1 if precision == "mixed" else 0)
        s = hfdib.Solver(case, device=str(dev), stream=stream, **opts)
        for _ in range(args.warmup):
            s.sweep(1, read=False)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        clocks = ClockSampler(local)
        stream.synchronize()
        barrier()
        torch.cuda.synchronize(dev)
        clocks.start()
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(float(k))
            ev[k][0].record(stream)
            s.sweep(1, read=False)
            ev[k][1].record(stream)
        stream.synchronize()
        torch.cuda.synchronize(dev)
        barrier()
        clk = clocks.stop()
        t_dev = sum(a.elapsed_time(b) for a, b in ev) / 1e3
        hist = s.history(args.steps)
        piters = hist[:, 7]
        fixed, per_it = s.launch_counts()
        launches = int(args.steps * fixed + per_it * piters.sum())
        t_dev = max_over_ranks(t_dev, dist, dev)
        # roofline of the dominant kernel class (host-driven sweeps, event pairs)
        prof = s.profile(3)
        dname, (dus, dcalls) = max(prof.items(), key=lambda kv: kv[1][0])
        avg_us = dus / max(dcalls, 1)
        if dname == "pcg":
            # per CG iteration: FP64 CG vectors (13 words) + the V-cycle (26
            # words x 4/3 for the coarse levels) in the preconditioner's type
            wv = 4 if precision == "mixed" else 8
            bpc = (8 * (7 + 6) + int(wv * 26 * 4 / 3)) * PCG_ITERS_FACTOR(piters)
        else:
            bpc = BYTES_PER_CELL.get(dname, 0)
        achieved = bpc * N / (avg_us * 1e-6) / 1e9
        total = sum(x[0] for x in prof.values())
        traffic = TRAFFIC.get((dname, precision))
        roof = {"bound": "hbm", "kernel": dname, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_kind, "traffic": traffic,
                "traffic_note": "ncu DRAM bytes of one launch; the pressure hierarchy is L2-resident at this size"
                if traffic else None,
                "algorithmic_bytes_per_launch": bpc * N, "avg_launch_us": avg_us,
                "class_share": {k: round(v[0] / total, 4) for k, v in prof.items()}}
        # FP64-ALU roofline of the assembly classes (live event timing)
        alu = {}
        for cls, fl in FP64_FLOPS.items():
            if cls in prof and prof[cls][1] > 0:
                us = prof[cls][0] / prof[cls][1]
                gf = fl / (us * 1e-6) / 1e9
                alu[cls] = {"achieved": gf, "avg_launch_us": us, "flops_per_launch": fl}
        top = max(alu, key=lambda c: prof[c][0]) if alu else None
        roof_alu = None
        if top:
            roof_alu = {"bound": "alu", "kernel": top, "achieved": alu[top]["achieved"], "peak": FP64_PEAK_GFLOPS,
                        "unit": "GFLOP/s (FP64)", "frac": alu[top]["achieved"] / FP64_PEAK_GFLOPS,
                        "peak_source": "nominal", "per_class": alu}
        s.close()
        return dict(value=replica_rate(N * args.steps, world, t_dev), ms=1e3 * t_dev / args.steps, clocks=clk,
                    launches=launches, piters=float(piters.mean()), roofline=roof, roofline_alu=roof_alu)

    res = {p: timed_sweeps(p) for p in ("mixed", "fp64")}
    head = res["mixed"]
    out = {"metric": METRIC, "value": head["value"], "unit": "cell-updates/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32+f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "grid": [NX, NY], "cells": N, "model": "komega_sst",
                      "Re_h": 36000, "precision": "mixed (FP32 inner sweeps + FP32 multigrid, FP64 defects)",
                      "l2": "flushed (512 MB write) between timed steps",
                      "parallelism": "replicas" if world > 1 else "single",
                      "freeze_switch": FREEZE, "p_reltol": P_RELTOL, "pcg_iters_mean": head["piters"]},
           "gpu_launches": head["launches"], "clocks": head["clocks"], "roofline": head["roofline"],
           "roofline_alu": head["roofline_alu"],
           "fp64": {"value": res["fp64"]["value"], "ms_per_step": res["fp64"]["ms"],
                    "roofline": res["fp64"]["roofline"], "roofline_alu": res["fp64"]["roofline_alu"],
                    "clocks": res["fp64"]["clocks"],
                    "pcg_iters_mean": res["fp64"]["piters"]}}


    # converged solves (both precisions) and the end-to-end leg (mixed, public
    # API from host arrays)
    def solve_leg(precision, e2e):
        o = dict(freeze_switch=FREEZE, p_reltol=P_RELTOL, precision=1 if precision == "mixed" else 0)
        lam_h = torch.from_numpy(np.ascontiguousarray(case["lam"])).pin_memory()
        yw_h = torch.from_numpy(np.ascontiguousarray(case["ywall"])).pin_memory()
        barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            lam_d = lam_h.to(dev, non_blocking=True)
            yw_d = yw_h.to(dev, non_blocking=True)
        s2 = hfdib.Solver(dict(case, lam=lam_d, ywall=yw_d), device=str(dev), stream=stream, **o)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc, iters, r = s2.solve(tol=TOL, max_iter=MAX_SOLVE_SWEEPS, check_every=100)
        e1.record(stream)
        host = {n: s2.field(n).cpu() for n in ("ux", "uy", "p", "k", "omega")}
        torch.cuda.synchronize(dev)
        t_wall = time.perf_counter() - t0
        t_solve = e0.elapsed_time(e1) / 1e3
        s2.close()
        barrier()
        t_wall = max_over_ranks(t_wall, dist, dev)
        t_solve = max_over_ranks(t_solve, dist, dev)
        conv = rc == 0
        leg = {"converged": conv, "sweeps": iters, "seconds": t_solve,
               "solves_per_s": replica_rate(1, world, t_solve) if conv else 0.0,
               "final_max_residual": float(max(r[:6])), "tol": TOL}
        if e2e:
            d2h = sum(v.numel() * 8 for v in host.values()) + 8 * hfdib.NRES * ((iters + 99) // 100)
            leg["e2e"] = {"value": replica_rate(N * iters, world, t_wall), "unit": "cell-updates/s",
                          "h2d_bytes_per_step": 2 * N * 8, "d2h_bytes_per_step": d2h,
                          "step": "host lambda/ywall -> create (IB geometry) -> solve to 1e-6 -> host fields",
                          "solves_per_s": replica_rate(1, world, t_wall) if conv else 0.0}
        return leg

    if not args.no_solve:
        lm = solve_leg("mixed", True)
        lf = solve_leg("fp64", False)
        out["solves_per_s"] = lm["solves_per_s"]
        out["e2e"] = lm.pop("e2e")
        out["solve"] = lm
        out["fp64"]["solve"] = lf
        out["fp64"]["solves_per_s"] = lf["solves_per_s"]
    if rank == 0 and fut_naca:
        out["batch"] = batch_leg(hfdib, torch, [f.result() for f in fut_naca], dev, args.steps, args.warmup)
    if rank == 0 and fut_grf:
        out["adjoint"] = adjoint_leg(hfdib, torch, [f.result() for f in fut_grf], dev)
    if pool is not None:
        pool.shutdown()
    if rank == 0 and not args.no_cpu:
        r = oracle_rate(seconds=15.0)
        out["cpu_baseline"] = {"value": r["cells"] * r["sweeps"] / r["seconds"], "unit": "cell-updates/s",
                               "cores": 1, "kind": "oracle",
                               "sample": "%d full-size FP64 oracle sweeps of the same workload" % r["sweeps"]}
    if rank == 0:
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
