"""Benchmark: fine DOF-substeps/s of the two-level LPBF heat solve on GB300.

One step = one macro step of Algorithm 1 (predictor, m fine micro steps,
restriction, correction) of the 10 x 5 x 2 mm multi-track workload (80x40x16
coarse hexes, 65x65x33-node fine patch, m = 8); the default K = 500 steps is
the first quarter of the 2000-step, 10-track scan.  Metric: fine DOF-substeps/s = fine patch nodes x micro steps
solved / time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (torchrun, one rank per GPU): N independent replicas of the workload,
no collective on the data path (the patch solve does not shard); value = the
work of all ranks / the slowest rank's time.  --impl reference times the FP64
CPU oracle on a bounded sample of the same workload (rank 0 only).
"""
from __future__ import annotations

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

from paper_2110_12932_gb300 import ranks, workloads  # noqa: E402

WORKLOAD = "multitrack_10mm"
METRIC = "fine DOF-substeps/s"
FLOPS_APPLY_PER_ELEM = 65   # Hadamard-factored matrix-free apply, FP64 flops per element
FLOPS_VEC_PER_NODE = 14     # PCG vector update, fused dots, p = z + beta p
# dram__bytes_read.sum + dram__bytes_write.sum of one FP64 fine micro-step launch of
# this workload, from the ncu capture summarised in
# profiles/solve_kernel_fp64_multitrack_10mm.md (the patch is L2-resident)
FINE_LAUNCH_DRAM_BYTES = 3.026432e6 + 1.040640e6


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mode", default="plain", choices=["plain", "batch", "serve", "roofline"],
                    help="plain: the 10 mm multi-track plate (FP64 headline + precision form); "
                         "batch: 64 uneven jobs in the batched FP32-refined form")
    ap.add_argument("--jobs", type=int, default=64)
    ap.add_argument("--rate", type=float, default=2.0, help="serve: arrivals per second")
    ap.add_argument("--duration", type=float, default=30.0, help="serve: seconds of arrivals")
    ap.add_argument("--mem-cap-gb", type=float, default=120.0)
    ap.add_argument("--launches-per-round", type=int, default=10)
    ap.add_argument("--coupling-sweeps", type=int, default=1,
                    help="plain: corrections of the iterated two-level coupling per macro step (1 = one pass)")
    ap.add_argument("--latent", type=float, default=0.0,
                    help="plain: latent heat of fusion [J/kg] (0 = none; Ti64-like 2.86e5)")
    ap.add_argument("--picard", type=int, default=1,
                    help="plain: Picard iterations per backward-Euler step (1 = coefficients lagged)")
    ap.add_argument("--inner-tiles", type=int, default=0, choices=[0, 1, 2],
                    help="batch / serve: tiling of the FP32 inner CG (0 by mesh size, 1 element tiles, 2 wide tiles)")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(n_gpus):
    return ranks.init("nccl")


barrier = ranks.barrier
max_over_ranks = ranks.max_over_ranks
sum_over_ranks = ranks.sum_over_ranks


def fine_nodes(cfg):
    return workloads.fine_nodes(cfg)


def oracle_solves(o):
    """The oracle's Algorithm-1 sequence one solve at a time: yields "coarse"
    or "fine" after each solve."""
    while True:
        o.predict()
        yield "coarse"
        for i in range(o.m):
            o.fine_substep(i)
            yield "fine"
        o.restrict_and_correct()
        o.n += 1
        yield "coarse"


def oracle_sample(cfg, budget_s, max_solves=None, warmup=0):
    """Times the oracle solve by solve through the workload's sequence until
    the budget is spent (with at least one coarse and one fine solve done) and
    scales the mean solve times to one macro step (2 coarse + m fine solves):
    returns (fine DOF-substeps/s, solves, coarse solves, fine solves, seconds)."""
    import time as _t

    from oracle import twolevel as TL
    o = TL.TwoLevel(cfg, energy=False)
    seq = oracle_solves(o)
    for _ in range(warmup):
        next(seq)
    tc = tf = 0.0
    nc = nf = 0
    t_all = _t.perf_counter()
    while True:
        t0 = _t.perf_counter()
        kind = next(seq)
        dt = _t.perf_counter() - t0
        if kind == "coarse":
            tc, nc = tc + dt, nc + 1
        else:
            tf, nf = tf + dt, nf + 1
        done = nc + nf
        if nc and nf and (_t.perf_counter() - t_all > budget_s or (max_solves and done >= max_solves)):
            break
    m = cfg["m"]
    t_macro = 2 * tc / nc + m * tf / nf
    return m * fine_nodes(cfg) / t_macro, done, nc, nf, _t.perf_counter() - t_all


def cpu_baseline(cfg, budget_s=20.0):
    """The oracle as it stands on a bounded sample of the same workload."""
    val, done, nc, nf, dt = oracle_sample(cfg, budget_s)
    return {"value": val, "unit": METRIC, "cores": 1, "kind": "oracle",
            "sample": f"first {done} solves of {cfg['name']} ({nc} coarse, {nf} fine), single-threaded SciPy, "
                      f"{dt:.1f} s, mean solve times scaled to a macro step (2 coarse + {cfg['m']} fine); "
                      f"host has {os.cpu_count()} cores"}


def run_reference(args):
    """The oracle on the same workload: a step is one solve of its Algorithm-1
    sequence (coarse predictor / corrector or fine micro step); the value
    scales the mean coarse and fine solve times to a macro step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cfg = workloads.workload(args.workload)
    budget = 120.0
    t_start = time.perf_counter()
    warm = max(0, min(args.warmup, 1))
    val, done, nc, nf, dt = oracle_sample(cfg, budget, max_solves=max(2, args.steps), warmup=warm)
    sample = (f"{done} solves of {cfg['name']} ({nc} coarse, {nf} fine) after {warm} warm-up solve, "
              f"single-threaded FP64 SciPy oracle, {dt:.1f} s (time-capped at {budget:.0f} s), mean solve "
              f"times scaled to a macro step (2 coarse + {cfg['m']} fine)")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "DOF-substeps/s",
            "n_gpus": args.gpus, "steps": done, "warmup": warm,
            "ms_per_step": 1e3 * dt / max(done, 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": cfg["name"], "fine_nodes": fine_nodes(cfg), "m": cfg["m"],
                       "step": "one oracle solve"},
            "cpu_baseline": {"value": val, "unit": "DOF-substeps/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": "DOF-substeps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t_start}
    print(json.dumps(line), flush=True)
    return 0


def l2_flush(buf):
    buf.fill_(1.0)


def timed_run(tl, torch, cfg, K, sp, stream, flush, sample_every=50):
    """K macro steps of a fresh problem, each bracketed by CUDA events on the
    library's stream, L2 flushed between steps outside the events; every
    `sample_every`-th macro step also times each fine launch separately."""
    m = cfg["m"]
    prob = tl.Problem(cfg, stream=sp)
    st0 = prob.stats()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    fine_ev = []
    for k in range(K):
        l2_flush(flush)
        ev[k][0].record(stream)
        prob.predict()
        for i in range(m):
            if k % sample_every == 0:
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                prob.fine_substeps(1)
                b.record(stream)
                fine_ev.append((a, b))
            else:
                prob.fine_substeps(1)
        prob.restrict()
        prob.correct()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    status = prob.sync()
    if status != 0:
        raise RuntimeError(f"device status {status}")
    dev_ms = sum(a.elapsed_time(b) for a, b in ev)
    st = prob.stats()
    st["launches"] -= st0["launches"]
    fine_ms = [a.elapsed_time(b) for a, b in fine_ev]
    Tf, _ = prob.temperature(tl.TL_FINE)
    Tc, _ = prob.temperature(tl.TL_COARSE)
    sf = prob.state(tl.TL_FINE)
    prob.close()
    return dev_ms, fine_ms, st, Tf, Tc, sf


def fine_flops(cfg, iters_per_launch):
    r = cfg["r"]
    ne = (cfg["pNXc"] * r) * (cfg["pNYc"] * r) * (cfg["pNZc"] * r)
    nfn = fine_nodes(cfg)
    return iters_per_launch * (FLOPS_APPLY_PER_ELEM * ne + FLOPS_VEC_PER_NODE * nfn) + 2 * FLOPS_APPLY_PER_ELEM * ne


def run_ours(args):
    import numpy as np
    import torch

    from paper_2110_12932_gb300 import build as tlbuild
    from paper_2110_12932_gb300 import tl

    rank, ws, local = dist_setup(args.gpus)
    tlbuild.build()
    tl.load()
    form = dict(coupling_sweeps=args.coupling_sweeps, latent=args.latent, picard_iters=args.picard)
    cfg = workloads.workload(args.workload, precision=0, tol=1e-12, **form)
    cfg_ref = workloads.workload(args.workload, precision=1, tol=1e-10, tol_inner=1e-5, **form)
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    nfn = fine_nodes(cfg)
    m = cfg["m"]
    r = cfg["r"]
    ne = (cfg["pNXc"] * r) * (cfg["pNYc"] * r) * (cfg["pNZc"] * r)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2
    K = args.steps

    # warm-up on throw-away problems
    for c in (cfg, cfg_ref):
        wp = tl.Problem(c, stream=sp)
        for _ in range(args.warmup):
            wp.macro_steps(1)
        wp.close()

    clocks = ClockSampler(local)
    barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    t_wall = time.perf_counter()
    dev_ms, fine_ms, st, Tf64, Tc64, sf64 = timed_run(tl, torch, cfg, K, sp, stream, flush)
    wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    barrier(ws)
    dev_ms = max_over_ranks(dev_ms, ws)
    work = sum_over_ranks(K * m * nfn, ws)
    value = work / (dev_ms / 1e3)
    fine_iters = st["cg_iters_fine"] / max(1, st["solves_fine"])
    launch_s = statistics.mean(fine_ms) / 1e3
    picard = max(1, args.picard)  # solves per fine micro step; fine_ms times the whole micro step
    achieved = picard * fine_flops(cfg, fine_iters) / launch_s / 1e12
    peak = FP64_PEAK_TFLOPS   # FP64 FMA: 2 DFMA/clk/SM = 4 flop/clk/SM at 2.07 GHz
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": FINE_LAUNCH_DRAM_BYTES,
                "kernel": "tl::solve_kernel (FP64 fine micro step)",
                "launch_ms": statistics.mean(fine_ms), "cg_iters_per_launch": fine_iters,
                "flops_per_launch": picard * fine_flops(cfg, fine_iters),
                "peak_note": "FP64 pipe, derived: 152 SMs x 4 flop/clk x 2.07 GHz; a DFMA loop measured 1.20 TFLOP/s. "
                             "Counts the FP64 flops of the apply (65 per element) and of the vector work (14 per node) "
                             "per CG iteration; the FP32 preconditioner filter is not counted"}

    # ---- the precision form on the same workload (FP32 inner CG, FP64 defect correction)
    barrier(ws)
    dev_ms_r, fine_ms_r, st_r, Tf32, Tc32, sf32 = timed_run(tl, torch, cfg_ref, K, sp, stream, flush)
    dev_ms_r = max_over_ranks(dev_ms_r, ws)
    value_r = work / (dev_ms_r / 1e3)
    refined = {
        "value": value_r, "unit": "DOF-substeps/s", "ms_per_step": dev_ms_r / K, "speedup_vs_fp64": value_r / value,
        "tol": cfg_ref["tol"], "tol_inner": cfg_ref["tol_inner"],
        "rel_l2_vs_fp64": {"fine": float(np.linalg.norm(Tf32 - Tf64) / np.linalg.norm(Tf64)),
                           "coarse": float(np.linalg.norm(Tc32 - Tc64) / np.linalg.norm(Tc64))},
        "melt_mask_agreement": float(np.mean((sf32 == tl.MELTED) == (sf64 == tl.MELTED))),
        "fine_launch_ms": statistics.mean(fine_ms_r),
        "inner_iters_per_solve": st_r["cg_iters_fine"] / max(1, st_r["solves_fine"]),
        "outer_iters_per_solve": st_r["outer_iters_fine"] / max(1, st_r["solves_fine"]),
        "gpu_launches": int(sum_over_ranks(st_r["launches"], ws)),
    }

    # ---- end to end through the public API: create, K steps, host read-back each step
    torch.cuda.synchronize()
    barrier(ws)
    t0 = time.perf_counter()
    p2 = tl.Problem(cfg, stream=sp)
    host = None
    for k in range(K):
        p2.macro_steps(1)
        host, _ = p2.temperature(tl.TL_FINE)
    p2.close()
    e2e_s = max_over_ranks(time.perf_counter() - t0, ws)
    e2e = {"value": work / e2e_s, "unit": "DOF-substeps/s", "h2d_bytes_per_step": 0,
           "d2h_bytes_per_step": int(host.nbytes), "wall_s": e2e_s,
           "note": "tl_create_problem + per step tl_macro_steps(1) + tl_get_temperature(fine) into a host buffer; "
                   "step inputs (laser positions, weights) travel as launch parameters"}

    launches = int(sum_over_ranks(st["launches"], ws))
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline and ws == 1:
            cpu = cpu_baseline(cfg)
        line = {"metric": METRIC, "value": value, "unit": "DOF-substeps/s", "n_gpus": ws, "steps": K,
                "warmup": args.warmup, "ms_per_step": dev_ms / K, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": cfg["name"], "fine_nodes": nfn, "fine_elements": ne,
                           "coarse_nodes": (cfg["NXc"] + 1) * (cfg["NYc"] + 1) * (cfg["NZc"] + 1),
                           "m": m, "r": r, "tol": cfg["tol"], "precision": "fp64",
                           "coupling_sweeps": args.coupling_sweeps, "latent": args.latent,
                           "picard_iters": args.picard,
                           "parallelism": f"replicas{ws}" if ws > 1 else "single",
                           "l2": "flushed (256 MB write) between timed macro steps, outside the events"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk, "wall_s": wall,
                "coupling_resolves_per_step": st.get("coupling_resolves", 0) / max(1, K),
                "cg_iters": {"fine_per_solve": fine_iters,
                             "coarse_per_solve": st["cg_iters_coarse"] / max(1, st["solves_coarse"])},
                "fp32_refined": refined}
        print(json.dumps(line), flush=True)
    ranks.finish(ws)
    return 0


def run_batch(args):
    """64 independent seeded jobs (2-8 mm plates, 32^3 ... 96x96x48 fine
    patches, r = m in {4, 8}) advanced together in the batched FP32-refined
    form until every job finished its scan; compared with the same jobs run
    one at a time on the plain FP64 path (a timed sample of each job's first
    macro steps, extrapolated to its full scan)."""
    import torch

    from paper_2110_12932_gb300 import build as tlbuild
    from paper_2110_12932_gb300 import tl

    rank, ws, local = dist_setup(args.gpus)
    tlbuild.build()
    tl.load()
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    # jobs are dealt round-robin to the ranks (no exchange between them)
    jobs = ranks.deal(workloads.batch_jobs(args.jobs), rank, ws)
    for j in jobs:
        j.update(precision=1, tol=1e-10, tol_inner=1e-5, inner_tiles=args.inner_tiles)
    work = sum(fine_nodes(j) * j["m"] * j["macro_steps"] for j in jobs)

    # warm-up: one short batch
    wb = tl.Batch(launches_per_round=args.launches_per_round, max_jobs=len(jobs), stream=sp)
    wps = [tl.Problem(j, stream=sp) for j in jobs[:8]]
    for p in wps:
        wb.add(p, 1)
    wb.run()
    wb.close()
    for p in wps:
        p.close()

    probs = [tl.Problem(j, stream=sp) for j in jobs]
    batch = tl.Batch(launches_per_round=args.launches_per_round, max_jobs=len(jobs), stream=sp)
    for p, j in zip(probs, jobs):
        batch.add(p, j["macro_steps"])
    clocks = ClockSampler(local)
    barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record(stream)
    rounds = []
    while batch.jobs:
        ra, rb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ra.record(stream)
        act = batch.round()
        rb.record(stream)
        rounds.append((act, ra, rb))
        batch.poll()
    e1.record(stream)
    torch.cuda.synchronize()
    by_active = {}
    for act, ra, rb in rounds:
        k = "1" if act <= 1 else ("2-8" if act <= 8 else ("9-32" if act <= 32 else "33+"))
        c, ms = by_active.get(k, (0, 0.0))
        by_active[k] = (c + 1, ms + ra.elapsed_time(rb))
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    dev_s = max_over_ranks(e0.elapsed_time(e1) / 1e3, ws)
    info = batch.info()
    stats = [p.stats() for p in probs]
    status = [p.sync() for p in probs]
    batch.close()
    for p in probs:
        p.close()
    total_work = sum_over_ranks(work, ws)
    launches = int(sum_over_ranks(info["launches"], ws))
    # plain FP64 one at a time: time each job's first macro steps alone
    sample_steps = 3
    alone_s = 0.0
    alone_work = 0
    for j in jobs:
        c = dict(j, precision=0, tol=1e-12)
        p = tl.Problem(c, stream=sp)
        p.macro_steps(1)  # warm
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(sample_steps):
            p.predict()
            p.fine_substeps(c["m"])
            p.restrict()
            p.correct()
        b.record(stream)
        torch.cuda.synchronize()
        alone_s += a.elapsed_time(b) / 1e3 * (j["macro_steps"] / sample_steps)
        alone_work += fine_nodes(j) * j["m"] * j["macro_steps"]
        p.close()
    if rank == 0:
        line = {"metric": METRIC, "value": total_work / dev_s, "unit": "DOF-substeps/s", "n_gpus": ws,
                "steps": info["launches"], "warmup": 1, "ms_per_step": 1e3 * dev_s / max(1, info["launches"]),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
                "data": "synthetic",
                "config": {"workload": f"batch_jobs({args.jobs}, seed 20211025)", "jobs": len(jobs),
                           "fine_dof_substeps": total_work, "precision": "fp32_refined", "tol": 1e-10,
                           "launches_per_round": args.launches_per_round,
                           "inner_tiles": args.inner_tiles,
                           "step": "one batched cooperative launch (each job's next solve)"},
                "gpu_launches": launches, "clocks": clk, "wall_s": wall,
                "all_ok": all(s == 0 for s in status),
                "rounds_by_active_jobs": {k: {"rounds": c, "ms": ms} for k, (c, ms) in by_active.items()},
                "cg_iters_fine_per_solve": sum(s["cg_iters_fine"] for s in stats) / max(1, sum(s["solves_fine"] for s in stats)),
                "plain_fp64_one_at_a_time": {
                    "value": alone_work / alone_s, "unit": "DOF-substeps/s",
                    "sample": f"first {sample_steps} macro steps of each job alone (after 1 warm-up), FP64 tol 1e-12, "
                              "extrapolated linearly to each job's scan"},
                "speedup_vs_plain_fp64": (total_work / dev_s) / (alone_work / alone_s)}
        print(json.dumps(line), flush=True)
    ranks.finish(ws)
    return 0


def fp64_service_estimate(tl, torch, cfg, sp, stream, sample_steps=2):
    """Seconds the plain FP64 path needs for the whole job alone: its first
    macro steps timed on the device, extrapolated to the job's scan."""
    c = dict(cfg, precision=0, tol=1e-12)
    p = tl.Problem(c, stream=sp)
    p.macro_steps(1)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    p.macro_steps(sample_steps)
    b.record(stream)
    torch.cuda.synchronize()
    p.close()
    return a.elapsed_time(b) / 1e3 * c["macro_steps"] / sample_steps


def run_serve(args):
    """Poisson stream of jobs (batch_jobs shapes plus 10 % of the 20 mm plate
    truncated to 200 macro steps), admitted by free slots and a device-memory
    budget, served by continuous batching; compared with serving the same
    arrivals one job at a time, first come first served, on the plain FP64
    path (service times from timed samples)."""
    import numpy as np
    import torch

    from paper_2110_12932_gb300 import build as tlbuild
    from paper_2110_12932_gb300 import serve, tl

    rank, ws, local = dist_setup(args.gpus)
    tlbuild.build()
    tl.load()
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    arrivals = ranks.deal(workloads.serving_arrivals(args.rate, args.duration), rank, ws)
    for _, c in arrivals:
        c["inner_tiles"] = args.inner_tiles
    work = sum(fine_nodes(c) * c["m"] * c["macro_steps"] for _, c in arrivals)
    srv = serve.Server(mem_cap_bytes=args.mem_cap_gb * 1e9, max_jobs=256,
                       launches_per_round=args.launches_per_round, stream=sp)
    wt = workloads.batch_jobs(2)
    for c in wt:  # warm-up
        c["macro_steps"] = 1
    srv.run([(0.0, c) for c in wt])
    clocks = ClockSampler(local)
    barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    rep = srv.run(arrivals)
    clk = clocks.stop()
    srv.close()
    # one at a time on the plain FP64 path: service time per distinct shape
    cache = {}
    service = []
    for _, c in arrivals:
        key = (c["name"].startswith("serve_large"), c["NXc"], c["NYc"], c["NZc"], c["pNXc"], c["pNYc"],
               c["pNZc"], c["r"], c["macro_steps"])
        if key not in cache:
            cache[key] = fp64_service_estimate(tl, torch, c, sp, stream)
        service.append(cache[key])
    fifo = serve.fifo_one_at_a_time(arrivals, service)
    value = ranks.aggregate_rate(rep["fine_dof_substeps"], rep["busy_s"], ws)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "DOF-substeps/s", "n_gpus": ws,
                "steps": rep["rounds"], "warmup": 1, "ms_per_step": 1e3 * rep["busy_s"] / max(1, rep["rounds"]),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
                "data": "synthetic",
                "config": {"workload": "serving_arrivals", "rate_per_s": args.rate, "duration_s": args.duration,
                           "jobs": len(arrivals), "large_jobs": sum(c["name"].startswith("serve_large")
                                                                  for _, c in arrivals),
                           "mem_cap_gb": args.mem_cap_gb, "precision": "fp32_refined", "tol": 1e-10,
                           "step": "one batch round", "offered_dof_substeps": work},
                "job_latency_s": rep["job_latency_s"], "coarse_step_latency_ms": rep["coarse_step_latency_ms"],
                "wall_s": rep["wall_s"], "busy_s": rep["busy_s"], "peak_admitted_gb": rep["peak_admitted_bytes"] / 1e9,
                "all_ok": rep["all_ok"], "clocks": clk,
                "plain_fp64_one_at_a_time": {
                    "throughput": work / sum(service),
                    "job_latency_s": {"p50": float(np.percentile(fifo, 50)), "p99": float(np.percentile(fifo, 99))},
                    "sample": "service time per job shape from its first 2 macro steps alone (FP64, tol 1e-12), "
                              "extrapolated; first come first served"}}
        print(json.dumps(line), flush=True)
    ranks.finish(ws)
    return 0


# Algorithmic bytes per node of one CG iteration of the default form (the
# tensor-preconditioned CG, three phases; elements ~ nodes):
#  update: reads r, q, x, u, p, s (solve precision) and sq (FP32), writes
#   p, s, r, x (solve precision) and v (FP32); exchange partials on tile faces
#   are not counted;
#  preconditioner: reads v and sq (FP32) and r, writes u (solve precision);
#   the v halo comes from L2 and is not counted;
#  apply: FP32 on wide tiles reads u and two element coefficients and writes
#   the partial q; FP64 on element tiles reads u and eight FP64 eigenvalues
#   per element and writes q.
UPDATE_BYTES = {"fp32": 12 * 4, "fp64": 10 * 8 + 2 * 4}
PRECOND_BYTES = {"fp32": 4 * 4, "fp64": 2 * 4 + 2 * 8}
APPLY_BYTES = {"fp32": 4 * 4, "fp64": 2 * 8 + 8 * 8}
# FP64 flops of the FP64 form's phases (the FP32 preconditioner filter runs on
# the FP32 pipe and is not counted): update 5 FMA per node, <r,u> 1 FMA per
# node, apply FLOPS_APPLY_PER_ELEM per element plus <w,u>.
UPDATE_FLOPS_FP64 = 10
PRECOND_FLOPS_FP64 = 2
HBM_GBS = 6688.8  # measured copy bandwidth of this GB300 (read + write bytes)
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12


def run_roofline(args):
    """A 256 x 256 x 128-element fine patch (8.5M nodes; 32 x 32 x 16 coarse
    elements refined 8x, plate 40 x 40 x 20 coarse): one micro step in each
    precision, per-phase times of the CG iterations from the device phase
    tracer (block 0's view: a phase ends when the grid barrier after it is
    passed)."""
    import torch

    from paper_2110_12932_gb300 import build as tlbuild
    from paper_2110_12932_gb300 import tl

    tlbuild.build()
    tl.load()
    base = workloads.workload("multitrack_10mm", Lx=5e-3, Ly=5e-3, Lz=2.5e-3, NXc=40, NYc=40, NZc=20,
                              pNXc=32, pNYc=32, pNZc=16, r=8, m=8,
                              tracks=[(1e-3, 2.5e-3, 4e-3, 2.5e-3, 0.8)])
    nn = fine_nodes(base)
    ne = 256 * 256 * 128
    out = {}
    names = {v: k for k, v in tl.TRACE_MARKS.items()}
    for prec in ("fp32", "fp64"):
        cfg = dict(base, precision=1 if prec == "fp32" else 0, tol=1e-10 if prec == "fp32" else 1e-12)
        p = tl.Problem(cfg)
        p.macro_steps(1)           # warm-up macro step
        p.predict()
        p.fine_substeps(1)
        torch.cuda.synchronize()
        ev = [e for e in p.trace(tl.TL_FINE) if e[0] not in (names["rr_value"], names["breakdown_value"])]
        p.close()
        launch = (ev[-1][1] - ev[0][1]) / 1e9
        ends = [b for (m, b) in ev if m == names["cg_pass"]]
        t = statistics.median([(y - x) / 1e9 for x, y in zip(ends, ends[1:])]) if len(ends) > 1 else float("nan")
        seg = {}
        for (m0, a), (m1, b) in zip(ev, ev[1:]):
            seg.setdefault((m0, m1), []).append((b - a) / 1e9)

        def med(a, b):
            return statistics.median(seg[(names[a], names[b])])

        tu = med("cg_pass", "cg_u_start") + med("cg_u_start", "cg_u_end") + med("cg_u_end", "cg_update")
        tp = med("cg_update", "cg_precond")
        ta = med("cg_precond", "cg_apply") + med("cg_apply", "cg_pass")
        bu, bp, ba = UPDATE_BYTES[prec] * nn, PRECOND_BYTES[prec] * nn, APPLY_BYTES[prec] * nn

        def phase(us, byt):
            return {"us": 1e6 * us, "bytes": byt, "GBps": byt / us / 1e9, "frac_of_measured_hbm": byt / us / 1e9 / HBM_GBS}

        o = {"launch_ms": 1e3 * launch, "cg_iterations": len(ends), "iteration_us": 1e6 * t,
             "scheme": "tensor-preconditioned CG, three phases; apply on "
                       + ("wide tiles" if prec == "fp32" else "element tiles"),
             "update_phase": dict(phase(tu, bu), block0_share_us=1e6 * med("cg_u_start", "cg_u_end"),
                                  reduce_and_barrier_us=1e6 * med("cg_u_end", "cg_update")),
             "precond_phase": phase(tp, bp),
             "apply_phase": phase(ta, ba),
             "bytes_per_iteration": bu + bp + ba, "GBps": (bu + bp + ba) / t / 1e9,
             "frac_of_measured_hbm": (bu + bp + ba) / t / 1e9 / HBM_GBS}
        if prec == "fp64":
            fa = FLOPS_APPLY_PER_ELEM * ne + 2 * nn
            o["apply_phase"].update({"fp64_flops": fa, "TFLOPs": fa / ta / 1e12,
                                     "frac_of_fp64_peak": fa / ta / 1e12 / FP64_PEAK_TFLOPS})
            fi = fa + (UPDATE_FLOPS_FP64 + PRECOND_FLOPS_FP64) * nn
            o.update({"fp64_flops_per_iteration": fi, "TFLOPs": fi / t / 1e12,
                      "frac_of_fp64_peak": fi / t / 1e12 / FP64_PEAK_TFLOPS})
        out[prec] = o
    line = {"metric": "CG iteration throughput (update, preconditioner, matrix-free apply)", "mode": "roofline",
            "config": {"fine_nodes": nn, "fine_elements": ne,
                       "bytes_per_node": {"update": UPDATE_BYTES, "precond": PRECOND_BYTES, "apply": APPLY_BYTES},
                       "fp64_flops": {"apply_per_element": FLOPS_APPLY_PER_ELEM, "update_per_node": UPDATE_FLOPS_FP64,
                                      "precond_per_node": PRECOND_FLOPS_FP64},
                       "hbm_peak_GBps": HBM_GBS, "fp64_peak_TFLOPs": FP64_PEAK_TFLOPS},
            "results": out}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "batch":
        return run_batch(args)
    if args.mode == "serve":
        return run_serve(args)
    if args.mode == "roofline":
        return run_roofline(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
