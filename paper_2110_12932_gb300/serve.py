"""Continuous-batching request loop for two-level LPBF jobs.

Jobs (scan path + process parameters + plate size) arrive over time.  Between
batch rounds the loop admits every arrived job for which a batch slot is free
and whose device memory fits under the budget, keeps each admitted job's
coarse and fine state resident on the device, and advances all admitted jobs
together with the native batched kernel (tl_batch_round: every job performs
its next solves on its own slice of the grid).  Finished jobs leave the batch,
free their memory and make room for waiting ones.

A job whose solve fails (a CG cap, a barrier time-out) leaves the batch after
the round in which it failed and is reported with its status.

Latency per job = completion - arrival (queueing included); latency per coarse
step = the wall time of a round divided by the macro steps a job completed in
it, one sample per completed macro step.  The paper itself is serial; it notes
the method is embarrassingly parallel (Section 5.3).
"""
from __future__ import annotations

import collections
import time

import numpy as np

from . import tl, workloads

# Allocation granularity of the estimate: the CUDA allocator gives blocks of
# more than 1 MiB whole 2 MiB pages and packs smaller blocks (512-byte
# aligned) into shared 2 MiB pages, one page allowed per problem.
ALLOC_PAGE = 2 << 20
ALLOC_SMALL = 1 << 20
ALLOC_ROUND = 512
XB = 7        # exchange planes per partial buffer
RS_N = 9      # reduction rows
MAXRECT = 8   # load-table factors
TRACE_CAP = 1024


def _level_arrays(nnx, nny, nnz, nx, ny, nz, state_bytes, cfg, coarse):
    """Byte sizes of the device arrays one level holds (the layout the
    library allocates for a level)."""
    nn, ne = nnx * nny * nnz, nx * ny * nz
    xs = ((nn + 3) & ~3) * XB
    prec = int(cfg.get("precision", 0))
    a = [8 * nn] * 4 + [8 * nnx * nny, 8 * MAXRECT * (nnx + nny), 8 * nn, 8 * xs]
    if prec == 0:
        a += [8 * nn] * 6 + [8 * xs]
    a += [8 * nn, 8 * ne, 8 * ne, 64 * ne]
    if prec == 1:
        a += [4 * nn] * 4 + [4 * xs, 4 * nn, 4 * xs] + [4 * nn] * 5 + [8 * ne]
    if coarse:
        a.append(8 * nn)
    if int(cfg.get("coupling_sweeps", 1)) > 1:
        a += ([8 * nn] * 2 if coarse else []) + [ne]
    if int(cfg.get("picard_iters", 1)) > 1:
        a.append(8 * nn)
    a += [16 * TRACE_CAP, state_bytes, ne]
    if cfg.get("h_conv", 0.0) > 0 or cfg.get("emissivity", 0.0) > 0:
        a.append(8 * nx * ny)
        if prec == 1:
            a.append(4 * nx * ny)
    return a


def job_bytes(cfg):
    """Device memory a job holds while resident: every array of both levels
    (the fine level's states in the plate-wide map), the reduction slots and
    the small per-problem words, with the allocator's granularity (blocks
    above ALLOC_SMALL in whole ALLOC_PAGE pages, smaller ones rounded to
    ALLOC_ROUND, plus one page for them)."""
    r = cfg["r"]
    fx, fy, fz = cfg["pNXc"] * r, cfg["pNYc"] * r, cfg["pNZc"] * r
    cx, cy, cz = cfg["NXc"], cfg["NYc"], cfg["NZc"]
    arrays = _level_arrays(cx + 1, cy + 1, cz + 1, cx, cy, cz, cx * cy * cz, cfg, True)
    arrays += _level_arrays(fx + 1, fy + 1, fz + 1, fx, fy, fz, cx * r * cy * r * fz, cfg, False)
    grid = 2048  # reduction width: at most the grid cap
    arrays += [16, 8 * RS_N * grid, 4 * RS_N * grid, 256, 16, 16]

    def rounded(b):
        g = ALLOC_PAGE if b > ALLOC_SMALL else ALLOC_ROUND
        return (b + g - 1) // g * g
    return sum(rounded(b) for b in arrays) + ALLOC_PAGE


class Server:
    def __init__(self, mem_cap_bytes=120e9, max_jobs=256, launches_per_round=10, stream=None):
        self.mem_cap = float(mem_cap_bytes)
        self.max_jobs = int(max_jobs)
        self.stream = stream
        self.batch = tl.Batch(launches_per_round=launches_per_round, max_jobs=max_jobs, stream=stream)

    def close(self):
        self.batch.close()

    def run(self, arrivals, on_done=None, idle_sleep=2e-4):
        """Serve `arrivals` = [(t_arrival_s, cfg), ...] in wall-clock time.
        on_done(key, problem, record) is called for each finished job before
        its problem is released.  Returns a report dict."""
        t0 = time.perf_counter()
        queue = collections.deque(sorted(((float(t), k, cfg) for k, (t, cfg) in enumerate(arrivals)),
                                         key=lambda x: (x[0], x[1])))
        active = {}          # id(problem) -> record
        mem_used = 0.0
        peak_mem = 0.0
        step_lat = []
        job_lat = []
        done = []
        rounds = 0
        work_done = 0
        busy_s = 0.0
        while queue or active:
            now = time.perf_counter() - t0
            # admission: arrived jobs in order, while a slot and memory are free
            while queue and queue[0][0] <= now and len(active) < self.max_jobs:
                ta, key, cfg = queue[0]
                need = job_bytes(cfg)
                if mem_used + need > self.mem_cap:
                    break
                queue.popleft()
                p = tl.Problem(cfg, stream=self.stream)
                self.batch.add(p, cfg["macro_steps"])
                mem_used += need
                peak_mem = max(peak_mem, mem_used)
                active[id(p)] = dict(key=key, problem=p, cfg=cfg, arrival=ta,
                                     admitted=time.perf_counter() - t0, steps=0, bytes=need)
            if not active:
                if queue:
                    time.sleep(max(0.0, min(idle_sleep, queue[0][0] - (time.perf_counter() - t0))))
                continue
            r0 = time.perf_counter()
            self.batch.round()
            finished = self.batch.poll()
            r1 = time.perf_counter()
            rounds += 1
            busy_s += r1 - r0
            for rec in active.values():
                steps = rec["problem"].stats()["macro_steps"]
                d = steps - rec["steps"]
                if d > 0:
                    step_lat.extend([(r1 - r0) / d] * d)
                    work_done += d * rec["cfg"]["m"] * workloads.fine_nodes(rec["cfg"])
                    rec["steps"] = steps
            for p in finished:
                rec = active.pop(id(p))
                rec["done"] = r1 - t0
                rec["latency"] = rec["done"] - rec["arrival"]
                job_lat.append(rec["latency"])
                rec["status"] = p.sync()
                if on_done is not None:
                    on_done(rec["key"], p, rec)
                p.close()
                mem_used -= rec["bytes"]
                done.append({k: v for k, v in rec.items() if k != "problem"})
        wall = time.perf_counter() - t0

        def pct(v, q):
            return float(np.percentile(v, q)) if len(v) else None

        return {
            "jobs": len(done), "rounds": rounds, "wall_s": wall, "busy_s": busy_s,
            "fine_dof_substeps": work_done,
            "throughput": work_done / busy_s if busy_s > 0 else None,
            "job_latency_s": {"p50": pct(job_lat, 50), "p99": pct(job_lat, 99), "max": pct(job_lat, 100)},
            "coarse_step_latency_ms": {"p50": None if not step_lat else 1e3 * pct(step_lat, 50),
                                       "p99": None if not step_lat else 1e3 * pct(step_lat, 99)},
            "peak_admitted_bytes": peak_mem, "all_ok": all(d["status"] == 0 for d in done),
            "failed": sum(d["status"] != 0 for d in done),
            "done": done,
        }


def fifo_one_at_a_time(arrivals, service_s):
    """Latencies of the same arrivals served one job at a time in arrival
    order, job k taking service_s[k] seconds."""
    t = 0.0
    lat = []
    for (ta, _), s in sorted(zip(arrivals, service_s), key=lambda x: x[0][0]):
        t = max(t, ta) + s
        lat.append(t - ta)
    return lat
