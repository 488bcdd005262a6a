"""Continuous batching: jobs that arrive while others run are admitted as
slots and memory free up; each result equals the job run alone (within the
parity tolerance of its precision)."""
import numpy as np
import pytest

from paper_2110_12932_gb300 import build as tlbuild
from paper_2110_12932_gb300 import serve, tl, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    tlbuild.build()
    return tl.load()


def _jobs():
    base = workloads.workload("single_track_tiny")
    jobs = [
        dict(base, macro_steps=12),
        dict(base, macro_steps=7, P=150.0, pNXc=9, pNYc=3, pNZc=2, r=4, m=2),
        dict(base, macro_steps=9, precision=tl.TL_FP32_REFINED, tol=1e-10, tol_inner=1e-5),
        dict(base, macro_steps=5, tracks=[(0.2e-3, 0.3e-3, 1.8e-3, 0.3e-3, 1.2)]),
        dict(base, macro_steps=10, NXc=13, NYc=7, NZc=5, Lx=13 * 125e-6, Ly=7 * 125e-6, Lz=5 * 125e-6,
             pNXc=5, pNYc=3, pNZc=3, r=3, m=3, tracks=[(0.0, 0.45e-3, 13 * 125e-6, 0.45e-3, 0.8)]),
    ]
    return jobs


def test_results_same_alone_and_in_the_mix():
    jobs = _jobs()
    alone = []
    for cfg in jobs:
        p = tl.Problem(cfg)
        p.macro_steps(cfg["macro_steps"])
        alone.append(p.temperature(tl.TL_FINE)[0])
        p.close()
    arrivals = [(0.0, jobs[0]), (0.0, jobs[1]), (0.005, jobs[2]), (0.01, jobs[3]), (0.02, jobs[4])]
    # room for two resident jobs at a time: the later ones wait for a slot
    cap = 2.2 * max(serve.job_bytes(c) for c in jobs)
    got = {}
    srv = serve.Server(mem_cap_bytes=cap, max_jobs=2, launches_per_round=4)
    rep = srv.run(arrivals, on_done=lambda k, p, rec: got.__setitem__(k, p.temperature(tl.TL_FINE)[0]))
    srv.close()
    assert rep["jobs"] == len(jobs) and rep["all_ok"]
    assert rep["peak_admitted_bytes"] <= cap
    waited = [d for d in rep["done"] if d["admitted"] > d["arrival"] + 1e-3]
    assert waited, "some job must have waited for a slot"
    for k, cfg in enumerate(jobs):
        tol = 1e-6 if cfg.get("precision", 0) == tl.TL_FP32_REFINED else 1e-9
        rel = np.linalg.norm(got[k] - alone[k]) / np.linalg.norm(alone[k])
        assert rel <= tol, (k, rel)
    assert rep["job_latency_s"]["p99"] >= rep["job_latency_s"]["p50"] > 0
    assert rep["coarse_step_latency_ms"]["p50"] > 0


def test_fifo_reference_latencies():
    lat = serve.fifo_one_at_a_time([(0.0, None), (0.5, None), (0.6, None)], [1.0, 1.0, 1.0])
    assert lat == [1.0, 1.5, 2.4]


def test_failing_job_is_evicted_and_the_others_are_undisturbed():
    """One job cannot converge (max_iter = 1): its first failed solve ends its
    work in that round, the next poll reports it with TL_ENOCONV long before
    its scan would end, and every other job's result equals its run alone."""
    jobs = _jobs()[:3]
    bad = dict(jobs[0], max_iter=1, macro_steps=40, name="bad")
    alone = []
    for cfg in jobs:
        p = tl.Problem(cfg)
        p.macro_steps(cfg["macro_steps"])
        alone.append(p.temperature(tl.TL_FINE)[0])
        p.close()
    arrivals = [(0.0, jobs[0]), (0.0, bad), (0.0, jobs[1]), (0.002, jobs[2])]
    got, steps = {}, {}

    def on_done(k, p, rec):
        got[k] = p.temperature(tl.TL_FINE)[0]
        steps[k] = rec["steps"]

    srv = serve.Server(mem_cap_bytes=1e12, max_jobs=8, launches_per_round=4)
    rep = srv.run(arrivals, on_done=on_done)
    srv.close()
    assert rep["jobs"] == 4 and not rep["all_ok"]
    status = {d["key"]: d["status"] for d in rep["done"]}
    assert status[1] == tl.TL_ENOCONV
    assert all(status[k] == tl.TL_OK for k in (0, 2, 3))
    assert rep["failed"] == 1
    assert steps[1] < bad["macro_steps"]
    order = [d["key"] for d in rep["done"]]
    assert order.index(1) < order.index(0), "the failed job leaves before the healthy ones finish"
    for k, idx in ((0, 0), (2, 1), (3, 2)):
        cfg = jobs[idx]
        tol = 1e-6 if cfg.get("precision", 0) == tl.TL_FP32_REFINED else 1e-9
        rel = np.linalg.norm(got[k] - alone[idx]) / np.linalg.norm(alone[idx])
        assert rel <= tol, (k, rel)


@pytest.mark.parametrize("name,precision", [("multitrack_10mm", 0), ("multitrack_10mm", 1), ("multitrack_20mm", 0),
                                            ("multitrack_20mm", 1)])
def test_admission_model_covers_the_real_allocation(name, precision):
    """serve.job_bytes (the admission budget's estimate) against the device
    memory problems take (free memory before and after creating two of them,
    the library allocating with cudaMalloc; two so that the driver's page
    packing of small blocks averages out): never below it, at most 30 %
    above."""
    torch = pytest.importorskip("torch")
    cfg = workloads.workload(name, precision=precision, tol=1e-10 if precision else 1e-12)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    ps = [tl.Problem(cfg), tl.Problem(cfg)]
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    for p in ps:
        p.close()
    used = (free0 - free1) / 2
    est = serve.job_bytes(cfg)
    assert used > 0
    assert used <= est <= 1.3 * used, (used, est, est / used)
