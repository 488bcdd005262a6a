"""Multi-rank host logic on the CPU: two gloo ranks deal jobs, arrivals and
replicas without overlap and reduce the reported numbers (the slowest rank's
time, the sum of the ranks' work)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2110_12932_gb300 import ranks, workloads


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    r, w, local = ranks.init("gloo")
    assert (r, w, local) == (rank, ws, rank)
    jobs = ranks.deal(workloads.batch_jobs(10), r, w)
    arrivals = ranks.deal(workloads.serving_arrivals(2.0, 5.0), r, w)
    work = sum(workloads.fine_nodes(j) * j["m"] * j["macro_steps"] for j in jobs)
    secs = 1.0 + r  # rank r "takes" 1 + r seconds
    ranks.barrier(w)
    out[rank] = dict(jobs=[j["name"] for j in jobs], arrivals=[t for t, _ in arrivals], work=work,
                     max_t=ranks.max_over_ranks(secs, w), sum_work=ranks.sum_over_ranks(work, w),
                     rate=ranks.aggregate_rate(work, secs, w))
    ranks.finish(w)


def test_two_gloo_ranks_deal_and_reduce():
    ws = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank_main, args=(k, ws, port, out)) for k in range(ws)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        codes = [p.exitcode for p in procs]
        res = dict(out)
    assert codes == [0, 0], codes
    all_jobs = [j["name"] for j in workloads.batch_jobs(10)]
    dealt = res[0]["jobs"] + res[1]["jobs"]
    assert sorted(dealt) == sorted(all_jobs) and len(set(dealt)) == len(all_jobs)
    assert res[0]["jobs"] == all_jobs[0::2] and res[1]["jobs"] == all_jobs[1::2]
    all_arr = [t for t, _ in workloads.serving_arrivals(2.0, 5.0)]
    assert sorted(res[0]["arrivals"] + res[1]["arrivals"]) == sorted(all_arr)
    total = res[0]["work"] + res[1]["work"]
    for k in range(ws):
        assert res[k]["max_t"] == 2.0
        assert res[k]["sum_work"] == pytest.approx(total, rel=0, abs=0.5)
        assert res[k]["rate"] == pytest.approx(total / 2.0)


def test_single_rank_is_identity(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert ranks.world() == (0, 1, 0)
    items = list(range(7))
    assert ranks.deal(items, 0, 1) == items
    assert ranks.max_over_ranks(3.5, 1) == 3.5
    assert ranks.sum_over_ranks(4, 1) == 4
    assert ranks.aggregate_rate(10.0, 2.0, 1) == 5.0
