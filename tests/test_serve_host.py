"""Host logic of the serving loop (admission, completion, accounting) on CPU:
the batch backend is replaced by a fake that advances every active job by one
macro step per round, so no GPU is needed."""
import pytest

from paper_2110_12932_gb300 import serve, tl, workloads


class FakeProblem:
    live = 0

    def __init__(self, cfg, stream=None):
        self.cfg = cfg
        self.steps = 0
        self.target = None
        FakeProblem.live += 1

    def stats(self):
        return {"macro_steps": self.steps}

    def sync(self):
        return 0

    def close(self):
        FakeProblem.live -= 1


class FakeBatch:
    def __init__(self, launches_per_round=10, max_jobs=256, stream=None):
        self.jobs = []
        self.max_active = 0

    def add(self, p, macro_steps):
        p.target = macro_steps
        self.jobs.append(p)
        self.max_active = max(self.max_active, len(self.jobs))

    def round(self):
        for p in self.jobs:
            p.steps += 1

    def poll(self):
        done = [p for p in self.jobs if p.steps >= p.target]
        self.jobs = [p for p in self.jobs if p.steps < p.target]
        return done

    def close(self):
        pass


@pytest.fixture
def fake_backend(monkeypatch):
    monkeypatch.setattr(tl, "Problem", FakeProblem)
    monkeypatch.setattr(tl, "Batch", FakeBatch)
    FakeProblem.live = 0
    yield


def _jobs(n, steps=3):
    out = []
    for c in workloads.batch_jobs(n):
        c = dict(c)
        c["macro_steps"] = steps
        out.append((0.0, c))
    return out


def test_all_jobs_finish_and_work_is_counted(fake_backend):
    arrivals = _jobs(6)
    srv = serve.Server(mem_cap_bytes=1e15, max_jobs=64)
    rep = srv.run(arrivals)
    srv.close()
    assert rep["jobs"] == 6 and rep["all_ok"] and FakeProblem.live == 0
    assert rep["fine_dof_substeps"] == sum(3 * c["m"] * workloads.fine_nodes(c) for _, c in arrivals)
    assert sorted(d["key"] for d in rep["done"]) == list(range(6))
    assert all(d["latency"] >= 0 for d in rep["done"])


def test_slot_cap_limits_active_jobs(fake_backend):
    srv = serve.Server(mem_cap_bytes=1e15, max_jobs=2)
    rep = srv.run(_jobs(5))
    assert srv.batch.max_active == 2 and rep["jobs"] == 5
    srv.close()


def test_memory_budget_limits_admission_in_arrival_order(fake_backend):
    arrivals = _jobs(5)
    sizes = [serve.job_bytes(c) for _, c in arrivals]
    cap = max(sizes) + min(sizes) - 1      # never room for the two largest together
    srv = serve.Server(mem_cap_bytes=cap, max_jobs=64)
    rep = srv.run(arrivals)
    srv.close()
    assert rep["jobs"] == 5 and rep["peak_admitted_bytes"] <= cap
    admitted = sorted(rep["done"], key=lambda d: (d["admitted"], d["key"]))
    assert [d["key"] for d in admitted] == sorted(d["key"] for d in admitted)  # head of line first


def test_job_bytes_grows_with_the_mesh():
    small = workloads.workload("single_track_tiny")
    big = workloads.workload("multitrack_10mm")
    assert 0 < serve.job_bytes(small) < serve.job_bytes(big)
    assert serve.job_bytes(dict(big, precision=1)) != serve.job_bytes(big)


def test_fifo_one_at_a_time_latencies():
    arrivals = [(0.0, None), (1.0, None), (1.5, None), (10.0, None)]
    lat = serve.fifo_one_at_a_time(arrivals, [2.0, 2.0, 1.0, 0.5])
    # finish times 2, 4, 5, 10.5
    assert lat == pytest.approx([2.0, 3.0, 3.5, 0.5])
