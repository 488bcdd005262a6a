"""Batched jobs: uneven problems advanced by one persistent kernel per launch
must give the same results as each problem run alone (up to rounding: the
grid slice changes the summation order) and as the FP64 oracle."""
import numpy as np
import pytest

from oracle import twolevel as TL
from paper_2110_12932_gb300 import build as tlbuild
from paper_2110_12932_gb300 import tl, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    tlbuild.build()
    return tl.load()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _mixed_jobs():
    a = workloads.workload("single_track_tiny")
    b = workloads.workload("single_track_tiny", pNXc=9, pNYc=3, pNZc=2, r=4, m=2)
    c = workloads.workload("single_track_tiny", NXc=13, NYc=7, NZc=5, Lx=13 * 125e-6, Ly=7 * 125e-6,
                           Lz=5 * 125e-6, pNXc=5, pNYc=3, pNZc=3, r=3, m=3,
                           tracks=[(0.0, 0.45e-3, 13 * 125e-6, 0.45e-3, 0.8)])
    d = workloads.workload("single_track_tiny", r=1, m=1, coarse_source=1, pNXc=6, pNYc=4, pNZc=2)
    return [a, b, c, d]


# precision None: jobs alternate between the FP64 and the refined path (the
# batch then runs the kernel that holds both); inner_tiles 2 forces the wide
# two-phase inner CG on these small patches.
@pytest.mark.parametrize("precision,tol,inner_tiles", [(0, 1e-9, 0), (1, 1e-6, 1), (1, 1e-6, 2), (None, 1e-6, 0)])
def test_batch_equals_alone(precision, tol, inner_tiles):
    cfgs = []
    for k, c in enumerate(_mixed_jobs()):
        pr = (k % 2) if precision is None else precision
        cfgs.append(dict(c, precision=pr, tol=1e-12 if pr == 0 else 1e-10, tol_inner=1e-5, inner_tiles=inner_tiles))
    steps = [12, 9, 7, 15]
    alone = []
    for c, n in zip(cfgs, steps):
        p = tl.Problem(c)
        p.macro_steps(n)
        alone.append((p.temperature(tl.TL_FINE)[0], p.temperature(tl.TL_COARSE)[0], p.state(tl.TL_FINE)))
        p.close()
    batch = tl.Batch(launches_per_round=5, max_jobs=16)
    probs = [tl.Problem(c) for c in cfgs]
    for p, n in zip(probs, steps):
        batch.add(p, n)
    done = batch.run()
    assert len(done) == len(probs)
    info = batch.info()
    assert info["active"] == 0 and info["launches"] > 0
    for p, n, (Tf, Tc, sf) in zip(probs, steps, alone):
        st = p.stats()
        assert st["macro_steps"] == n
        assert p.sync() == tl.TL_OK
        assert rel(p.temperature(tl.TL_FINE)[0], Tf) <= tol
        assert rel(p.temperature(tl.TL_COARSE)[0], Tc) <= tol
        assert np.array_equal(p.state(tl.TL_FINE), sf)
        p.close()
    batch.close()


def test_batch_against_oracle():
    cfg = workloads.workload("single_track_tiny")
    p = tl.Problem(cfg)
    q = tl.Problem(workloads.workload("single_track_tiny", pNXc=9, pNYc=3, pNZc=2, r=4, m=2))
    batch = tl.Batch(launches_per_round=3, max_jobs=4)
    batch.add(p, 20)
    batch.add(q, 5)
    batch.run()
    ref = TL.TwoLevel(cfg).run(20)
    Tf, org = p.temperature(tl.TL_FINE)
    assert tuple(org) == tuple(ref.origin)
    assert rel(Tf, ref.Tf) <= 1e-9 and rel(p.temperature(tl.TL_COARSE)[0], ref.Tc) <= 1e-9
    assert np.array_equal(p.state(tl.TL_FINE), ref.fine_state().reshape(-1))
    st = p.stats()
    for lvl in ("fine", "coarse"):
        s, l, f = (st[f"energy_{lvl}_{k}"] for k in ("stored", "laser", "flux"))
        assert abs(s - l - f) <= 1e-9 * max(abs(s), abs(l))
    p.close()
    q.close()
    batch.close()


def test_batch_admits_and_retires_between_rounds():
    batch = tl.Batch(launches_per_round=4, max_jobs=2)
    cfg = workloads.workload("single_track_tiny")
    a, b, c = (tl.Problem(cfg) for _ in range(3))
    batch.add(a, 2)
    batch.add(b, 1)
    with pytest.raises(tl.TLError):
        batch.add(c, 1)            # both slots taken
    finished = []
    while len(finished) < 2:
        batch.round()
        finished += batch.poll()
    batch.add(c, 2)                # a slot freed up
    finished += batch.run()
    assert [p.stats()["macro_steps"] for p in (a, b, c)] == [2, 1, 2]
    ref = tl.Problem(cfg)
    ref.macro_steps(2)
    assert rel(c.temperature(tl.TL_FINE)[0], ref.temperature(tl.TL_FINE)[0]) <= 1e-9
    for p in (a, b, c, ref):
        p.close()
    batch.close()


def test_many_small_slices_keep_every_barrier():
    """48 small jobs share each launch (slices of a few blocks, short phases):
    a barrier that let a block into its next phase early, or lost an arrival,
    would end in a time-out (a nonzero status) or a wrong field.  Every job
    must finish with status 0 and equal its solo run."""
    base = workloads.workload("single_track_tiny")
    jobs = []
    for k in range(48):
        c = dict(base, macro_steps=6 + k % 5, P=120.0 + 3.0 * k)
        if k % 3 == 1:
            c.update(precision=tl.TL_FP32_REFINED, tol=1e-10, tol_inner=1e-5)
        if k % 4 == 2:
            c.update(pNXc=3, pNYc=2, pNZc=1, r=2, m=2)
        jobs.append(c)
    probs = [tl.Problem(c) for c in jobs]
    b = tl.Batch(launches_per_round=10, max_jobs=64)
    for p, c in zip(probs, jobs):
        b.add(p, c["macro_steps"])
    b.run()
    b.close()
    for k, (p, c) in enumerate(zip(probs, jobs)):
        assert p.sync() == tl.TL_OK, k
        got = p.temperature(tl.TL_FINE)[0]
        p.close()
        if k % 6 == 0 or k % 6 == 1:  # a sample of solo runs
            q = tl.Problem(c)
            q.macro_steps(c["macro_steps"])
            want = q.temperature(tl.TL_FINE)[0]
            q.close()
            tol = 1e-6 if c.get("precision", 0) == tl.TL_FP32_REFINED else 1e-9
            assert np.linalg.norm(got - want) <= tol * np.linalg.norm(want), k
