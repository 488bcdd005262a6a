"""Failure paths that leave the GPU usable: a device barrier wait that runs out
(TL_ETIMEOUT), a device allocation that fails (TL_ENOMEM), and a CG solve that
reaches its cap inside a batch (the job leaves the batch, the others are not
disturbed).  None of them faults or hangs the device: the time-out is a
bounded wait under a 1 ns limit, the allocation failure comes from the
caller's allocator hook, the cap from max_iter = 1."""
import ctypes as C

import numpy as np
import pytest

from paper_2110_12932_gb300 import build as tlbuild
from paper_2110_12932_gb300 import tl, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    tlbuild.build()
    return tl.load()


def _snapshot(p):
    return (p.temperature(tl.TL_FINE), p.temperature(tl.TL_COARSE)[0], p.state(tl.TL_FINE), p.state(tl.TL_COARSE))


def test_barrier_timeout_is_reported_and_keeps_the_last_good_step():
    """A problem restored from a checkpoint runs its next macro step with a
    1 ns barrier limit: some wait runs out, every block leaves at that
    barrier, tl_macro_steps reports TL_ETIMEOUT, and the fields, origin and
    states stay those of the checkpoint; the handle stays failed (later
    steps are no-ops, checkpoints are refused)."""
    cfg = workloads.workload("multitrack_10mm")
    good = tl.Problem(cfg)
    # a step whose patch does not move, so that nothing but the solves could change the state
    origins = []
    for _ in range(6):
        good.macro_steps(1)
        origins.append(tuple(good.stats()["origin"]))
    ck = None
    probe = tl.Problem(cfg)
    for k in range(1, 6):
        probe.macro_steps(1)
        if origins[k] == origins[k - 1]:
            ck = probe.checkpoint()
            break
    assert ck is not None
    want = _snapshot(probe)
    probe.close()
    good.close()

    bad = tl.Problem(dict(cfg, barrier_timeout=1e-9))
    bad.restore(ck)
    assert tl.tl_macro_steps(bad.h, 1) == tl.TL_ETIMEOUT
    assert bad.sync() == tl.TL_ETIMEOUT
    got = _snapshot(bad)
    assert got[0][1] == want[0][1]                       # origin
    assert np.array_equal(got[0][0], want[0][0])         # fine field
    assert np.array_equal(got[1], want[1])               # coarse field
    assert np.array_equal(got[2], want[2]) and np.array_equal(got[3], want[3])
    assert tl.tl_macro_steps(bad.h, 1) == tl.TL_ETIMEOUT
    assert np.array_equal(bad.temperature(tl.TL_COARSE)[0], want[1])
    assert tl.tl_checkpoint_save(bad.h)[0] == tl.TL_ESTATE
    bad.close()


def test_allocation_failure_reports_enomem_and_frees_everything():
    """The caller's allocator returns NULL on its k-th call: tl_create_problem
    returns TL_ENOMEM, returns every block it got, and *out stays NULL; with
    no failure the same hooks carry a whole run."""
    torch = pytest.importorskip("torch")
    dev = torch.cuda.current_device()
    cfg = workloads.workload("single_track_tiny")
    for fail_at in (1, 7, 40, None):
        live, calls = {}, {"n": 0}

        def alloc(size, stream, ctx):
            calls["n"] += 1
            if fail_at is not None and calls["n"] == fail_at:
                return None
            ptr = torch.cuda.caching_allocator_alloc(size, dev, stream or 0)
            live[ptr] = size
            return ptr

        def free(ptr, stream, ctx):
            assert ptr in live
            del live[ptr]
            torch.cuda.caching_allocator_delete(ptr)

        a_fn, f_fn = tl.ALLOC_FN(alloc), tl.FREE_FN(free)
        c, keep = tl.make_config(cfg)
        c.alloc, c.free = a_fn, f_fn
        h = C.c_void_p()
        st = tl.load().tl_create_problem(C.byref(c), C.byref(h))
        if fail_at is not None and fail_at <= calls["n"]:
            assert st == tl.TL_ENOMEM, (fail_at, st)
            assert not h.value
            assert not live, (fail_at, len(live))
        else:
            assert st == tl.TL_OK and h.value
            assert fail_at is None or calls["n"] < fail_at
            assert tl.tl_macro_steps(h, 3) == tl.TL_OK
            T = tl.tl_get_temperature(h, tl.TL_FINE)[1]
            assert T.max() > cfg["T0"] + 100.0
            tl.tl_destroy_problem(h)
            assert not live
        torch.cuda.synchronize()
