"""Checkpoint / resume: a run stopped between macro steps, saved, restored
into a fresh problem and continued is bit-identical to one that never
stopped (temperatures, origin, states, counters and energy account)."""
import numpy as np
import pytest

from paper_2110_12932_gb300 import build as tlbuild
from paper_2110_12932_gb300 import tl, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    tlbuild.build()
    return tl.load()


def snapshot(p):
    Tf, org = p.temperature(tl.TL_FINE)
    Tc, _ = p.temperature(tl.TL_COARSE)
    st = p.stats()
    keep = {k: v for k, v in st.items() if k not in ("launches", "time")}
    return Tf, tuple(org), Tc, p.state(tl.TL_FINE), p.state(tl.TL_COARSE), keep


@pytest.mark.parametrize("precision,sweeps", [(tl.TL_FP64, 1), (tl.TL_FP32_REFINED, 1), (tl.TL_FP64, 4)])
def test_resume_is_bit_identical(precision, sweeps):
    cfg = workloads.workload("single_track_tiny", precision=precision,
                             tol=1e-12 if precision == tl.TL_FP64 else 1e-10, coupling_sweeps=sweeps)
    a = tl.Problem(cfg)
    a.macro_steps(24)
    ref = snapshot(a)
    a.close()

    b = tl.Problem(cfg)
    b.macro_steps(11)
    buf = b.checkpoint()
    b.close()
    c = tl.Problem(cfg)
    c.restore(buf)
    c.macro_steps(13)
    got = snapshot(c)
    c.close()
    for x, y in zip(ref[:5], got[:5]):
        if isinstance(x, np.ndarray):
            assert np.array_equal(x, y)
        else:
            assert x == y
    assert ref[5] == got[5]


def test_checkpoint_errors():
    cfg = workloads.workload("single_track_tiny")
    p = tl.Problem(cfg)
    p.macro_steps(2)
    buf = p.checkpoint()
    p.predict()  # inside a macro step: no checkpoint, no restore
    st, _ = tl.tl_checkpoint_save(p.h)
    assert st == tl.TL_ESTATE
    assert tl.tl_checkpoint_load(p.h, buf) == tl.TL_ESTATE
    p.close()
    q = tl.Problem(dict(cfg, pNXc=3))  # another patch size: rejected
    assert tl.tl_checkpoint_load(q.h, buf) == tl.TL_EINVAL
    assert tl.tl_checkpoint_load(q.h, buf[:-1]) == tl.TL_EINVAL
    q.close()
    r = tl.Problem(cfg)
    bad = buf.copy()
    bad[0] ^= 0xFF  # not a checkpoint
    assert tl.tl_checkpoint_load(r.h, bad) == tl.TL_EINVAL
    r.restore(buf)
    r.close()


@pytest.mark.parametrize("over", [dict(P=150.0), dict(k0=7.0), dict(tol=1e-11), dict(coarse_source=1),
                                  dict(tracks=[(0.0, 0.5e-3, 1.9e-3, 0.5e-3, 0.8)]), dict(interface_coupling=1)])
def test_checkpoint_from_another_configuration_is_refused(over):
    """Same mesh and sizes, one value that changes the physics or the solver:
    the buffer is refused (TL_EINVAL) and the problem is untouched; the time
    limit of the barriers does not change the results and is accepted."""
    cfg = workloads.workload("single_track_tiny")
    p = tl.Problem(cfg)
    p.macro_steps(2)
    buf = p.checkpoint()
    p.close()
    q = tl.Problem(dict(cfg, **over))
    before = q.temperature(tl.TL_FINE)[0]
    assert tl.tl_checkpoint_load(q.h, buf) == tl.TL_EINVAL
    assert np.array_equal(q.temperature(tl.TL_FINE)[0], before)
    q.close()
    ok = tl.Problem(dict(cfg, barrier_timeout=5.0))
    ok.restore(buf)
    ok.close()
