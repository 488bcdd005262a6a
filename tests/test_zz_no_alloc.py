"""tl_box_step_noalloc: the single backward-Euler step for callers that may not
allocate device memory (its scratch is a fixed array inside the library).

Checked against the regular two-level entry points: with the patch covering
the whole plate and one micro step per macro step, every tl_macro_steps(1)
is exactly one such step on the fine mesh, so two calls in a row must give
the same temperatures (relative L2 <= 1e-9, the parity tolerance of the other
GPU tests) and the same element states.  It is also checked against the FP64 oracle's
single-level step (Section 2.1's backward-Euler step of the whole plate) for
several steps, and a call that reaches its iteration cap must leave T_out and
the states untouched.  This file is collected last so that a run stopping at
the first failure has already run every other test.
"""
import numpy as np
import pytest

from oracle import twolevel as TL
from paper_2110_12932_gb300 import build as tlbuild
from paper_2110_12932_gb300 import tl, workloads

pytestmark = pytest.mark.gpu

TOL = 1e-9


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    tlbuild.build()
    tl.load()
    return torch


def _desc(cfg, nx, ny, nz, dt, t):
    d = tl.tl_box_step_desc()
    for f in ("Lx", "Ly", "Lz", "T_bottom", "rho", "c0", "c1", "k0", "k1", "Tref", "powder_factor", "T_melt",
              "P", "eta", "radius", "tol", "max_iter"):
        setattr(d, f, cfg[f])
    d.nx, d.ny, d.nz, d.dt = nx, ny, nz, dt
    # laser position on the single straight track at the end of the step
    (x0, y0, x1, y1, v) = cfg["tracks"][0]
    length = ((x1 - x0) ** 2 + (y1 - y0) ** 2) ** 0.5
    f = v * t / length
    d.laser_on = int(f <= 1.0)
    d.xc, d.yc = x0 + f * (x1 - x0), y0 + f * (y1 - y0)
    return d


def test_noalloc_step_matches_two_level_entry_points(torch_cuda):
    torch = torch_cuda
    r = 2
    cfg = workloads.workload("single_track_tiny", pNXc=16, pNYc=8, pNZc=4, r=r, m=1)
    nx, ny, nz = 16 * r, 8 * r, 4 * r
    nn = (nx + 1) * (ny + 1) * (nz + 1)
    assert nn <= tl.TL_NOALLOC_MAX_NODES

    prob = tl.Problem(cfg)
    T = torch.full((nn,), cfg["T0"], dtype=torch.float64, device="cuda")
    hz = cfg["Lz"] / nz
    ke = np.arange(nz)
    layer = np.where(cfg["Lz"] - (ke + 0.5) * hz < cfg["powder_depth"], tl.POWDER, tl.SOLID)
    state0 = np.repeat(layer, nx * ny).astype(np.uint8)
    state = torch.from_numpy(state0).to("cuda")
    stream = torch.cuda.current_stream().cuda_stream
    dt = cfg["dt_coarse"] / cfg["m"]
    for n in range(2):
        prob.macro_steps(1)
        Tf, org = prob.temperature(tl.TL_FINE)
        sf = prob.state(tl.TL_FINE)
        assert tuple(org) == (0, 0, 0)
        d = _desc(cfg, nx, ny, nz, dt, (n + 1) * dt)
        st = tl.tl_box_step_noalloc(d, T.data_ptr(), T.data_ptr(), state.data_ptr(), stream)
        assert st == tl.TL_OK, tl.tl_status_string(st)
        torch.cuda.synchronize()
        got = T.cpu().numpy()
        rel = np.linalg.norm(got - Tf) / np.linalg.norm(Tf)
        assert rel <= TOL, (n, rel)
        assert np.array_equal(state.cpu().numpy(), sf), n
    assert float(T.max()) > cfg["T0"] + 100.0   # the laser heated the plate
    prob.close()


def test_noalloc_rejects_meshes_beyond_its_scratch(torch_cuda):
    torch = torch_cuda
    cfg = workloads.workload("single_track_tiny")
    d = _desc(cfg, 64, 32, 32, 1e-5, 1e-5)       # 65 * 33 * 33 nodes > 65536
    T = torch.zeros(1, dtype=torch.float64, device="cuda")
    s = torch.zeros(1, dtype=torch.uint8, device="cuda")
    st = tl.tl_box_step_noalloc(d, T.data_ptr(), T.data_ptr(), s.data_ptr(), None)
    assert st == tl.TL_EINVAL


def _initial_state(cfg, nx, ny, nz):
    hz = cfg["Lz"] / nz
    ke = np.arange(nz)
    layer = np.where(cfg["Lz"] - (ke + 0.5) * hz < cfg["powder_depth"], tl.POWDER, tl.SOLID)
    return np.repeat(layer, nx * ny).astype(np.uint8)


def test_noalloc_steps_match_the_oracle_single_level(torch_cuda):
    """Six steps of 12.5 us on a 32 x 16 x 8 mesh of the 2 x 1 x 0.5 mm plate
    against the oracle's single-level solve: relative L2 <= 1e-9 after every
    step, element states bit-exact (no element mean within 1e-6 K of T_melt)."""
    torch = torch_cuda
    cfg = workloads.workload("single_track_tiny", tracks=[(0.6e-3, 0.5e-3, 1.8e-3, 0.5e-3, 0.8)])
    nx, ny, nz = 32, 16, 8
    dt = 12.5e-6
    nn = (nx + 1) * (ny + 1) * (nz + 1)
    ref = TL.SingleLevel(cfg, nx, ny, nz, dt)
    T = torch.full((nn,), cfg["T0"], dtype=torch.float64, device="cuda")
    state = torch.from_numpy(_initial_state(cfg, nx, ny, nz)).to("cuda")
    assert np.array_equal(state.cpu().numpy(), ref.state)
    stream = torch.cuda.current_stream().cuda_stream
    for n in range(6):
        ref.step()
        d = _desc(cfg, nx, ny, nz, dt, (n + 1) * dt)
        st = tl.tl_box_step_noalloc(d, T.data_ptr(), T.data_ptr(), state.data_ptr(), stream)
        assert st == tl.TL_OK, tl.tl_status_string(st)
        got = T.cpu().numpy()
        rel = np.linalg.norm(got - ref.T) / np.linalg.norm(ref.T)
        assert rel <= TOL, (n, rel)
        ties = np.abs(ref.mesh.element_mean(ref.T) - cfg["T_melt"]) < 1e-6
        assert not ties.any()
        assert np.array_equal(state.cpu().numpy(), ref.state), n
    assert np.count_nonzero(ref.state == TL.MELTED) > 0


def test_noalloc_iteration_cap_leaves_output_and_state(torch_cuda):
    """max_iter = 1 cannot reach the tolerance: TL_ENOCONV, and neither T_out
    (a separate buffer here) nor the states change."""
    torch = torch_cuda
    cfg = workloads.workload("single_track_tiny", max_iter=1)
    nx, ny, nz = 16, 8, 4
    nn = (nx + 1) * (ny + 1) * (nz + 1)
    T_in = torch.full((nn,), cfg["T0"], dtype=torch.float64, device="cuda")
    T_out = torch.full((nn,), -1.0, dtype=torch.float64, device="cuda")
    s0 = _initial_state(cfg, nx, ny, nz)
    state = torch.from_numpy(s0).to("cuda")
    d = _desc(cfg, nx, ny, nz, 50e-6, 250e-6)
    assert d.laser_on
    st = tl.tl_box_step_noalloc(d, T_in.data_ptr(), T_out.data_ptr(), state.data_ptr(), None)
    assert st == tl.TL_ENOCONV
    assert bool((T_out == -1.0).all())
    assert np.array_equal(state.cpu().numpy(), s0)
    # the next call with a workable cap succeeds (the shared scratch was reset)
    d.max_iter = 2000
    st = tl.tl_box_step_noalloc(d, T_in.data_ptr(), T_out.data_ptr(), state.data_ptr(), None)
    assert st == tl.TL_OK
    assert float(T_out.max()) > cfg["T0"]
