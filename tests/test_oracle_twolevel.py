"""Pins of the two-level oracle (Algorithm 1) against closed forms, identities
and invariants (no GPU)."""
from math import cos, pi, sin

import numpy as np
import pytest

from oracle import fem
from oracle import twolevel as TL
from paper_2110_12932_gb300 import workloads as W


def _constant_props(cfg):
    cfg = dict(cfg)
    cfg.update(c1=0.0, k1=0.0, powder_depth=0.0)
    return cfg


def test_discrete_eigenmode_decay():
    """Constant properties, no laser: T - Tb = A cos(pi x/Lx) cos(pi y/Ly)
    sin(pi z/(2 Lz)) is an exact eigenvector of the Q1 pencil (adiabatic
    sides and top, Dirichlet bottom), so backward Euler multiplies it by
    (1 + dt lambda_h)^-1 per step with
    lambda_h = (k/rho c) sum_d (6/h_d^2)(1 - cos th_d)/(2 + cos th_d)."""
    cfg = _constant_props(W.single_track_tiny())
    cfg["P"] = 0.0
    nx, ny, nz = 12, 6, 5
    dt = 2e-4
    sl = TL.SingleLevel(cfg, nx, ny, nz, dt)
    x, y, z = sl.mesh.node_xyz()
    Lx, Ly, Lz = cfg["Lx"], cfg["Ly"], cfg["Lz"]
    mode = np.cos(pi * x / Lx) * np.cos(pi * y / Ly) * np.sin(pi * z / (2 * Lz))
    A0 = 400.0
    sl.T = cfg["T_bottom"] + A0 * mode
    hx, hy, hz = Lx / nx, Ly / ny, Lz / nz
    th = (pi * hx / Lx, pi * hy / Ly, pi * hz / (2 * Lz))
    lam = sum(6 / h ** 2 * (1 - cos(t)) / (2 + cos(t)) for h, t in zip((hx, hy, hz), th))
    lam *= cfg["k0"] / (cfg["rho"] * cfg["c0"])
    for n in range(1, 6):
        sl.step()
        expect = cfg["T_bottom"] + A0 * (1 + dt * lam) ** (-n) * mode
        assert np.abs(sl.T - expect).max() < 1e-9, n


def test_continuum_convergence_of_eigenvalue():
    """The discrete eigenvalue converges to the continuum one at O(h^2)."""
    k, rc = 6.7, 4430 * 526.0
    L = (2e-3, 1e-3, 0.5e-3)
    lam_c = k / rc * pi ** 2 * (1 / L[0] ** 2 + 1 / L[1] ** 2 + 1 / (4 * L[2] ** 2))
    errs = []
    for n in (4, 8, 16, 32):
        h = (L[0] / n, L[1] / n, L[2] / n)
        th = (pi * h[0] / L[0], pi * h[1] / L[1], pi * h[2] / (2 * L[2]))
        lam = k / rc * sum(6 / hh ** 2 * (1 - cos(t)) / (2 + cos(t)) for hh, t in zip(h, th))
        errs.append(abs(lam - lam_c) / lam_c)
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(3.8 < q < 4.2 for q in ratios)


def test_energy_identity_every_solve():
    """Stored heat = laser input + heat through the Dirichlet rows, per solve,
    on both levels (exact for the direct solves)."""
    o = TL.TwoLevel(W.single_track_tiny())
    o.run(8)
    for kind, e in o.step_energy:
        scale = max(abs(e["stored"]), abs(e["laser"]), 1e-12)
        assert abs(e["stored"] - e["laser"] - e["flux"]) <= 1e-10 * scale, kind
    assert o.energy["fine_laser"] > 0


def test_patch_covering_plate_equals_single_level():
    """Patch = whole plate: no interface, so every micro step is the
    single-level fine backward-Euler step (identity stated in Section 5.1)."""
    cfg = W.single_track_tiny()
    cfg.update(NXc=8, NYc=4, NZc=2, pNXc=8, pNYc=4, pNZc=2, r=2, m=2)
    o = TL.TwoLevel(cfg)
    sl = TL.SingleLevel(cfg, 16, 8, 4, cfg["dt_coarse"] / 2)
    for n in range(6):
        o.macro_step()
        sl.step()
        sl.step()
        assert o.origin == (0, 0, 0)
        rel = np.linalg.norm(o.Tf - sl.T) / np.linalg.norm(sl.T)
        assert rel < 1e-12, (n, rel)
    assert np.array_equal(o.fine_state().reshape(-1), sl.state)


def test_unit_ratios_equal_single_level_coarse():
    """r = 1, m = 1 and the Gaussian on the coarse level: the predictor is
    the single-level step, the patch solve reproduces it by uniqueness and
    the correction keeps it, for any patch position."""
    cfg = W.single_track_tiny()
    cfg.update(r=1, m=1, coarse_source=1, pNXc=6, pNYc=4, pNZc=2)
    o = TL.TwoLevel(cfg)
    sl = TL.SingleLevel(cfg, cfg["NXc"], cfg["NYc"], cfg["NZc"], cfg["dt_coarse"])
    moved = 0
    for n in range(20):
        before = o.origin
        o.macro_step()
        moved += before != o.origin
        sl.step()
        rel = np.linalg.norm(o.Tc - sl.T) / np.linalg.norm(sl.T)
        assert rel < 1e-12, (n, rel)
    assert moved >= 3


def test_patch_motion_copies_overlap_and_interpolates_new_nodes():
    o = TL.TwoLevel(W.single_track_tiny())
    o.run(3)
    # force a move by one coarse element in +x
    old = o.origin
    Tf_old = o.Tf.copy()
    new = (old[0] + 1, old[1], old[2])
    o._origin_for = lambda n, prev: new
    assert o.move_patch()
    r = o.r
    nx, ny, nz = o.nf
    mesh = o.fine_mesh()
    i, j, k = mesh.node_ijk()
    src_i = i + r
    inside = src_i <= nx
    src = src_i + (nx + 1) * (j + (ny + 1) * k)
    assert np.array_equal(o.Tf[inside], Tf_old[src[inside]])
    x, y, z = mesh.node_xyz()
    interp = fem.trilinear(o.coarse, o.Tc, x, y, z)
    assert np.allclose(o.Tf[~inside], interp[~inside], rtol=1e-13, atol=0)


def test_state_rule():
    mat = TL.Material(W.single_track_tiny())
    state = np.array([TL.POWDER, TL.POWDER, TL.SOLID, TL.MELTED, TL.MELTED], dtype=np.uint8)
    Tbar = np.array([1000.0, 2000.0, 1900.0, 1000.0, 1900.0000001])
    new = mat.update_state(Tbar, state)
    assert list(new) == [TL.POWDER, TL.MELTED, TL.SOLID, TL.SOLID, TL.MELTED]
    rc, k = mat.coefficients(np.array([293.0, 293.0]), np.array([TL.POWDER, TL.SOLID]))
    assert rc[0] == rc[1] == 4430 * 526.0
    assert k[1] == 6.7 and abs(k[0] - 0.067) < 1e-15


def test_initial_powder_layer():
    o = TL.TwoLevel(W.single_track_tiny())
    # fine elements are 31.25 um: centroids at 15.6 and 46.9 um below the top are powder
    mz = o.map_dims[2]
    layers = o.state_map[:, 0, 0]
    assert list(layers[mz - 2:]) == [TL.POWDER, TL.POWDER]
    assert np.all(layers[:mz - 2] == TL.SOLID)
    # no coarse element (125 um) is powder
    assert np.all(o.state_c == TL.SOLID)


def test_scan_path_times_and_positions():
    cfg = W.multitrack_10mm()
    path = TL.ScanPath(cfg["tracks"])
    assert abs(path.t_end[-1] - 0.1) < 1e-15
    x, y = path.position(0.0)
    assert (x, y) == (1e-3, 2.05e-3)
    x, y = path.position(0.01 + 0.005)       # middle of the second track (returning)
    assert abs(x - 5e-3) < 1e-15 and abs(y - 2.15e-3) < 1e-15
    assert path.position(0.1 + 1e-9) is None


@pytest.mark.slow
def test_error_grows_with_time_ratio():
    """Section 5.1's setting: identical spatial discretisation on both levels
    (r = 1, the Gaussian on the coarse level too) isolates the temporal error
    of the multirate scheme; at fixed micro step it is zero for m = 1 and
    grows with the macro step Dt = m dt."""
    base = W.single_track_tiny()
    base.update(NXc=32, NYc=16, NZc=8, pNXc=8, pNYc=6, pNZc=3, r=1, coarse_source=1)
    dt = 25e-6
    nsteps = 16
    ref = TL.SingleLevel(base, base["NXc"], base["NYc"], base["NZc"], dt)
    for _ in range(nsteps):
        ref.step()
    errs = []
    for m in (1, 2, 4, 8):
        cfg = dict(base, m=m, dt_coarse=dt * m)
        o = TL.TwoLevel(cfg)
        o.run(nsteps // m)
        mesh = o.fine_mesh()
        x, y, z = mesh.node_xyz()
        gi = np.rint(x / ref.mesh.hx).astype(int)
        gj = np.rint(y / ref.mesh.hy).astype(int)
        gk = np.rint(z / ref.mesh.hz).astype(int)
        Tref = ref.T[ref.mesh.node_id(gi, gj, gk)]
        errs.append(np.linalg.norm(o.Tf - Tref) / np.linalg.norm(Tref))
    assert errs[0] < 1e-12, errs
    assert errs[0] < errs[1] < errs[2] < errs[3], errs


# ---- iterated two-level coupling at the correction step ---------------------

def _run(cfg, n, energy=False):
    o = TL.TwoLevel(cfg, energy=energy)
    hist = []
    for _ in range(n):
        o.macro_step()
        hist.append(list(getattr(o, "coupling_history", [])))
    return o, hist


def test_coupling_one_sweep_is_the_plain_correction():
    cfg = W.single_track_tiny()
    a, _ = _run(cfg, 6)
    b, _ = _run(dict(cfg, coupling_sweeps=1), 6)
    assert np.array_equal(a.Tc, b.Tc) and np.array_equal(a.Tf, b.Tf)


def test_coupling_contracts_to_a_fixed_point():
    """The sweeps of the coupled correction contract: every change of the
    coarse field is smaller than the previous one and the last is below the
    tolerance; the converged field differs from the one-sweep correction by a
    small but non-zero amount (the iteration does something)."""
    cfg = W.single_track_tiny()
    one, _ = _run(cfg, 8)
    it, hist = _run(dict(cfg, coupling_sweeps=30, coupling_tol=1e-13), 8)
    for h in hist:
        assert len(h) >= 1 and h[-1] <= 1e-13
        assert all(b < a for a, b in zip(h, h[1:])), h
    d = np.linalg.norm(it.Tc - one.Tc) / np.linalg.norm(one.Tc)
    assert 1e-12 < d < 1e-3, d


def test_coupling_keeps_the_unit_ratio_identity():
    """r = m = 1 with the Gaussian on both levels: the corrected field equals
    the predictor, so re-solving reproduces the same fine field and the first
    re-solve already meets any tolerance; the result stays the single-level
    solve."""
    cfg = W.single_track_tiny()
    cfg.update(r=1, m=1, coarse_source=1, pNXc=6, pNYc=4, pNZc=2, coupling_sweeps=5, coupling_tol=1e-12)
    o = TL.TwoLevel(cfg)
    sl = TL.SingleLevel(cfg, cfg["NXc"], cfg["NYc"], cfg["NZc"], cfg["dt_coarse"])
    for n in range(10):
        o.macro_step()
        sl.step()
        assert len(o.coupling_history) == 1 and o.coupling_history[0] <= 1e-12
        assert np.linalg.norm(o.Tc - sl.T) / np.linalg.norm(sl.T) < 1e-12


def test_coupling_energy_account_counts_final_solves():
    """With re-solves the account keeps one fine entry per micro step and one
    coarse entry per correction, and each satisfies the energy identity."""
    cfg = dict(W.single_track_tiny(), coupling_sweeps=6, coupling_tol=1e-12)
    o, hist = _run(cfg, 5, energy=True)
    assert sum(len(h) for h in hist) > 5  # re-solves happened
    fine = [e for lvl, e in o.step_energy if lvl == "fine"]
    coarse = [e for lvl, e in o.step_energy if lvl == "coarse"]
    assert len(fine) == 5 * cfg["m"] and len(coarse) == 5
    for e in fine + coarse:
        assert abs(e["stored"] - e["laser"] - e["flux"]) <= 1e-9 * max(abs(e["stored"]), abs(e["laser"]), 1e-30)
    for lvl in ("fine", "coarse"):
        tot = sum(e["stored"] for l2, e in o.step_energy if l2 == lvl)
        assert abs(tot - o.energy[f"{lvl}_stored"]) <= 1e-9 * abs(tot)


# ---- latent heat (Eq. thermalEqn's phase-change term) and Picard iterations --

def _latent_material(**over):
    return TL.Material(W.workload("single_track_tiny", latent=2.86e5, **over))


def test_phase_change_sigmoid_derivative_and_integral():
    """f_pc' is the derivative of f_pc (central differences) and integrates to
    the sigmoid's full rise, 1 (a wrong factor of S/2 or a missing T fails)."""
    from scipy.integrate import quad
    mat = _latent_material()
    T = np.linspace(mat.Tm - 300.0, mat.Tm + 300.0, 61)
    h = 1e-3
    fd = (mat.fpc(T + h) - mat.fpc(T - h)) / (2 * h)
    assert np.max(np.abs(mat.fpc_prime(T) - fd)) <= 1e-6 * np.max(fd)
    total, _ = quad(lambda x: float(mat.fpc_prime(x)), mat.Tm - 1500.0, mat.Tm + 1500.0, points=[mat.Tm], limit=200)
    assert abs(total - 1.0) <= 1e-10
    assert abs(mat.fpc(mat.Tm) - 0.5) <= 1e-15 and mat.fpc(mat.Tm - 2000.0) < 1e-15


def test_phase_change_secant():
    """The secant is the difference quotient of f_pc, the derivative in the
    limit; the two branches meet at the switch |S dT| = 1e-3."""
    mat = _latent_material()
    a = np.array([1800.0, 1890.0, 1900.5, 1950.0])
    b = a + 37.0
    assert np.allclose(mat.fpc_secant(b, a), (mat.fpc(b) - mat.fpc(a)) / 37.0, rtol=1e-13, atol=0)
    assert np.allclose(mat.fpc_secant(a, a), mat.fpc_prime(a), rtol=1e-15, atol=0)
    d = 1e-3 / mat.S
    below = mat.fpc_secant(a + d * (1 - 1e-9), a)
    above = mat.fpc_secant(a + d * (1 + 1e-9), a)
    assert np.allclose(below, above, rtol=1e-6, atol=0)


def test_picard_reaches_the_nonlinear_backward_euler_step():
    """With enough Picard iterations the step satisfies the nonlinear
    backward-Euler equation with its coefficients (latent secant, c(T), k(T))
    taken at its own result; one lagged solve does not."""
    dt = 50e-6
    res = {}
    for K in (1, 30):
        cfg = W.workload("single_track_tiny", latent=2.86e5, picard_iters=K)
        sl = TL.SingleLevel(cfg, 16, 8, 4, dt)
        for _ in range(3):
            sl.step()
        T0, st = sl.T.copy(), sl.state.copy()
        sl.step()
        mesh = sl.mesh
        rc, k = sl.mat.coefficients(mesh.element_mean(sl.T), st, mesh.element_mean(T0))
        A = mesh.assemble(rc / dt, k)
        S = mesh.assemble(rc / dt, np.zeros_like(k))
        pos = sl.path.position(4 * dt)
        F = fem.gaussian_surface_load(mesh, pos[0], pos[1], cfg["P"], cfg["eta"], cfg["radius"])
        free = np.setdiff1d(np.arange(mesh.nnode), sl.dir_idx)
        res[K] = np.linalg.norm((A @ sl.T - S @ T0 - F)[free]) / np.linalg.norm(F)
    assert res[30] <= 1e-9
    assert res[1] >= 1e-3


def test_latent_heat_energy_identity_every_solve():
    """Each solve's stored heat (with the latent secant) equals the laser input
    plus the Dirichlet flux, with Picard iterations on both levels."""
    cfg = W.workload("single_track_tiny", latent=2.86e5, picard_iters=3)
    ref = TL.TwoLevel(cfg, energy=True).run(3)
    assert len(ref.step_energy) == 3 * (cfg["m"] + 1)
    for _, e in ref.step_energy:
        scale = max(abs(e["stored"]), abs(e["laser"]), 1e-30)
        assert abs(e["stored"] - e["laser"] - e["flux"]) <= 1e-10 * scale


def test_latent_heat_changes_the_solution_and_zero_latent_does_not():
    base = TL.TwoLevel(W.workload("single_track_tiny"), energy=False).run(2)
    zero = TL.TwoLevel(W.workload("single_track_tiny", latent=0.0, picard_iters=1), energy=False).run(2)
    lat = TL.TwoLevel(W.workload("single_track_tiny", latent=2.86e5, picard_iters=3), energy=False).run(2)
    assert np.array_equal(base.Tf, zero.Tf) and np.array_equal(base.Tc, zero.Tc)
    assert np.max(np.abs(lat.Tf - base.Tf)) > 1.0


# ---- top-surface heat loss: convection and radiation (Section 3.1) ---------

def _steady_cfg(**over):
    base = dict(tracks=[], powder_depth=0.0, c1=0.0, k1=0.0, T0=1500.0, T_bottom=1500.0, T_amb=293.0)
    base.update(over)
    return W.workload("single_track_tiny", **base)


@pytest.mark.parametrize("eps", [0.0, 0.6])
def test_steady_profile_with_surface_losses(eps):
    """Constant k, Dirichlet bottom, top losing h (T - T_amb) + sigma eps
    (T^4 - T_amb^4): the steady field is linear in z, T_top the root of
    k (T_top - T_b) / Lz + q(T_top) = 0 (found here by a bracketing root
    finder), and Q1 elements reproduce it exactly; one huge time step with
    Picard iterations reaches it.  A wrong sign, scale or T_amb term fails."""
    from scipy.optimize import brentq
    cfg = _steady_cfg(h_conv=4.0e4, emissivity=eps, picard_iters=40 if eps else 1)
    sl = TL.SingleLevel(cfg, 4, 2, 8, 1e9)
    sl.step()
    k, Lz, Tb, Ta = cfg["k0"], cfg["Lz"], cfg["T_bottom"], cfg["T_amb"]
    sigma = TL.SIGMA_SB

    def residual(Tt):
        return k * (Tt - Tb) / Lz + cfg["h_conv"] * (Tt - Ta) + sigma * eps * (Tt ** 4 - Ta ** 4)

    Tt = brentq(residual, Ta, Tb, xtol=1e-14, rtol=1e-15)
    _, _, z = sl.mesh.node_xyz()
    expect = Tb + (Tt - Tb) * z / Lz
    assert Tt < Tb - 10.0
    assert np.max(np.abs(sl.T - expect)) <= 1e-8 * Tb


def test_surface_loss_energy_identity_every_solve():
    """stored = laser + Dirichlet flux - surface loss for every solve, with
    convection on both levels and radiation on the local one."""
    cfg = W.workload("single_track_tiny", h_conv=50.0, emissivity=0.5, T_amb=293.0, picard_iters=3)
    ref = TL.TwoLevel(cfg, energy=True).run(3)
    assert ref.energy["fine_loss"] > 0 and ref.energy["coarse_loss"] != 0
    for _, e in ref.step_energy:
        scale = max(abs(e["stored"]), abs(e["laser"]), abs(e["loss"]), 1e-30)
        assert abs(e["stored"] - e["laser"] - e["flux"] + e["loss"]) <= 1e-10 * scale


def test_surface_off_is_the_plain_step():
    base = TL.TwoLevel(W.workload("single_track_tiny"), energy=True).run(2)
    off = TL.TwoLevel(W.workload("single_track_tiny", h_conv=0.0, emissivity=0.0), energy=True).run(2)
    assert np.array_equal(base.Tf, off.Tf) and np.array_equal(base.Tc, off.Tc)
    assert off.energy["fine_loss"] == 0.0 and off.energy["coarse_loss"] == 0.0
