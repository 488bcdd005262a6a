"""Further pins of the oracle (no GPU): the coarse box source against its
integrals, the injection set against its definition, the CG branch of the
sparse solver against a direct solve, the convergence of the oracle's own
solutions under refinement, and the saw-tooth of the multirate scheme's error
(Section 5.1)."""
from math import cos, exp, pi, sin

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import fem
from oracle import twolevel as TL
from paper_2110_12932_gb300 import workloads as W


# ---- coarse box source (Section 5.2, Q+ on the swept box; reading 4) --------

def _laser_on_pieces(tracks, t0, t1):
    """(track, a, b) laser-on intervals within [t0, t1], written out from the
    track lengths and speeds (tracks back to back from t = 0)."""
    out, t = [], 0.0
    for j, (x0, y0, x1, y1, v) in enumerate(tracks):
        d = ((x1 - x0) ** 2 + (y1 - y0) ** 2) ** 0.5 / v
        a, b = max(t0, t), min(t1, t + d)
        if b > a:
            out.append((j, a - t, b - t))
        t += d
    return out


def _expected_moments(cfg, n):
    """Sum, x- and y-moments of int q dA over the rectangles swept in macro
    step n: each track piece sweeps R x v (b - a) at intensity
    q = eta P / (R v Dt)."""
    Dt, R = cfg["dt_coarse"], cfg["radius"]
    s0 = sx = sy = 0.0
    for j, a, b in _laser_on_pieces(cfg["tracks"], n * Dt, (n + 1) * Dt):
        x0, y0, x1, y1, v = cfg["tracks"][j]
        assert y0 == y1, "the test scans along x"
        q = cfg["eta"] * cfg["P"] / (R * v * Dt)
        xa = x0 + (x1 - x0) * a * v / abs(x1 - x0)
        xb = x0 + (x1 - x0) * b * v / abs(x1 - x0)
        lo, hi = min(xa, xb), max(xa, xb)
        area = R * (hi - lo)
        s0 += q * area
        sx += q * R * (hi * hi - lo * lo) / 2.0
        sy += q * area * y0
    return s0, sx, sy


def _turning_cfg():
    cfg = W.single_track_tiny()
    # 1.03 mm tracks at 0.8 m/s last 25.75 macro steps: steps 25 and 51 hold
    # the turns, step 77 the end of the scan
    cfg["tracks"] = W.raster_tracks(0.5e-3, 1.53e-3, 0.5e-3, 3, 100e-6, 0.8)
    return cfg


@pytest.mark.parametrize("n", [0, 7, 25, 51, 77, 80])
def test_coarse_box_source_power_and_first_moments(n):
    """Bilinear hats sum to one and reproduce linear functions, so
    sum_i F_i = int q dA and sum_i F_i x_i = int q x dA exactly: the load of
    macro step n carries eta P (laser-on time) / Dt and is centred where the
    laser swept, split between tracks at a turn (n = 25, 51) and zero once
    the scan has ended (n = 80)."""
    cfg = _turning_cfg()
    o = TL.TwoLevel(cfg, energy=False)
    F = o.coarse_load(n)
    x, y, _ = o.coarse.node_xyz()
    s0, sx, sy = _expected_moments(cfg, n)
    on_time = sum(b - a for _, a, b in _laser_on_pieces(cfg["tracks"], n * o.Dt, (n + 1) * o.Dt))
    assert abs(s0 * o.Dt - cfg["eta"] * cfg["P"] * on_time) <= 1e-12 * cfg["eta"] * cfg["P"] * o.Dt
    scale = cfg["eta"] * cfg["P"]
    assert abs(F.sum() - s0) <= 1e-12 * scale
    assert abs(F @ x - sx) <= 1e-12 * scale * cfg["Lx"]
    assert abs(F @ y - sy) <= 1e-12 * scale * cfg["Ly"]
    if n in (25, 51):
        assert len(_laser_on_pieces(cfg["tracks"], n * o.Dt, (n + 1) * o.Dt)) == 2
    if n == 80:
        assert s0 == 0.0 and not F.any()
    else:
        assert s0 > 0.0


# ---- injection set (Algorithm 1's correction input; reading 3) --------------

@pytest.mark.parametrize("origin", [(5, 2, 2), (0, 2, 2), (12, 4, 2), (7, 0, 2)])
def test_injection_set_is_the_coarse_nodes_at_free_fine_nodes(origin):
    """The coarse nodes whose values the correction takes from the fine field
    are exactly those that coincide with a fine node that is not Dirichlet
    data of the local problem, on interior and plate-edge patch positions
    with r = 4."""
    o = TL.TwoLevel(W.single_track_tiny(), energy=False)
    r = o.r
    o.origin = origin
    mesh = o.fine_mesh(origin)
    dir_idx, _ = o.fine_dirichlet(origin)
    free = np.ones(mesh.nnode, dtype=bool)
    free[dir_idx] = False
    i, j, k = mesh.node_ijk()
    on_coarse = free & (i % r == 0) & (j % r == 0) & (k % r == 0)
    want = set(o.coarse.node_id(i[on_coarse] // r + origin[0], j[on_coarse] // r + origin[1],
                                k[on_coarse] // r + origin[2]).tolist())
    (i0, i1), (j0, j1), (k0, k1) = o.injection_box(origin)
    I, J, K = np.meshgrid(np.arange(i0, i1 + 1), np.arange(j0, j1 + 1), np.arange(k0, k1 + 1), indexing="ij")
    got = set(o.coarse.node_id(I.ravel(), J.ravel(), K.ravel()).tolist())
    assert got == want
    assert len(want) > 0


# ---- the CG branch of the sparse solver --------------------------------------

def test_solve_spd_cg_branch_matches_direct_solve():
    """Above 60000 unknowns solve_spd switches from SuperLU to preconditioned
    CG at a relative residual of 1e-14.  On a 67725-node system of the fine
    micro step's kind (a 300 x 14 x 14 bar of 15.6 um elements, random
    element heat capacities and conductivities in the workloads' ranges,
    powder elements included, Dirichlet bottom) the CG result matches SuperLU
    to 1e-12."""
    rng = np.random.default_rng(7)
    h = 125e-6 / 8
    mesh = fem.BoxMesh(300, 14, 14, h, h, h)
    dt = 50e-6 / 8
    Tb = rng.uniform(293.0, 2500.0, mesh.nelem)
    s_e = 4430.0 * (526.0 + 0.15 * (Tb - 293.0)) / dt
    k_e = (6.7 + 0.011 * (Tb - 293.0)) * np.where(rng.uniform(size=mesh.nelem) < 0.2, 0.01, 1.0)
    A = mesh.assemble(s_e, k_e)
    _, _, kk = mesh.node_ijk()
    dir_idx = np.flatnonzero(kk == 0)
    g = np.full(dir_idx.size, 293.0)
    b = rng.normal(size=mesh.nnode) * 1e-3
    free = np.flatnonzero(kk != 0)
    assert free.size > 60000
    x = fem.solve_dirichlet(A, b, dir_idx, g)
    A_ff = A[free][:, free].tocsc()
    rhs = b[free] - A[free][:, dir_idx] @ g
    xd = spla.splu(A_ff, permc_spec="MMD_AT_PLUS_A").solve(rhs)
    assert np.linalg.norm(x[free] - xd) <= 1e-12 * np.linalg.norm(xd)
    assert np.array_equal(x[dir_idx], g)


# ---- convergence under refinement of the oracle's own solutions ------------

def test_eigenmode_solution_converges_at_second_order():
    """Constant properties, no laser: from T - T_b = A cos(pi x/Lx)
    cos(pi y/Ly) sin(pi z/(2 Lz)) the heat equation decays the mode as
    exp(-lambda t), lambda = (k/rho c) pi^2 (1/Lx^2 + 1/Ly^2 + 1/(4 Lz^2)).
    The oracle's single-level backward-Euler solutions on three meshes with
    dt ~ h^2 approach it at O(h^2) + O(dt): the error falls ~4x per halving."""
    cfg = W.single_track_tiny()
    cfg.update(c1=0.0, k1=0.0, powder_depth=0.0, P=0.0, tracks=[])
    Lx, Ly, Lz = cfg["Lx"], cfg["Ly"], cfg["Lz"]
    lam = cfg["k0"] / (cfg["rho"] * cfg["c0"]) * pi ** 2 * (1 / Lx ** 2 + 1 / Ly ** 2 + 1 / (4 * Lz ** 2))
    t_end = 0.5 / lam
    A0 = 300.0
    errs = []
    for s in (1, 2, 4):
        nsteps = 3 * s * s
        sl = TL.SingleLevel(cfg, 4 * s, 2 * s, 2 * s, t_end / nsteps)
        x, y, z = sl.mesh.node_xyz()
        mode = np.cos(pi * x / Lx) * np.cos(pi * y / Ly) * np.sin(pi * z / (2 * Lz))
        sl.T = cfg["T_bottom"] + A0 * mode
        for _ in range(nsteps):
            sl.step()
        exact = cfg["T_bottom"] + A0 * exp(-lam * t_end) * mode
        errs.append(np.abs(sl.T - exact).max())
    q = [errs[0] / errs[1], errs[1] / errs[2]]
    assert all(3.3 < v < 4.7 for v in q), (errs, q)


# ---- the saw-tooth of the multirate scheme's error (Section 5.1) -----------

def test_error_saw_tooth_within_macro_steps():
    """Section 5.1's setting (r = 1, the Gaussian on both levels) against the
    single-level solve at the micro step: within every macro step the fine
    error is largest at its last micro step (whose Dirichlet data is the
    predictor's), falls at the first micro step of the next macro step (whose
    data starts from the corrected field), and the correction cuts the coarse
    error far below the predictor's."""
    base = W.single_track_tiny()
    base.update(NXc=32, NYc=16, NZc=8, pNXc=8, pNYc=6, pNZc=3, r=1, coarse_source=1)
    dt, m, nmacro = 25e-6, 4, 6
    ref = TL.SingleLevel(base, 32, 16, 8, dt)
    refT = [ref.T.copy()]
    for _ in range(m * nmacro):
        ref.step()
        refT.append(ref.T.copy())
    o = TL.TwoLevel(dict(base, m=m, dt_coarse=dt * m), energy=False)

    def rel_rise(T, Tref):
        return np.linalg.norm(T - Tref) / np.linalg.norm(Tref - base["T0"])

    fine, pred, corr = [], [], []
    for n in range(nmacro):
        o.predict()
        pred.append(rel_rise(o.Tc_pred, refT[(n + 1) * m]))
        errs = []
        for i in range(m):
            o.fine_substep(i)
            mesh = o.fine_mesh()
            x, y, z = mesh.node_xyz()
            ids = ref.mesh.node_id(np.rint(x / ref.mesh.hx).astype(int), np.rint(y / ref.mesh.hy).astype(int),
                                   np.rint(z / ref.mesh.hz).astype(int))
            errs.append(rel_rise(o.Tf, refT[n * m + i + 1][ids]))
        o.restrict_and_correct()
        o.n += 1
        corr.append(rel_rise(o.Tc, refT[(n + 1) * m]))
        fine.append(errs)
    for n, e in enumerate(fine):
        assert int(np.argmax(e)) == m - 1, (n, e)
        if n + 1 < nmacro:
            assert fine[n + 1][0] < e[-1], (n, e, fine[n + 1])
    assert all(c < 0.05 * p for c, p in zip(corr, pred)), (corr, pred)


# ---- flux-jump coupling (Section 3, Eqs. deltaDef and globalPbmAlternate) ----

def test_flux_jump_vanishes_when_the_conductivities_agree():
    """With one conductivity law on both levels and no powder (kappa_+ ==
    kappa_- everywhere) the interface term is zero, so the global problem of
    Eq. globalPbmAlternate is the plain coarse heat equation: T+ equals the
    single-level coarse solve for any patch position (the heat capacity may
    still depend on T)."""
    cfg = W.workload("single_track_tiny", interface_coupling=1, coarse_source=1, k1=0.0, powder_depth=0.0)
    o = TL.TwoLevel(cfg)
    sl = TL.SingleLevel(cfg, cfg["NXc"], cfg["NYc"], cfg["NZc"], cfg["dt_coarse"])
    moved = 0
    for n in range(12):
        before = o.origin
        o.macro_step()
        moved += before != o.origin
        sl.step()
        assert not o.interface_load().any()
        assert np.linalg.norm(o.Tc - sl.T) / np.linalg.norm(sl.T) < 1e-12, n
    assert moved >= 2


def test_flux_jump_load_of_a_linear_field():
    """T- = T0 + a x + b y + c z has dT-/dn = +-a, +-b, -c on the patch faces;
    with constant kappa_- and kappa_+ each coarse node interior to a face
    plane gets (kappa_+ - kappa_-) (n . grad T) h1 h2 (the integral of its hat
    over the plane), and the loads of the x+ face plane sum to
    (kappa_+ - kappa_-) a times its area."""
    cfg = W.workload("single_track_tiny", interface_coupling=1)
    o = TL.TwoLevel(cfg, energy=False)
    o.origin = (5, 2, 2)                     # every side and the bottom immersed
    assert o.interface_faces() == (True, True, True, True, True)
    x, y, z = o.fine_mesh().node_xyz()
    a, b, c = 3.0e5, -1.0e5, 2.0e5
    T = 293.0 + a * x + b * y + c * z
    km, kp = 2.0, 5.0
    G = o.interface_load(Tf=T, k_fine=km, k_coarse=kp)
    C = o.coarse
    hx, hy, hz = o.hc
    (i0, j0, k0), (pnx, pny, pnz) = o.origin, o.pN
    I, J, K = C.node_ijk()
    jump = kp - km
    xp = (I == i0 + pnx) & (J > j0) & (J < j0 + pny) & (K > k0) & (K < k0 + pnz)
    ym = (J == j0) & (I > i0) & (I < i0 + pnx) & (K > k0) & (K < k0 + pnz)
    zb = (K == k0) & (I > i0) & (I < i0 + pnx) & (J > j0) & (J < j0 + pny)
    assert np.allclose(G[xp], jump * a * hy * hz, rtol=1e-12, atol=0)
    assert np.allclose(G[ym], jump * (-b) * hx * hz, rtol=1e-12, atol=0)
    assert np.allclose(G[zb], jump * (-c) * hx * hy, rtol=1e-12, atol=0)
    plane = (I == i0 + pnx) & (J >= j0) & (J <= j0 + pny) & (K >= k0) & (K <= k0 + pnz)
    # edge nodes of the plane also carry the y / z faces' loads: take the x+ part alone
    Gx = o.interface_load(Tf=T, k_fine=km, k_coarse=kp) - o.interface_load(Tf=293.0 + b * y + c * z, k_fine=km,
                                                                             k_coarse=kp)
    assert abs(Gx[plane].sum() - jump * a * (pny * hy) * (pnz * hz)) <= 1e-12 * abs(jump * a * pny * hy * pnz * hz)


def test_flux_jump_load_against_fine_quadrature():
    """A random fine field and random conductivities: the 2 x 2 Gauss face
    integrals equal an independent 5 x 5 Gauss evaluation of
    int_gamma (kappa_+ - kappa_-) dT-/dn phi_I dA, with dT-/dn taken by a
    one-sided difference of the trilinear interpolant (exact inside an
    element) and phi_I from the trilinear interpolant of a unit coarse field."""
    rng = np.random.default_rng(3)
    cfg = W.workload("single_track_tiny", interface_coupling=1, pNXc=3, pNYc=2, pNZc=2, r=2)
    o = TL.TwoLevel(cfg, energy=False)
    o.origin = (4, 3, 2)
    mesh, C = o.fine_mesh(), o.coarse
    T = rng.uniform(300.0, 2000.0, mesh.nnode)
    kf = rng.uniform(0.05, 20.0, mesh.nelem)
    kc = rng.uniform(0.05, 20.0, C.nelem)
    G = o.interface_load(Tf=T, k_fine=kf, k_coarse=kc)
    xg, wg = np.polynomial.legendre.leggauss(5)
    xg, wg = 0.5 * (xg + 1.0), 0.5 * wg
    hf, hc = o.hf, o.hc
    org = np.array([o.origin[d] * hc[d] for d in range(3)])
    ext = np.array([o.pN[d] * hc[d] for d in range(3)])
    eps = 1e-3
    want = np.zeros(C.nnode)
    for d, side in ((0, 0), (0, 1), (1, 0), (1, 1), (2, 0)):
        a1, a2 = [ax for ax in range(3) if ax != d]
        n1, n2 = int(round(ext[a1] / hf[a1])), int(round(ext[a2] / hf[a2]))
        for e1 in range(n1):
            for e2 in range(n2):
                for q1, w1 in zip(xg, wg):
                    for q2, w2 in zip(xg, wg):
                        p = org.copy()
                        p[d] += ext[d] if side else 0.0
                        p[a1] += (e1 + q1) * hf[a1]
                        p[a2] += (e2 + q2) * hf[a2]
                        inward = -1.0 if side else 1.0
                        pin = p.copy()
                        pin[d] += inward * eps * hf[d]
                        local = fem.BoxMesh(*o.nf, *hf, origin=tuple(org))
                        t0 = fem.trilinear(local, T, *[np.array([v]) for v in p])[0]
                        t1 = fem.trilinear(local, T, *[np.array([v]) for v in pin])[0]
                        dTdn = (t0 - t1) / (eps * hf[d])
                        ie = [min(int((p[ax] - org[ax]) / hf[ax]), o.nf[ax] - 1) for ax in range(3)]
                        ie[d] = 0 if side == 0 else o.nf[d] - 1
                        km = kf[ie[0] + o.nf[0] * (ie[1] + o.nf[1] * ie[2])]
                        ce = [int(p[ax] / hc[ax]) for ax in range(3)]
                        ce[d] = o.origin[d] + (o.pN[d] if side else -1)
                        kp = kc[ce[0] + C.nx * (ce[1] + C.ny * ce[2])]
                        wgt = (kp - km) * dTdn * w1 * w2 * hf[a1] * hf[a2]
                        # hats of the eight nodes of the coarse cell holding p: the
                        # interpolant of a unit field at each
                        base = [int(np.floor(p[ax] / hc[ax] + 1e-12)) for ax in range(3)]
                        for cand in range(8):
                            nid = C.node_id(*[base[ax] + ((cand >> ax) & 1) for ax in range(3)])
                            e = np.zeros(C.nnode)
                            e[nid] = 1.0
                            want[nid] += wgt * fem.trilinear(C, e, *[np.array([v]) for v in p])[0]
    assert np.allclose(G, want, rtol=1e-9, atol=1e-12 * np.abs(want).max())
