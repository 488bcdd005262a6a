"""Spatiotemporal two-level method (Algorithm 1, Section 4), FP64 oracle.

Test infrastructure only (see the package docstring).

Problem (Section 2.1, Eq. thermalEqn): plate [0,Lx]x[0,Ly]x[0,Lz],
Dirichlet T_bottom on z = 0, adiabatic sides, a laser flux on the top
surface z = Lz, which also loses heat (Section 3.1; off by default): by
convection h_conv (T - T_amb) on both levels and by radiation
sigma eps (T^4 - T_amb^4) on the local level only (see Surface).  Material: rho constant, c(T) = c0 + c1 (T - Tref),
k(T) = k0 + k1 (T - Tref); powder elements use powder_factor * k.  Latent
heat (latent = chi > 0): f_pc(T) = (1 + tanh(S (T - Tm))) / 2 with
Tm = (T_solidus + T_liquidus) / 2 and S = pc_sharpness (Eq. 2dPhaseChange of
Section 5.1 prints its derivative (S/2)(1 - tanh^2(S (T - Tm))) with the
argument garbled).  Backward Euler applied to the term chi rho d f_pc/dt
gives chi rho (f_pc(T^{n+1}) - f_pc(T^n)) / dt; per element it enters the
heat capacity as the secant chi (f_pc(Tb) - f_pc(Tb0)) / (Tb - Tb0) of the
element means Tb (of the temperature the coefficients are taken at) and Tb0
(of the step's start), the derivative f_pc' at the midpoint when
|S (Tb - Tb0)| < 1e-3.

Two levels (Section 3, Eqs. localProblem and globalPbmAlternate):
  global (coarse) mesh of NXc x NYc x NZc hexes over the plate;
  local (fine) patch of pNXc x pNYc x pNZc coarse hexes at the top surface,
  each refined r times per direction, origin on a coarse node, following the
  laser (Section 5.2: the local mesh moves, no projection).

One macro step t_n -> t_n + Dt (Algorithm 1), this oracle's reading:
  1. Patch motion: origin = clamp(floor((x_l - patch_len/2)/h_c + 0.5)) for
     the laser position x_l at t_n + Dt/2 (kept if the laser is off then).
     Fine nodes inside the old patch keep their values; new nodes get the
     trilinear interpolant of the current coarse field.
  2. Predictor: one backward-Euler step of size Dt on the coarse mesh from
     T+^n -> T~+ (coefficients at T+^n, coarse source over [t_n, t_n+Dt]).
  3. For i = 0..m-1, the time-local problem Eq. (localProblemTime): one
     backward-Euler step of size dt = Dt/m on the patch, Dirichlet data on
     the patch faces interior to the plate (gamma_D) equal to
     (1-w) I(T+^n) + w I(T~+) with w = (i+1)/m (the solve of micro step i
     produces time t_n + (i+1) dt; the printed weight i/m is available with
     bc_weight_literal = 1), patch faces on the plate's sides adiabatic,
     patch nodes on the plate's bottom at T_bottom.  Surface Gaussian at the
     laser position at t_n + (i+1) dt.
  4. Correction: inject the fine values at the coarse nodes that coincide
     with free fine nodes, then redo the coarse backward-Euler step from
     T+^n with those nodes held as Dirichlet data -> T+^{n+1}.
  5. Iterated coupling (coupling_sweeps > 1; the paper solves the local and
     global problems of the correction step iteratively until convergence,
     Section 3 after Eq. localProblem, and Algorithm 1's correction step):
     re-solve the last micro step from its starting fine field and states
     with the corrected coarse field in place of T~+ in its Dirichlet data,
     inject again and redo step 4 from T+^n (coarse states as at t_n), until
     max|T+^{n+1,(k)} - T+^{n+1,(k-1)}| <= coupling_tol max|T+^{n+1,(k)}| or
     coupling_sweeps corrections were made.  Only the final solves count in
     the energy account.
  6. Flux-jump coupling (interface_coupling = 1; the alternate global problem
     of Section 3, Eq. globalPbmAlternate): instead of steps 4-5 the
     correction redoes the coarse backward-Euler step from T+^n with only the
     plate's own boundary conditions and the interface load
     G_I = int_gamma (kappa_+ - kappa_-) dT-/dn phi_I dA added to its source
     (see interface_load); the fine field enters the global problem through
     that load alone.

Coefficients are lagged: each backward-Euler step evaluates rho c_e and k_e
at the element mean of the step's starting temperature and the element's
state at that time (with latent heat: the derivative f_pc'(Tb0)).  With
picard_iters = K > 1 each step is K solves from the same starting
temperature T^n, solve j taking its coefficients from the temperature T*_j:
T*_0 = T^n, T*_{j+1} = T*_j + (T_j - T*_j) / 2 for the result T_j of solve j
(Picard iteration of the nonlinear backward-Euler step, relaxed by 1/2: the
plain iteration falls into a two-cycle on the latent-heat peak); the states
stay those of the step's start, and the last solve's coefficients enter the
energy account.  State rule after every step: element mean T_e of the
new temperature; MELTED if T_e > T_melt; else POWDER if it was POWDER; else
SOLID.  Initially an element is POWDER iff its centroid lies within
powder_depth of the top surface, else SOLID.  The fine states live in a
plate-wide map at fine resolution over the patch's depth range, so that
material the patch consolidated keeps its state after the patch has moved
on.

Laser sources (Section 5.2): fine level, the surface Gaussian
q = 3 eta P / (pi R^2) exp(-3 rho^2 / R^2) (integrates to eta P); coarse
level, the surface analogue of the distributed source Q+ = P eta /(r d v Dt):
intensity eta P /(R v Dt) on the axis-aligned rectangle swept by the laser
during the macro step, R wide, integrated exactly against the bilinear hats
(coarse_source = 0), or the fine Gaussian at t_n + Dt (coarse_source = 1).

Scan path: tracks (x0, y0, x1, y1, v) run back to back from t = 0; the laser
is at track j for t in [t_start_j, t_end_j] (first matching track) and off
after the last one.
"""
from __future__ import annotations

from math import floor, hypot

import numpy as np

from . import fem

POWDER, SOLID, MELTED = 0, 1, 2


class ScanPath:
    """Piecewise-linear laser path; times accumulate track durations."""

    def __init__(self, tracks):
        self.tracks = [tuple(float(v) for v in t) for t in tracks]
        self.t_start, self.t_end, self.dur = [], [], []
        t = 0.0
        for (x0, y0, x1, y1, v) in self.tracks:
            d = hypot(x1 - x0, y1 - y0) / v
            self.t_start.append(t)
            self.dur.append(d)
            t = t + d
            self.t_end.append(t)

    def position(self, t):
        """(x, y) of the laser at time t, or None when it is off."""
        for j, (x0, y0, x1, y1, v) in enumerate(self.tracks):
            if t <= self.t_end[j]:
                f = (t - self.t_start[j]) / self.dur[j]
                return (x0 + f * (x1 - x0), y0 + f * (y1 - y0))
        return None

    def swept_pieces(self, ta, tb):
        """Pieces of the path traversed in [ta, tb]: (track, tau_a, tau_b)."""
        out = []
        for j in range(len(self.tracks)):
            a = max(ta, self.t_start[j])
            b = min(tb, self.t_end[j])
            if b > a:
                out.append((j, a, b))
        return out


class Material:
    def __init__(self, cfg):
        self.rho = cfg["rho"]
        self.c0, self.c1 = cfg["c0"], cfg["c1"]
        self.k0, self.k1 = cfg["k0"], cfg["k1"]
        self.Tref = cfg["Tref"]
        self.powder_factor = cfg["powder_factor"]
        self.T_melt = cfg["T_melt"]
        self.latent = float(cfg.get("latent", 0.0))
        self.Tm = 0.5 * (float(cfg.get("T_solidus", 0.0)) + float(cfg.get("T_liquidus", 0.0)))
        self.S = float(cfg.get("pc_sharpness", 0.0))

    def fpc(self, T):
        """The phase-change sigmoid f_pc(T) = (1 + tanh(S (T - Tm))) / 2."""
        return 0.5 * (1.0 + np.tanh(self.S * (T - self.Tm)))

    def fpc_prime(self, T):
        """d f_pc / dT = (S/2)(1 - tanh^2(S (T - Tm)))."""
        th = np.tanh(self.S * (T - self.Tm))
        return 0.5 * self.S * (1.0 - th * th)

    def fpc_secant(self, Tb, Tb0):
        """(f_pc(Tb) - f_pc(Tb0)) / (Tb - Tb0); f_pc' at the midpoint when
        |S (Tb - Tb0)| < 1e-3."""
        d = Tb - Tb0
        near = np.abs(self.S * d) < 1e-3
        quot = (self.fpc(Tb) - self.fpc(Tb0)) / np.where(near, 1.0, d)
        return np.where(near, self.fpc_prime(0.5 * (Tb + Tb0)), quot)

    def coefficients(self, Tbar, state, Tbar0=None):
        """(rho c_e, k_e) at element-mean temperature Tbar and state; Tbar0 =
        the element means at the step's start (default Tbar) for the latent
        heat's secant."""
        if self.latent:
            lat = self.fpc_secant(Tbar, Tbar if Tbar0 is None else Tbar0)
            rc = self.rho * (self.c0 + self.c1 * (Tbar - self.Tref) + self.latent * lat)
        else:
            rc = self.rho * (self.c0 + self.c1 * (Tbar - self.Tref))
        k = self.k0 + self.k1 * (Tbar - self.Tref)
        k = np.where(state == POWDER, self.powder_factor * k, k)
        return rc, k

    def update_state(self, Tbar, state):
        """State after a step whose end temperature has element means Tbar."""
        new = np.where(state == POWDER, POWDER, SOLID).astype(np.uint8)
        new[Tbar > self.T_melt] = MELTED
        return new


# Stefan-Boltzmann constant (CODATA 2018); Section 3.1 prints 5.87e-8.
SIGMA_SB = 5.670374419e-8


class Surface:
    """Heat loss through the top surface (Section 3.1): convection
    h_conv (T - T_amb) on both levels, plus radiation
    sigma eps (T^4 - T_amb^4) on the local (fine) level.  Backward Euler with
    the radiation written as h_rad(T*) (T - T_amb),
    h_rad = sigma eps (T*^2 + T_amb^2)(T* + T_amb), per top face at the face
    mean of the coefficient temperature T* (exact at a Picard fixed point)."""

    def __init__(self, cfg, radiation):
        self.h = float(cfg.get("h_conv", 0.0))
        self.eps = float(cfg.get("emissivity", 0.0)) if radiation else 0.0
        self.T_amb = float(cfg.get("T_amb", 293.0))
        self.sigma = float(cfg.get("sigma_sb", SIGMA_SB))

    def active(self):
        return self.h != 0.0 or self.eps != 0.0

    def coefficient(self, Tf):
        """Transfer coefficient per face at face-mean temperatures Tf."""
        if self.eps == 0.0:
            return np.full(np.shape(Tf), self.h)
        Ta = self.T_amb
        return self.h + self.sigma * self.eps * (Tf * Tf + Ta * Ta) * (Tf + Ta)

    def matrix(self, mesh, Ts):
        return fem.top_face_matrix(mesh, self.coefficient(fem.top_face_mean(mesh, Ts)))


def initial_state(mesh, Lz, powder_depth):
    """POWDER iff the element centroid is within powder_depth of the top."""
    _, _, ke = mesh.elem_ijk
    zc = mesh.origin[2] + (ke + 0.5) * mesh.hz
    return np.where(Lz - zc < powder_depth, POWDER, SOLID).astype(np.uint8)


def be_step(mesh, T, s_e, k_e, F, dir_idx, g, H=None, T_amb=0.0):
    """One backward-Euler step (S + K + H) T' = S T + F + H T_amb with
    T'[dir_idx] = g, S = sum_e s_e Mhat (s_e = rho c_e / dt),
    K = sum_e k_e Khat, H the top-surface transfer matrix (none: adiabatic
    top); returns T'."""
    A = mesh.assemble(s_e, k_e)
    S = mesh.assemble(s_e, np.zeros_like(k_e))
    b = S @ T + F
    if H is not None:
        A = A + H
        b = b + H @ np.full(mesh.nnode, float(T_amb))
    Tn = fem.solve_dirichlet(A, b, dir_idx, g)
    return Tn


def be_picard(mesh, T, coeffs, dt, F, dir_idx, g, iters, surface=None):
    """Backward-Euler step from T with relaxed Picard iterations: solve j (of
    K = max(1, iters)) takes (rho c_e, k_e) = coeffs(element means of T*_j,
    element means of T) and the top-surface matrix of T*_j (surface, if
    active), T*_0 = T, T*_{j+1} = T*_j + (T_j - T*_j) / 2 for the result T_j
    of solve j.  Returns (T', rho c_e, k_e, H) of the last solve."""
    Tb0 = mesh.element_mean(T)
    Ts = T
    K = max(1, int(iters))
    on = surface is not None and surface.active()
    for j in range(K):
        rc, k = coeffs(mesh.element_mean(Ts), Tb0)
        H = surface.matrix(mesh, Ts) if on else None
        Tn = be_step(mesh, T, rc / dt, k, F, dir_idx, g, H, surface.T_amb if on else 0.0)
        if j + 1 < K:
            Ts = Ts + 0.5 * (Tn - Ts)
    return Tn, rc, k, H


def energy_terms(mesh, T, Tn, s_e, k_e, F, dir_idx, dt, H=None, T_amb=0.0):
    """Energy bookkeeping of one step (J): stored heat, laser input, the heat
    entering through the Dirichlet rows (their reactions) and the heat lost
    through the top surface; stored = laser + flux - loss."""
    S = mesh.assemble(s_e, np.zeros_like(k_e))
    K = mesh.assemble(np.zeros_like(s_e), k_e)
    u = Tn - T
    Su = S @ u
    R = Su + K @ Tn - F
    loss = 0.0
    if H is not None:
        q = H @ (Tn - T_amb)
        R = R + q
        loss = dt * float(q.sum())
    return dict(stored=dt * float(Su.sum()), laser=dt * float(F.sum()),
                flux=dt * float(R[dir_idx].sum()), loss=loss)


class SingleLevel:
    """Single-level backward-Euler solve of the whole plate on one mesh with
    the fine Gaussian source (reference for the identity tests)."""

    def __init__(self, cfg, nx, ny, nz, dt):
        self.cfg = cfg
        self.mesh = fem.BoxMesh(nx, ny, nz, cfg["Lx"] / nx, cfg["Ly"] / ny, cfg["Lz"] / nz)
        self.mat = Material(cfg)
        self.path = ScanPath(cfg["tracks"])
        self.dt = dt
        self.T = np.full(self.mesh.nnode, float(cfg["T0"]))
        self.state = initial_state(self.mesh, cfg["Lz"], cfg["powder_depth"])
        _, _, k = self.mesh.node_ijk()
        self.dir_idx = np.flatnonzero(k == 0)
        self.surface = Surface(cfg, radiation=True)
        self.nstep = 0

    def step(self):
        cfg, mesh = self.cfg, self.mesh
        t = (self.nstep + 1) * self.dt
        pos = self.path.position(t)
        if pos is None:
            F = np.zeros(mesh.nnode)
        else:
            F = fem.gaussian_surface_load(mesh, pos[0], pos[1], cfg["P"], cfg["eta"], cfg["radius"])
        g = np.full(len(self.dir_idx), float(cfg["T_bottom"]))
        st = self.state
        Tn, _, _, _ = be_picard(mesh, self.T, lambda Tb, Tb0: self.mat.coefficients(Tb, st, Tb0), self.dt, F,
                                self.dir_idx, g, cfg.get("picard_iters", 1), self.surface)
        self.state = self.mat.update_state(mesh.element_mean(Tn), self.state)
        self.T = Tn
        self.nstep += 1


class TwoLevel:
    """Algorithm 1 with the readings stated in the module docstring."""

    def __init__(self, cfg, energy=True):
        self.cfg = cfg
        self.track_energy = energy
        c = cfg
        self.NXc, self.NYc, self.NZc = c["NXc"], c["NYc"], c["NZc"]
        self.r, self.m = int(c["r"]), int(c["m"])
        self.hc = (c["Lx"] / self.NXc, c["Ly"] / self.NYc, c["Lz"] / self.NZc)
        self.coarse = fem.BoxMesh(self.NXc, self.NYc, self.NZc, *self.hc)
        self.pN = (c["pNXc"], c["pNYc"], c["pNZc"])
        r = self.r
        self.hf = (self.hc[0] / r, self.hc[1] / r, self.hc[2] / r)
        self.nf = (self.pN[0] * r, self.pN[1] * r, self.pN[2] * r)
        self.mat = Material(c)
        self.path = ScanPath(c["tracks"])
        self.Dt = float(c["dt_coarse"])
        self.dt = self.Dt / self.m
        self.Tc = np.full(self.coarse.nnode, float(c["T0"]))
        self.state_c = initial_state(self.coarse, c["Lz"], c["powder_depth"])
        # plate-wide fine state map over the patch's depth range
        self.ok = self.NZc - self.pN[2]
        self.map_dims = (self.NXc * r, self.NYc * r, self.pN[2] * r)
        mx, my, mz = self.map_dims
        ke = np.arange(mz)
        zc = (self.ok * r + ke + 0.5) * self.hf[2]
        layer = np.where(c["Lz"] - zc < c["powder_depth"], POWDER, SOLID).astype(np.uint8)
        self.state_map = np.broadcast_to(layer[:, None, None], (mz, my, mx)).copy()
        _, _, kc = self.coarse.node_ijk()
        self.coarse_bottom = np.flatnonzero(kc == 0)
        self.n = 0
        self.energy = dict(fine_stored=0.0, fine_laser=0.0, fine_flux=0.0, fine_loss=0.0,
                           coarse_stored=0.0, coarse_laser=0.0, coarse_flux=0.0, coarse_loss=0.0)
        self.surf_f = Surface(cfg, radiation=True)    # local domain: convection + radiation
        self.surf_c = Surface(cfg, radiation=False)   # global domain: convection
        self.step_energy = []          # per-solve energy terms (fine and coarse)
        self.origin = self._origin_for(0, None)
        self.Tf = self._interp_fine(self.Tc, self.origin)
        self.Tc_pred = None

    # -- geometry ---------------------------------------------------------
    def _origin_for(self, n, prev):
        pos = self.path.position(n * self.Dt + 0.5 * self.Dt)
        if pos is None:
            if prev is not None:
                return prev
            pos = (0.5 * self.cfg["Lx"], 0.5 * self.cfg["Ly"])
        oi = floor((pos[0] - 0.5 * self.pN[0] * self.hc[0]) / self.hc[0] + 0.5)
        oj = floor((pos[1] - 0.5 * self.pN[1] * self.hc[1]) / self.hc[1] + 0.5)
        oi = min(max(oi, 0), self.NXc - self.pN[0])
        oj = min(max(oj, 0), self.NYc - self.pN[1])
        return (int(oi), int(oj), int(self.ok))

    def fine_mesh(self, origin=None):
        o = self.origin if origin is None else origin
        return fem.BoxMesh(*self.nf, *self.hf,
                           origin=(o[0] * self.hc[0], o[1] * self.hc[1], o[2] * self.hc[2]))

    def _fine_global_ijk(self, origin):
        mesh = self.fine_mesh(origin)
        i, j, k = mesh.node_ijk()
        r = self.r
        return i + origin[0] * r, j + origin[1] * r, k + origin[2] * r

    def _interp_fine(self, Tc, origin):
        """Trilinear interpolant of the coarse field at the patch nodes, with
        exact fractional positions (fine index - r * coarse index) / r."""
        gi, gj, gk = self._fine_global_ijk(origin)
        r, C = self.r, self.coarse
        I = np.minimum(gi // r, C.nx - 1)
        J = np.minimum(gj // r, C.ny - 1)
        K = np.minimum(gk // r, C.nz - 1)
        tx, ty, tz = (gi - I * r) / r, (gj - J * r) / r, (gk - K * r) / r
        out = np.zeros(len(gi))
        for a in range(8):
            ax, ay, az = a & 1, (a >> 1) & 1, (a >> 2) & 1
            w = ((tx if ax else 1.0 - tx) * (ty if ay else 1.0 - ty)
                 * (tz if az else 1.0 - tz))
            out = out + w * Tc[C.node_id(I + ax, J + ay, K + az)]
        return out

    def dirichlet_faces(self, origin=None):
        """(x-, x+, y-, y+, z-) True where the patch face is interior to the
        plate (gamma_D).  The top face is never Dirichlet."""
        o = self.origin if origin is None else origin
        return (o[0] > 0, o[0] + self.pN[0] < self.NXc,
                o[1] > 0, o[1] + self.pN[1] < self.NYc, True)

    def fine_dirichlet(self, origin=None):
        """Ids of the fine Dirichlet nodes and a mask of those on the plate
        bottom (held at T_bottom); the others get coarse data."""
        o = self.origin if origin is None else origin
        mesh = self.fine_mesh(o)
        i, j, k = mesh.node_ijk()
        xm, xp, ym, yp, zm = self.dirichlet_faces(o)
        nx, ny, _ = self.nf
        d = np.zeros(mesh.nnode, dtype=bool)
        if xm:
            d |= i == 0
        if xp:
            d |= i == nx
        if ym:
            d |= j == 0
        if yp:
            d |= j == ny
        d |= k == 0
        idx = np.flatnonzero(d)
        on_bottom = (k[idx] + o[2] * self.r) == 0
        return idx, on_bottom

    def injection_box(self, origin=None):
        """Coarse node index ranges [lo, hi] (inclusive) that coincide with
        free fine nodes."""
        o = self.origin if origin is None else origin
        xm, xp, ym, yp, _ = self.dirichlet_faces(o)
        return ((o[0] + (1 if xm else 0), o[0] + self.pN[0] - (1 if xp else 0)),
                (o[1] + (1 if ym else 0), o[1] + self.pN[1] - (1 if yp else 0)),
                (o[2] + 1, self.NZc))

    def fine_state(self, origin=None):
        """View of the state map under the patch, in fine element order."""
        o = self.origin if origin is None else origin
        r = self.r
        nx, ny, nz = self.nf
        return self.state_map[:, o[1] * r:o[1] * r + ny, o[0] * r:o[0] * r + nx]

    # -- sources -----------------------------------------------------------
    def fine_load(self, mesh, t):
        pos = self.path.position(t)
        if pos is None:
            return np.zeros(mesh.nnode)
        c = self.cfg
        return fem.gaussian_surface_load(mesh, pos[0], pos[1], c["P"], c["eta"], c["radius"])

    def coarse_load(self, n):
        c = self.cfg
        t0, t1 = n * self.Dt, (n + 1) * self.Dt
        if int(c.get("coarse_source", 0)) == 1:
            pos = self.path.position(t1)
            if pos is None:
                return np.zeros(self.coarse.nnode)
            return fem.gaussian_surface_load(self.coarse, pos[0], pos[1], c["P"], c["eta"], c["radius"])
        R = c["radius"]
        rects = []
        for (j, ta, tb) in self.path.swept_pieces(t0, t1):
            x0, y0, x1, y1, v = self.path.tracks[j]
            fa = (ta - self.path.t_start[j]) / self.path.dur[j]
            fb = (tb - self.path.t_start[j]) / self.path.dur[j]
            xa, ya = x0 + fa * (x1 - x0), y0 + fa * (y1 - y0)
            xb, yb = x0 + fb * (x1 - x0), y0 + fb * (y1 - y0)
            q = c["eta"] * c["P"] / (R * v * self.Dt)
            if y0 == y1:
                rects.append((min(xa, xb), max(xa, xb), y0 - 0.5 * R, y0 + 0.5 * R, q))
            elif x0 == x1:
                rects.append((x0 - 0.5 * R, x0 + 0.5 * R, min(ya, yb), max(ya, yb), q))
            else:
                raise ValueError("box coarse source needs axis-aligned tracks")
        return fem.box_surface_load(self.coarse, rects)

    # -- Algorithm 1 ---------------------------------------------------------
    def move_patch(self):
        new = self._origin_for(self.n, self.origin)
        if new == self.origin:
            return False
        interp = self._interp_fine(self.Tc, new)
        old = self.origin
        r = self.r
        nx, ny, nz = self.nf
        mesh = self.fine_mesh(new)
        i, j, k = mesh.node_ijk()
        # position of each new node in the old patch's index frame
        oi = i + (new[0] - old[0]) * r
        oj = j + (new[1] - old[1]) * r
        inside = (oi >= 0) & (oi <= nx) & (oj >= 0) & (oj <= ny)
        T = interp.copy()
        old_id = oi + (nx + 1) * (oj + (ny + 1) * k)
        T[inside] = self.Tf[old_id[inside]]
        self.Tf = T
        self.origin = new
        return True

    def _coarse_coefficients(self, Tbar, Tbar0):
        return self.mat.coefficients(Tbar, self.state_c, Tbar0)

    def predict(self):
        self.move_patch()
        F = self.coarse_load(self.n)
        g = np.full(len(self.coarse_bottom), float(self.cfg["T_bottom"]))
        self.Tc_pred, _, _, _ = be_picard(self.coarse, self.Tc, self._coarse_coefficients, self.Dt, F,
                                          self.coarse_bottom, g, self.cfg.get("picard_iters", 1), self.surf_c)
        self._I_now = None
        self._I_pred = None

    def fine_substep(self, i, coarse_end=None):
        """Micro step i; coarse_end replaces the predictor T~+ in the
        Dirichlet data (re-solves of the iterated coupling)."""
        c = self.cfg
        mesh = self.fine_mesh()
        if self._I_now is None:
            self._I_now = self._interp_fine(self.Tc, self.origin)
            self._I_pred = self._interp_fine(self.Tc_pred, self.origin)
        I_end = self._I_pred if coarse_end is None else self._interp_fine(coarse_end, self.origin)
        w = (i / self.m) if int(c.get("bc_weight_literal", 0)) else ((i + 1) / self.m)
        idx, on_bottom = self.fine_dirichlet()
        g = (1.0 - w) * self._I_now[idx] + w * I_end[idx]
        g[on_bottom] = c["T_bottom"]
        st = self.fine_state()
        st_flat = st.reshape(-1)
        t = (self.n * self.m + i + 1) * self.dt
        F = self.fine_load(mesh, t)
        Tn, rc, k, H = be_picard(mesh, self.Tf, lambda Tb, Tb0: self.mat.coefficients(Tb, st_flat, Tb0), self.dt,
                                 F, idx, g, c.get("picard_iters", 1), self.surf_f)
        if i == self.m - 1:  # start of the last micro step: what a coupling re-solve starts from
            self._last_start = (self.Tf.copy(), st.copy())
        if self.track_energy:
            e = energy_terms(mesh, self.Tf, Tn, rc / self.dt, k, F, idx, self.dt, H, self.surf_f.T_amb)
            self._add_energy("fine", e)
            self._last_fine_e = e
        new_state = self.mat.update_state(mesh.element_mean(Tn), st_flat)
        st[...] = new_state.reshape(st.shape)
        self.Tf = Tn

    def _add_energy(self, level, e, sign=1.0):
        for key in ("stored", "laser", "flux", "loss"):
            self.energy[f"{level}_{key}"] += sign * e[key]
        if sign > 0:
            self.step_energy.append((level, e))
        else:  # the superseded solve is the latest entry of its level
            for j in range(len(self.step_energy) - 1, -1, -1):
                if self.step_energy[j][0] == level:
                    del self.step_energy[j]
                    break

    # -- flux-jump coupling (Section 3, Eqs. deltaDef and globalPbmAlternate) --
    def interface_faces(self, origin=None):
        """The patch faces immersed in the plate (the interface gamma): x-,
        x+, y-, y+ where the patch does not touch the plate's side, and the
        bottom unless it lies on the plate's bottom."""
        o = self.origin if origin is None else origin
        xm, xp, ym, yp, _ = self.dirichlet_faces(o)
        return (xm, xp, ym, yp, o[2] > 0)

    def interface_load(self, Tf=None, k_fine=None, k_coarse=None):
        """G_I = int_gamma (kappa_+ - kappa_-) dT-/dn phi_I dA for every coarse
        node I (Eq. deltaDef's functional of the flux jump), n the outward
        normal of the local domain.  dT-/dn is the normal derivative of the
        fine trilinear field inside the fine element next to the face;
        kappa_- that element's conductivity and kappa_+ the conductivity of the
        coarse element just outside the patch at that face; phi_I the coarse
        trilinear hats.  On each fine face the integrand is a product of two
        bilinear functions, integrated exactly by 2 x 2 Gauss points.
        Defaults: Tf the current fine field; kappa_- from its element means
        and the fine states; kappa_+ from the element means of the coarse field
        and the coarse states (the global step's own lagged coefficients)."""
        T = self.Tf if Tf is None else Tf
        mesh = self.fine_mesh()
        C = self.coarse
        if k_fine is None:
            _, k_fine = self.mat.coefficients(mesh.element_mean(T), self.fine_state().reshape(-1))
        if k_coarse is None:
            _, k_coarse = self.mat.coefficients(C.element_mean(self.Tc), self.state_c)
        k_fine = np.broadcast_to(np.asarray(k_fine, dtype=np.float64), (mesh.nelem,))
        k_coarse = np.broadcast_to(np.asarray(k_coarse, dtype=np.float64), (C.nelem,))
        o, r = self.origin, self.r
        nx, ny, nz = self.nf
        h = self.hf
        G = np.zeros(C.nnode)
        g = 1.0 / np.sqrt(3.0)
        gp = (0.5 * (1.0 - g), 0.5 * (1.0 + g))  # Gauss points on [0, 1], weights 1/2 each
        faces = self.interface_faces()
        # (normal axis d, side s (0 low, 1 high), outward sign)
        for d, side, on in ((0, 0, faces[0]), (0, 1, faces[1]), (1, 0, faces[2]), (1, 1, faces[3]),
                            (2, 0, faces[4])):
            if not on:
                continue
            a1, a2 = [ax for ax in range(3) if ax != d]
            n_t = (nx, ny, nz)
            cnt1, cnt2 = n_t[a1], n_t[a2]
            sign = 1.0 if side else -1.0
            e_d = 0 if side == 0 else n_t[d] - 1            # fine element index across d
            for u1 in range(2):
                for u2 in range(2):
                    xi1, xi2, w = gp[u1], gp[u2], 0.25
                    e1, e2 = np.meshgrid(np.arange(cnt1), np.arange(cnt2), indexing="ij")
                    e1, e2 = e1.ravel(), e2.ravel()
                    eidx = [0, 0, 0]
                    eidx[d], eidx[a1], eidx[a2] = np.full(e1.shape, e_d), e1, e2
                    # dT/dx_d in the element at in-plane reference point (xi1, xi2)
                    grad = np.zeros(e1.shape)
                    for b1 in range(2):
                        for b2 in range(2):
                            wt = (xi1 if b1 else 1.0 - xi1) * (xi2 if b2 else 1.0 - xi2)
                            nid = []
                            for bd in range(2):
                                idx = [None, None, None]
                                idx[d] = eidx[d] + bd
                                idx[a1] = eidx[a1] + b1
                                idx[a2] = eidx[a2] + b2
                                nid.append(mesh.node_id(idx[0], idx[1], idx[2]))
                            grad += wt * (T[nid[1]] - T[nid[0]]) / h[d]
                    dTdn = sign * grad
                    fe = eidx[0] + nx * (eidx[1] + ny * eidx[2])
                    kminus = k_fine[fe]
                    # global fine coordinates of the Gauss point (in fine index units)
                    gf = [None, None, None]
                    gf[d] = np.full(e1.shape, float((e_d + side) + [o[0], o[1], o[2]][d] * r))
                    gf[a1] = e1 + xi1 + [o[0], o[1], o[2]][a1] * r
                    gf[a2] = e2 + xi2 + [o[0], o[1], o[2]][a2] * r
                    # coarse element just outside the patch, and the hats of the face
                    cc = [np.floor(gf[ax] / r).astype(np.int64) for ax in range(3)]
                    out_d = [o[0], o[1], o[2]][d] + (self.pN[d] if side else 0) - (0 if side else 1)
                    cc[d] = np.full(e1.shape, out_d)
                    kplus = k_coarse[cc[0] + C.nx * (cc[1] + C.ny * cc[2])]
                    jump = (kplus - kminus) * dTdn * w * h[a1] * h[a2]
                    # coarse hats on the face plane: bilinear in the two in-plane axes
                    Id = [o[0], o[1], o[2]][d] + (self.pN[d] if side else 0)
                    for c1 in range(2):
                        for c2 in range(2):
                            ci = [None, None, None]
                            ci[d] = np.full(e1.shape, Id)
                            ci[a1] = cc[a1] + c1
                            ci[a2] = cc[a2] + c2
                            t1 = gf[a1] / r - cc[a1]
                            t2 = gf[a2] / r - cc[a2]
                            phi = (t1 if c1 else 1.0 - t1) * (t2 if c2 else 1.0 - t2)
                            np.add.at(G, C.node_id(ci[0], ci[1], ci[2]), jump * phi)
        return G

    def _flux_correction(self):
        """The global backward-Euler step of Eq. globalPbmAlternate from T+^n
        with the interface load of the fine field at the end of the macro step
        (not committed): returns (T+^{n+1}, coarse states, energy terms)."""
        c = self.cfg
        G = self.interface_load()
        F = self.coarse_load(self.n)
        g = np.full(len(self.coarse_bottom), float(c["T_bottom"]))
        Tn, rc, k, H = be_picard(self.coarse, self.Tc, self._coarse_coefficients, self.Dt, F + G,
                                 self.coarse_bottom, g, c.get("picard_iters", 1), self.surf_c)
        e = None
        if self.track_energy:
            e = energy_terms(self.coarse, self.Tc, Tn, rc / self.Dt, k, F + G, self.coarse_bottom, self.Dt, H,
                             self.surf_c.T_amb)
            gi = self.Dt * float(G.sum())
            e["laser"] -= gi       # the interface heat counts as flux through the boundary
            e["flux"] += gi
            e["interface"] = gi
        return Tn, self.mat.update_state(self.coarse.element_mean(Tn), self.state_c), e

    def restrict_and_correct(self):
        """Steps 4 and 5: correction, iterated with re-solves of the last
        micro step while coupling_sweeps allows and the coarse field moves."""
        c = self.cfg
        if int(c.get("interface_coupling", 0)) == 1:
            Tn, state, e = self._flux_correction()
            if self.track_energy:
                self._add_energy("coarse", e)
            self.state_c = state
            self.Tc = Tn
            self.Tc_pred = None
            return
        sweeps = int(c.get("coupling_sweeps", 1))
        tol = float(c.get("coupling_tol", 1e-10))
        Tn, state, e = self._correction()
        self.coupling_history = []
        for _ in range(1, sweeps):
            # last micro step again, from its start, ending on the corrected field
            T0f, st0 = self._last_start
            self.fine_state()[...] = st0
            self.Tf = T0f.copy()
            if self.track_energy:
                self._add_energy("fine", self._last_fine_e, sign=-1.0)
            self.fine_substep(self.m - 1, coarse_end=Tn)
            Tk, state_k, e_k = self._correction()
            diff = float(np.max(np.abs(Tk - Tn)) / np.max(np.abs(Tk)))
            self.coupling_history.append(diff)
            Tn, state, e = Tk, state_k, e_k
            if diff <= tol:
                break
        if self.track_energy:
            self._add_energy("coarse", e)
        self.state_c = state
        self.Tc = Tn
        self.Tc_pred = None

    def _correction(self):
        """Injection and the coarse re-solve from T+^n (step 4), not committed:
        returns (T+^{n+1}, coarse states, energy terms or None)."""
        c = self.cfg
        (i0, i1), (j0, j1), (k0, k1) = self.injection_box()
        I, J, K = np.meshgrid(np.arange(i0, i1 + 1), np.arange(j0, j1 + 1),
                              np.arange(k0, k1 + 1), indexing="ij")
        I, J, K = I.ravel(), J.ravel(), K.ravel()
        r, o = self.r, self.origin
        fi, fj, fk = (I - o[0]) * r, (J - o[1]) * r, (K - o[2]) * r
        nx, ny, _ = self.nf
        inj_vals = self.Tf[fi + (nx + 1) * (fj + (ny + 1) * fk)]
        inj_idx = self.coarse.node_id(I, J, K)
        F = self.coarse_load(self.n)
        dir_idx = np.concatenate([self.coarse_bottom, inj_idx])
        g = np.concatenate([np.full(len(self.coarse_bottom), float(c["T_bottom"])), inj_vals])
        Tn, rc, k, H = be_picard(self.coarse, self.Tc, self._coarse_coefficients, self.Dt, F, dir_idx, g,
                                 c.get("picard_iters", 1), self.surf_c)
        e = (energy_terms(self.coarse, self.Tc, Tn, rc / self.Dt, k, F, dir_idx, self.Dt, H, self.surf_c.T_amb)
             if self.track_energy else None)
        return Tn, self.mat.update_state(self.coarse.element_mean(Tn), self.state_c), e

    def macro_step(self):
        self.predict()
        for i in range(self.m):
            self.fine_substep(i)
        self.restrict_and_correct()
        self.n += 1

    def run(self, n_macro):
        for _ in range(n_macro):
            self.macro_step()
        return self

    def melt_mask_fine(self):
        return self.fine_state().reshape(-1) == MELTED
