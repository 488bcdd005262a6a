"""Q1 hexahedral finite elements on a uniform box mesh, FP64, assembled CSR.

Test infrastructure only (see the package docstring).

Discretisation of the heat equation Eq. (thermalEqn) (Section 2.1) without
the latent term: per element e with constant volumetric heat capacity
rho*c_e and conductivity k_e the element matrices are the exact integrals

    Mhat_e[a, b] = int_e phi_a phi_b        Khat_e[a, b] = int_e grad phi_a . grad phi_b

of trilinear shape functions.  On a box element they are Kronecker products
of the 1D linear-element matrices M1 = (h/6)[[2,1],[1,2]],
K1 = (1/h)[[1,-1],[-1,1]] (local node a = ax + 2 ay + 4 az, x fastest).

Mesh convention: nodes (i, j, k), i in [0, nx], x fastest; global node id
i + (nx+1) (j + (ny+1) k); element (ie, je, ke) id ie + nx (je + ny ke);
z = 0 is the bottom of the plate, z = Lz the top surface.
"""
from __future__ import annotations

from math import erf, exp, pi, sqrt

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def line_matrices(h):
    """1D linear element mass and stiffness matrices on an element of length h."""
    M = (h / 6.0) * np.array([[2.0, 1.0], [1.0, 2.0]])
    K = (1.0 / h) * np.array([[1.0, -1.0], [-1.0, 1.0]])
    return M, K


def element_matrices(hx, hy, hz):
    """Exact trilinear mass and stiffness matrices of an hx*hy*hz box element."""
    Mx, Kx = line_matrices(hx)
    My, Ky = line_matrices(hy)
    Mz, Kz = line_matrices(hz)
    M = np.kron(Mz, np.kron(My, Mx))
    K = (np.kron(Mz, np.kron(My, Kx)) + np.kron(Mz, np.kron(Ky, Mx))
         + np.kron(Kz, np.kron(My, Mx)))
    return M, K


class BoxMesh:
    """Uniform hexahedral mesh of nx*ny*nz elements of size hx*hy*hz whose
    node (0,0,0) sits at physical point ``origin``."""

    def __init__(self, nx, ny, nz, hx, hy, hz, origin=(0.0, 0.0, 0.0)):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.hx, self.hy, self.hz = float(hx), float(hy), float(hz)
        self.origin = tuple(float(o) for o in origin)
        self.nnx, self.nny, self.nnz = self.nx + 1, self.ny + 1, self.nz + 1
        self.nnode = self.nnx * self.nny * self.nnz
        self.nelem = self.nx * self.ny * self.nz
        ie, je, ke = np.meshgrid(np.arange(self.nx), np.arange(self.ny),
                                 np.arange(self.nz), indexing="ij")
        ie, je, ke = (a.transpose(2, 1, 0).ravel() for a in (ie, je, ke))
        conn = np.empty((self.nelem, 8), dtype=np.int64)
        for a in range(8):
            ax, ay, az = a & 1, (a >> 1) & 1, (a >> 2) & 1
            conn[:, a] = self.node_id(ie + ax, je + ay, ke + az)
        self.conn = conn
        self.elem_ijk = (ie, je, ke)

    def node_id(self, i, j, k):
        return i + self.nnx * (j + self.nny * k)

    def node_ijk(self):
        """Index arrays (i, j, k) of every node in id order."""
        n = np.arange(self.nnode)
        return n % self.nnx, (n // self.nnx) % self.nny, n // (self.nnx * self.nny)

    def node_xyz(self):
        i, j, k = self.node_ijk()
        return (self.origin[0] + i * self.hx, self.origin[1] + j * self.hy,
                self.origin[2] + k * self.hz)

    def top_nodes(self):
        """Ids of the nodes on the top face k = nz, ordered (i fastest, then j)."""
        j, i = np.meshgrid(np.arange(self.nny), np.arange(self.nnx), indexing="ij")
        return self.node_id(i.ravel(), j.ravel(), self.nz)

    def element_mean(self, T):
        """Element-mean of nodal T, summed in local node order 0..7 and scaled
        by 0.125 (the order both levels use for the state threshold)."""
        s = T[self.conn[:, 0]].copy()
        for a in range(1, 8):
            s = s + T[self.conn[:, a]]
        return s * 0.125

    def assemble(self, s_e, k_e):
        """CSR matrix sum_e s_e Mhat + k_e Khat."""
        M, K = element_matrices(self.hx, self.hy, self.hz)
        s_e = np.asarray(s_e, dtype=np.float64)
        k_e = np.asarray(k_e, dtype=np.float64)
        data = (s_e[:, None, None] * M[None] + k_e[:, None, None] * K[None])
        rows = np.repeat(self.conn[:, :, None], 8, axis=2)
        cols = np.repeat(self.conn[:, None, :], 8, axis=1)
        A = sp.coo_matrix((data.ravel(), (rows.ravel(), cols.ravel())),
                          shape=(self.nnode, self.nnode)).tocsr()
        A.sum_duplicates()
        return A


def top_face_matrix(mesh, h_f):
    """CSR matrix sum_f h_f int_f phi_a phi_b dA over the top faces (z = top,
    one per top-layer element, x fastest then y): the exact surface mass of
    the bilinear face hats, M1x (x) M1y per face (local face node
    a = ax + 2 ay), times the face's transfer coefficient h_f [W/(m^2 K)]."""
    Mx, _ = line_matrices(mesh.hx)
    My, _ = line_matrices(mesh.hy)
    Mf = np.kron(My, Mx)
    je, ie = np.meshgrid(np.arange(mesh.ny), np.arange(mesh.nx), indexing="ij")
    ie, je = ie.ravel(), je.ravel()
    conn = np.stack([mesh.node_id(ie + ax, je + ay, mesh.nz) for ay in (0, 1) for ax in (0, 1)], axis=1)
    h_f = np.broadcast_to(np.asarray(h_f, dtype=np.float64), (len(ie),))
    data = h_f[:, None, None] * Mf[None]
    rows = np.repeat(conn[:, :, None], 4, axis=2)
    cols = np.repeat(conn[:, None, :], 4, axis=1)
    H = sp.coo_matrix((data.ravel(), (rows.ravel(), cols.ravel())), shape=(mesh.nnode, mesh.nnode)).tocsr()
    H.sum_duplicates()
    return H


def top_face_mean(mesh, T):
    """Mean of the four nodal values of every top face (x fastest, then y)."""
    je, ie = np.meshgrid(np.arange(mesh.ny), np.arange(mesh.nx), indexing="ij")
    ie, je = ie.ravel(), je.ravel()
    s = T[mesh.node_id(ie, je, mesh.nz)].copy()
    s = s + T[mesh.node_id(ie + 1, je, mesh.nz)]
    s = s + T[mesh.node_id(ie, je + 1, mesh.nz)]
    s = s + T[mesh.node_id(ie + 1, je + 1, mesh.nz)]
    return s * 0.25


def solve_spd(A, b):
    """Solve the SPD system A x = b: SuperLU for small systems, CG to a
    relative residual of 1e-14 for large ones."""
    n = A.shape[0]
    if n == 0:
        return np.zeros(0)
    if n <= 60000:
        return spla.spsolve(A.tocsc(), b)
    d = A.diagonal()
    Pinv = sp.diags(1.0 / d)
    x, info = spla.cg(A, b, rtol=1e-14, atol=0.0, M=Pinv, maxiter=20000)
    if info != 0:
        raise RuntimeError(f"oracle CG did not converge (info={info})")
    return x


def solve_dirichlet(A, b, dir_idx, g):
    """Solve A x = b with x[dir_idx] = g prescribed: free rows of the system
    with the Dirichlet columns moved to the right-hand side."""
    n = A.shape[0]
    mask = np.zeros(n, dtype=bool)
    mask[dir_idx] = True
    free = np.flatnonzero(~mask)
    x = np.zeros(n)
    x[dir_idx] = g
    A_fD = A[free][:, dir_idx]
    A_ff = A[free][:, free]
    x[free] = solve_spd(A_ff.tocsr(), b[free] - A_fD @ np.asarray(g, dtype=np.float64))
    return x


# ---------------------------------------------------------------------------
# Laser loads (Section 5.2, Q_- and Q_+; surface form, see twolevel docstring)
# ---------------------------------------------------------------------------

def hat_gauss_1d(xs, xc, R):
    """G_i = int_{xs[0]}^{xs[-1]} hat_i(x) exp(-3 (x - xc)^2 / R^2) dx for the
    linear hat functions of the uniform node coordinates ``xs``, in closed
    form: on each element [a, b] the two linear weights integrate against the
    Gaussian as erf and exp terms."""
    n = len(xs)
    G = np.zeros(n)
    al = sqrt(3.0) / R
    for e in range(n - 1):
        a, b = float(xs[e]), float(xs[e + 1])
        h = b - a
        E0 = (sqrt(pi) / (2.0 * al)) * (erf(al * (b - xc)) - erf(al * (a - xc)))
        E1 = (exp(-(al * (a - xc)) ** 2) - exp(-(al * (b - xc)) ** 2)) / (2.0 * al * al)
        # int (x - a)/h g = (E1 + (xc - a) E0)/h ; int (b - x)/h g = ((b - xc) E0 - E1)/h
        G[e + 1] += (E1 + (xc - a) * E0) / h
        G[e] += ((b - xc) * E0 - E1) / h
    return G


def gaussian_surface_load(mesh, xc, yc, P, eta, R):
    """Nodal load F_i = int_top q phi_i dA of the surface Gaussian
    q = 3 eta P / (pi R^2) exp(-3 ((x-xc)^2 + (y-yc)^2) / R^2) on the top face
    of ``mesh``; zero elsewhere.  The exponent 3 is the paper's (Section 5.2);
    the amplitude makes q integrate to eta P over the plane."""
    F = np.zeros(mesh.nnode)
    xs = mesh.origin[0] + mesh.hx * np.arange(mesh.nnx)
    ys = mesh.origin[1] + mesh.hy * np.arange(mesh.nny)
    Gx = hat_gauss_1d(xs, xc, R)
    Gy = hat_gauss_1d(ys, yc, R)
    amp = 3.0 * eta * P / (pi * R * R)
    F[mesh.top_nodes()] = amp * np.outer(Gy, Gx).ravel()
    return F


def hat_box_1d(xs, a, b):
    """H_i = int_a^b hat_i(x) dx for the uniform node coordinates ``xs``
    (exact piecewise-quadratic antiderivative; [a, b] clipped to the mesh)."""
    n = len(xs)
    H = np.zeros(n)
    a = max(a, float(xs[0]))
    b = min(b, float(xs[-1]))
    if b <= a:
        return H
    for e in range(n - 1):
        x0, x1 = float(xs[e]), float(xs[e + 1])
        lo, hi = max(a, x0), min(b, x1)
        if hi <= lo:
            continue
        h = x1 - x0
        # rising weight (x - x0)/h goes to node e+1, falling (x1 - x)/h to node e
        H[e + 1] += ((hi - x0) ** 2 - (lo - x0) ** 2) / (2.0 * h)
        H[e] += ((x1 - lo) ** 2 - (x1 - hi) ** 2) / (2.0 * h)
    return H


def box_surface_load(mesh, rects):
    """Nodal load of piecewise-constant surface fluxes: ``rects`` is a list of
    (x0, x1, y0, y1, q) axis-aligned rectangles of intensity q on the top face."""
    F = np.zeros(mesh.nnode)
    xs = mesh.origin[0] + mesh.hx * np.arange(mesh.nnx)
    ys = mesh.origin[1] + mesh.hy * np.arange(mesh.nny)
    top = mesh.top_nodes()
    for (x0, x1, y0, y1, q) in rects:
        Hx = hat_box_1d(xs, x0, x1)
        Hy = hat_box_1d(ys, y0, y1)
        F[top] += q * np.outer(Hy, Hx).ravel()
    return F


def trilinear(coarse, Tc, x, y, z):
    """Trilinear interpolant of the nodal field Tc of BoxMesh ``coarse`` at
    physical points (x, y, z) (arrays), points inside the mesh."""
    fx = (np.asarray(x) - coarse.origin[0]) / coarse.hx
    fy = (np.asarray(y) - coarse.origin[1]) / coarse.hy
    fz = (np.asarray(z) - coarse.origin[2]) / coarse.hz
    I = np.clip(np.floor(fx).astype(np.int64), 0, coarse.nx - 1)
    J = np.clip(np.floor(fy).astype(np.int64), 0, coarse.ny - 1)
    K = np.clip(np.floor(fz).astype(np.int64), 0, coarse.nz - 1)
    tx, ty, tz = fx - I, fy - J, fz - K
    out = np.zeros(np.shape(fx))
    for a in range(8):
        ax, ay, az = a & 1, (a >> 1) & 1, (a >> 2) & 1
        w = ((tx if ax else 1.0 - tx) * (ty if ay else 1.0 - ty)
             * (tz if az else 1.0 - tz))
        out = out + w * Tc[coarse.node_id(I + ax, J + ay, K + az)]
    return out
