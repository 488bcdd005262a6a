"""Pins of the oracle's finite-element building blocks against quadrature,
closed forms and brute force (no GPU)."""
import itertools
from math import erf, exp, pi, sqrt

import numpy as np
import pytest
from scipy import integrate

from oracle import fem


def _gauss_element_matrices(hx, hy, hz):
    """Element matrices by 2-point Gauss quadrature of the trilinear shape
    functions (exact for these polynomial degrees), written independently of
    the Kronecker formula."""
    gp = [0.5 - 0.5 / sqrt(3.0), 0.5 + 0.5 / sqrt(3.0)]
    M = np.zeros((8, 8))
    K = np.zeros((8, 8))
    vol = hx * hy * hz
    for (u, v, w) in itertools.product(gp, gp, gp):
        N = np.zeros(8)
        dN = np.zeros((8, 3))
        for a in range(8):
            ax, ay, az = a & 1, (a >> 1) & 1, (a >> 2) & 1
            fx = u if ax else 1 - u
            fy = v if ay else 1 - v
            fz = w if az else 1 - w
            gx = (1 if ax else -1) / hx
            gy = (1 if ay else -1) / hy
            gz = (1 if az else -1) / hz
            N[a] = fx * fy * fz
            dN[a] = (gx * fy * fz, fx * gy * fz, fx * fy * gz)
        M += vol / 8 * np.outer(N, N)
        K += vol / 8 * dN @ dN.T
    return M, K


def test_element_matrices_match_quadrature():
    for h in [(1.0, 1.0, 1.0), (2e-5, 3e-5, 1.5e-5), (0.125, 0.5, 0.25)]:
        M, K = fem.element_matrices(*h)
        Mq, Kq = _gauss_element_matrices(*h)
        assert np.allclose(M, Mq, rtol=1e-13, atol=0)
        assert np.allclose(K, Kq, rtol=1e-12, atol=1e-12 * np.abs(Kq).max())
        # invariants: mass sums to the volume, constants are in K's kernel
        assert abs(M.sum() - h[0] * h[1] * h[2]) < 1e-14 * h[0] * h[1] * h[2]
        assert np.abs(K @ np.ones(8)).max() < 1e-12 * np.abs(K).max()


def test_assembly_row_sums_and_symmetry():
    mesh = fem.BoxMesh(3, 2, 4, 0.1, 0.2, 0.05)
    rng = np.random.default_rng(0)
    s = rng.uniform(1, 2, mesh.nelem)
    k = rng.uniform(1, 2, mesh.nelem)
    A = mesh.assemble(s, k)
    assert abs(A - A.T).max() < 1e-14
    K = mesh.assemble(np.zeros_like(s), k)
    assert np.abs(K @ np.ones(mesh.nnode)).max() < 1e-12
    S = mesh.assemble(s, np.zeros_like(k))
    # 1^T S 1 = sum_e s_e vol_e
    assert abs(S.sum() - (s * 0.1 * 0.2 * 0.05).sum()) < 1e-14


def test_hat_gauss_against_quadrature():
    xs = np.linspace(0.0, 1e-3, 17)
    xc, R = 0.37e-3, 50e-6
    G = fem.hat_gauss_1d(xs, xc, R)
    h = xs[1] - xs[0]

    def hat(i, x):
        return max(0.0, 1.0 - abs(x - xs[i]) / h)
    for i in range(len(xs)):
        a, b = max(xs[0], xs[i] - h), min(xs[-1], xs[i] + h)
        kinks = [p for p in (xs[i],) if a < p < b]
        val, _ = integrate.quad(lambda x: hat(i, x) * exp(-3 * (x - xc) ** 2 / R ** 2),
                                a, b, points=kinks or None, epsabs=1e-20, epsrel=1e-13)
        # relative to the total integral (tail cancellation is ~1e-16 of it)
        assert abs(G[i] - val) <= 1e-12 * max(abs(val), 1e-3 * R)
    # partition of unity: the sum is the integral over the mesh (erf form)
    al = sqrt(3) / R
    tot = sqrt(pi) / (2 * al) * (erf(al * (xs[-1] - xc)) - erf(al * (xs[0] - xc)))
    assert abs(G.sum() - tot) < 1e-14 * tot


def test_gaussian_load_total_power():
    # laser well inside the top face: sum of nodal loads = eta P
    mesh = fem.BoxMesh(32, 32, 2, 15.625e-6, 15.625e-6, 15.625e-6)
    F = fem.gaussian_surface_load(mesh, 0.25e-3, 0.26e-3, 195.0, 0.4, 50e-6)
    assert abs(F.sum() - 78.0) < 1e-12 * 78.0
    # non-negative up to the erf-difference cancellation in the far tail
    assert np.all(F[mesh.top_nodes()] >= -1e-15 * F.max())
    assert np.count_nonzero(F) <= mesh.nnx * mesh.nny
    # laser on an edge: half the power
    F2 = fem.gaussian_surface_load(mesh, 0.0, 0.25e-3, 195.0, 0.4, 50e-6)
    assert abs(F2.sum() - 39.0) < 1e-10 * 39.0


def test_hat_box_against_quadrature():
    xs = np.linspace(0.0, 1.0, 9)
    a, b = 0.2, 0.71
    H = fem.hat_box_1d(xs, a, b)
    h = xs[1] - xs[0]
    for i in range(len(xs)):
        kinks = [p for p in (xs[i] - h, xs[i], xs[i] + h) if a < p < b]
        val, _ = integrate.quad(lambda x: max(0.0, 1.0 - abs(x - xs[i]) / h), a, b,
                                points=kinks or None, epsabs=1e-15)
        assert abs(H[i] - val) < 1e-13
    assert abs(H.sum() - (b - a)) < 1e-15
    # clipped at the mesh ends
    assert abs(fem.hat_box_1d(xs, -0.3, 0.1).sum() - 0.1) < 1e-15


def test_trilinear_reproduces_trilinear_fields():
    mesh = fem.BoxMesh(4, 3, 2, 0.5, 0.25, 0.125)
    x, y, z = mesh.node_xyz()
    f = lambda x, y, z: 1 + 2 * x - 3 * y + 0.5 * z + 0.7 * x * y * z - x * z
    T = f(x, y, z)
    rng = np.random.default_rng(1)
    px = rng.uniform(0, 2, 50)
    py = rng.uniform(0, 0.75, 50)
    pz = rng.uniform(0, 0.25, 50)
    assert np.allclose(fem.trilinear(mesh, T, px, py, pz), f(px, py, pz), rtol=0, atol=1e-13)


def test_dense_brute_force_solve():
    """Tiny system: dense assembly from quadrature element matrices with
    explicit loops and numpy.linalg.solve against the sparse Dirichlet solve."""
    nx, ny, nz = 2, 2, 2
    h = (0.3, 0.2, 0.1)
    mesh = fem.BoxMesh(nx, ny, nz, *h)
    Mq, Kq = _gauss_element_matrices(*h)
    rng = np.random.default_rng(2)
    s = rng.uniform(1, 3, mesh.nelem)
    k = rng.uniform(0.1, 2, mesh.nelem)
    n = mesh.nnode
    A = np.zeros((n, n))
    e = 0
    for ke in range(nz):
        for je in range(ny):
            for ie in range(nx):
                nodes = [(ie + (a & 1)) + 3 * ((je + ((a >> 1) & 1)) + 3 * (ke + (a >> 2))) for a in range(8)]
                for a in range(8):
                    for b in range(8):
                        A[nodes[a], nodes[b]] += s[e] * Mq[a, b] + k[e] * Kq[a, b]
                e += 1
    b = rng.uniform(-1, 1, n)
    dir_idx = np.array([0, 1, 2, 3, 4, 5, 6, 7, 8])  # bottom layer
    g = rng.uniform(0, 1, len(dir_idx))
    Ad = A.copy()
    bd = b.copy()
    for i, gi in zip(dir_idx, g):
        Ad[i, :] = 0
        Ad[i, i] = 1
        bd[i] = gi
    x_dense = np.linalg.solve(Ad, bd)
    x = fem.solve_dirichlet(mesh.assemble(s, k), b, dir_idx, g)
    assert np.allclose(x, x_dense, rtol=1e-12, atol=1e-12)


def test_top_face_matrix_against_quadrature():
    """The top-surface transfer matrix equals 2 x 2 Gauss quadrature of the
    products of bilinear face hats, face by face, with per-face coefficients."""
    mesh = fem.BoxMesh(3, 2, 2, 0.1, 0.2, 0.3, origin=(0.5, -0.25, 1.0))
    rng = np.random.default_rng(7)
    h_f = rng.uniform(1.0, 5.0, mesh.nx * mesh.ny)
    H = fem.top_face_matrix(mesh, h_f).toarray()
    ref = np.zeros((mesh.nnode, mesh.nnode))
    gp = np.array([0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)])
    f = 0
    for je in range(mesh.ny):
        for ie in range(mesh.nx):
            nodes = [mesh.node_id(ie + ax, je + ay, mesh.nz) for ay in (0, 1) for ax in (0, 1)]
            for u in gp:
                for v in gp:
                    phi = np.array([(1 - u) * (1 - v), u * (1 - v), (1 - u) * v, u * v])
                    w = 0.25 * mesh.hx * mesh.hy
                    for a in range(4):
                        for b in range(4):
                            ref[nodes[a], nodes[b]] += h_f[f] * w * phi[a] * phi[b]
            f += 1
    assert np.allclose(H, ref, rtol=1e-13, atol=1e-16)
    assert abs(H.sum() - np.sum(h_f) * mesh.hx * mesh.hy) <= 1e-13 * H.sum()
