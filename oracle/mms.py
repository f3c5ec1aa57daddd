"""Manufactured-solution verification (oracle, test infrastructure only).

Section 3.1.1, Eqs. 4-8: with I_ion = 0, chi = Cm = 1 and sigma = I the monodomain equation
becomes dV/dt - lap V = 0; the target w = exp(-k t) cos(w1 x + w2 y - lam t) solves it with the
source r = dw/dt - lap w = exp(-kt)[-k cos(.) + lam sin(.)] + (w1^2 + w2^2) w (Eq. 7).
The paper does not print k, w1, w2, lam; the defaults below are our choice (any smooth choice
serves a convergence-rate check).

mms2d: the paper's setting - unit square, P1 triangles, Dirichlet data w on the whole boundary,
       Crank-Nicolson, PCG.
mms3d: the hot-path setting - P1 tetrahedra of the slab generator with zero-flux boundaries,
       w = exp(-k t) cos(pi x / Lx) cos(pi y / Ly) (zero normal derivative on every face),
       source r = (-k + pi^2/Lx^2 + pi^2/Ly^2) w injected through the I_stim slot of b.
Both use the source at theta-weighted time levels, theta r^{k+1} + (1 - theta) r^k.
"""
import numpy as np

from . import fem
from .monodomain import rhs
from .pcg import pcg

K_DECAY, W1, W2, LAM = 0.05, 2.0 * np.pi, np.pi, 1.0


def w2d(x, y, t, k=K_DECAY, w1=W1, w2=W2, lam=LAM):
    return np.exp(-k * t) * np.cos(w1 * x + w2 * y - lam * t)


def r2d(x, y, t, k=K_DECAY, w1=W1, w2=W2, lam=LAM):
    ph = w1 * x + w2 * y - lam * t
    e = np.exp(-k * t)
    return e * (-k * np.cos(ph) + lam * np.sin(ph)) + (w1 ** 2 + w2 ** 2) * e * np.cos(ph)


def unit_square_triangles(n):
    """n x n nodes on [0,1]^2, each square cut into two triangles along one diagonal."""
    g = np.linspace(0.0, 1.0, n)
    X, Y = np.meshgrid(g, g, indexing="xy")
    xy = np.stack([X.ravel(), Y.ravel()], axis=1)
    idx = np.arange(n * n).reshape(n, n)
    a = idx[:-1, :-1].ravel()
    b = idx[:-1, 1:].ravel()
    c = idx[1:, :-1].ravel()
    d = idx[1:, 1:].ravel()
    tris = np.concatenate([np.stack([a, b, d], 1), np.stack([a, d, c], 1)]).astype(np.int64)
    on_bnd = (xy[:, 0] == 0.0) | (xy[:, 0] == 1.0) | (xy[:, 1] == 0.0) | (xy[:, 1] == 1.0)
    return xy, tris, on_bnd


def mms2d(n, dt, t_end, theta=0.5, tol=1e-8):
    """Run the paper's 2D check; returns (L2 error at t_end, max nodal error at t_end)."""
    xy, tris, bnd = unit_square_triangles(n)
    Me, Ke = fem.tri_element_matrices(xy, tris)
    M = fem.assemble(tris, Me, xy.shape[0])
    K = fem.assemble(tris, Ke, xy.shape[0])
    A = fem.system_matrix(M, K, 1.0, 1.0, theta, dt)
    I = np.nonzero(~bnd)[0]
    B = np.nonzero(bnd)[0]
    A_II = A[I][:, I].tocsr()
    A_IB = A[I][:, B].tocsr()
    d_II = A_II.diagonal()
    x, y = xy[:, 0], xy[:, 1]
    V = w2d(x, y, 0.0)
    V_prev = V.copy()
    steps = int(round(t_end / dt))
    for k in range(steps):
        t0, t1 = k * dt, (k + 1) * dt
        src = theta * r2d(x, y, t1) + (1.0 - theta) * r2d(x, y, t0)
        b = rhs(M, K, V, np.zeros_like(V), src, 1.0, 1.0, theta, dt)
        wb = w2d(x[B], y[B], t1)
        x0 = (2.0 * V - V_prev)[I]
        vi, _, _, _ = pcg(A_II, b[I] - A_IB @ wb, x0, d_II, tol, tol, 10000)
        V_new = np.empty_like(V)
        V_new[I] = vi
        V_new[B] = wb
        V_prev, V = V, V_new
    e = V - w2d(x, y, steps * dt)
    return float(np.sqrt(e @ (M @ e))), float(np.abs(e).max())


def w3d(x, y, t, lx, ly, k=K_DECAY):
    return np.exp(-k * t) * np.cos(np.pi * x / lx) * np.cos(np.pi * y / ly)


def r3d(x, y, t, lx, ly, k=K_DECAY):
    return (-k + np.pi ** 2 / lx ** 2 + np.pi ** 2 / ly ** 2) * w3d(x, y, t, lx, ly, k)


def mms3d(mesh, lx, ly, dt, t_end, theta=0.5, tol=1e-12):
    """Zero-flux 3D check on a tetrahedral slab; returns (L2 error, max nodal error) at t_end."""
    xyz, tets = mesh.xyz, mesh.tets
    iso = np.tile(np.array([1.0, 0.0, 0.0]), (tets.shape[0], 1))
    M, K = fem.mass_stiffness(xyz, tets, iso, 1.0, 1.0)
    A = fem.system_matrix(M, K, 1.0, 1.0, theta, dt)
    d = A.diagonal()
    x, y = xyz[:, 0], xyz[:, 1]
    V = w3d(x, y, 0.0, lx, ly)
    V_prev = V.copy()
    steps = int(round(t_end / dt))
    for k in range(steps):
        t0, t1 = k * dt, (k + 1) * dt
        src = theta * r3d(x, y, t1, lx, ly) + (1.0 - theta) * r3d(x, y, t0, lx, ly)
        b = rhs(M, K, V, np.zeros_like(V), src, 1.0, 1.0, theta, dt)
        v_new, _, _, _ = pcg(A, b, 2.0 * V - V_prev, d, tol, tol, 10000)
        V_prev, V = V, v_new
    e = V - w3d(x, y, steps * dt, lx, ly)
    return float(np.sqrt(e @ (M @ e))), float(np.abs(e).max())
