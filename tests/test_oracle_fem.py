"""Pins of the oracle's P1 assembly (Section 2.2: linear finite elements, M and K).

Independent references: exact symbolic integration (sympy) of the P1 basis on rational
tetrahedra, the textbook stiffness of the unit right tetrahedron, a dense brute-force
assembly of two tetrahedra, and invariants that hold for any P1 mesh.
"""
import numpy as np
import pytest
import sympy as S

from oracle import fem
from paper_2510_12011_b300 import inputs as I


def _exact_local(P, sig):
    """Exact P1 mass and stiffness of the tetrahedron with rational vertices P (4x3) and
    conductivity matrix sig, by solving for the affine basis and integrating symbolically."""
    x, y, z = S.symbols("x y z")
    a = S.symbols("a0:4")
    phis = []
    for i in range(4):
        expr = a[0] + a[1] * x + a[2] * y + a[3] * z
        eqs = [expr.subs({x: P[j][0], y: P[j][1], z: P[j][2]}) - (1 if i == j else 0) for j in range(4)]
        sol = S.solve(eqs, a)
        phis.append(expr.subs(sol))
    u, v, w = S.symbols("u v w")
    P0 = S.Matrix(P[0])
    J = S.Matrix.hstack(*[S.Matrix(P[k]) - P0 for k in (1, 2, 3)])
    X = P0 + J * S.Matrix([u, v, w])
    detJ = abs(J.det())

    def integrate(f):
        g = f.subs({x: X[0], y: X[1], z: X[2]}, simultaneous=True)
        return detJ * S.integrate(g, (w, 0, 1 - u - v), (v, 0, 1 - u), (u, 0, 1))

    grads = [S.Matrix([S.diff(p, s) for s in (x, y, z)]) for p in phis]
    sigM = S.Matrix(sig)
    Mloc = [[integrate(phis[i] * phis[j]) for j in range(4)] for i in range(4)]
    vol = integrate(S.Integer(1))
    Kloc = [[vol * (grads[i].T * sigM * grads[j])[0, 0] for j in range(4)] for i in range(4)]
    return np.array(Mloc, dtype=float), np.array(Kloc, dtype=float)


def _sigma_rational(f, sl, st):
    f = [S.Rational(c) for c in f]
    return [[st * (1 if i == j else 0) + (sl - st) * f[i] * f[j] for j in range(3)] for i in range(3)]


TET = [[0, 0, 0], [S.Rational(3, 2), S.Rational(1, 5), 0], [S.Rational(1, 3), 1, S.Rational(1, 7)],
       [S.Rational(-1, 4), S.Rational(1, 2), S.Rational(6, 5)]]


def test_local_matrices_match_exact_integration():
    sl, st = S.Rational(17, 100), S.Rational(19, 1000)
    fr = [S.Rational(3, 5), S.Rational(4, 5), 0]
    Mx, Kx = _exact_local(TET, _sigma_rational(fr, sl, st))
    xyz = np.array(TET, dtype=float)
    sig = fem.conductivity_tensors(np.array([[0.6, 0.8, 0.0]]), 0.17, 0.019)
    Me, Ke = fem.tet_element_matrices(xyz, np.array([[0, 1, 2, 3]]), sig)
    assert np.allclose(Me[0], Mx, rtol=1e-13, atol=0)
    assert np.allclose(Ke[0], Kx, rtol=1e-12, atol=1e-15)


def test_negatively_oriented_tet_gives_same_matrices():
    xyz = np.array(TET, dtype=float)
    sig = fem.conductivity_tensors(np.array([[0.6, 0.8, 0.0]]), 0.17, 0.019)
    Me, Ke = fem.tet_element_matrices(xyz, np.array([[0, 1, 2, 3]]), sig)
    Me2, Ke2 = fem.tet_element_matrices(xyz, np.array([[1, 0, 2, 3]]), sig)
    p = [1, 0, 2, 3]
    assert np.allclose(Me2[0], Me[0][np.ix_(p, p)], rtol=1e-14)
    assert np.allclose(Ke2[0], Ke[0][np.ix_(p, p)], rtol=1e-13)


def test_unit_right_tet_textbook_stiffness():
    # Isotropic P1 stiffness of the tetrahedron (0,0,0),(1,0,0),(0,1,0),(0,0,1):
    # (1/6) [[3,-1,-1,-1],[-1,1,0,0],[-1,0,1,0],[-1,0,0,1]], mass (1/120)(1 + delta_ij).
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=float)
    sig = fem.conductivity_tensors(np.array([[1.0, 0.0, 0.0]]), 1.0, 1.0)
    Me, Ke = fem.tet_element_matrices(xyz, np.array([[0, 1, 2, 3]]), sig)
    Kt = np.array([[3, -1, -1, -1], [-1, 1, 0, 0], [-1, 0, 1, 0], [-1, 0, 0, 1]]) / 6.0
    assert np.allclose(Ke[0], Kt, atol=1e-15)
    assert np.allclose(Me[0], (np.ones((4, 4)) + np.eye(4)) / 120.0, atol=1e-17)


def test_two_element_brute_force_assembly():
    # two tetrahedra sharing the face (1, 2, 3); node 4 lies on the other side of it
    P = [TET[0], TET[1], TET[2], TET[3], [S.Rational(3, 2), S.Rational(3, 2), S.Rational(3, 2)]]
    tets = [[0, 1, 2, 3], [4, 1, 3, 2]]
    sl, st = S.Rational(17, 100), S.Rational(19, 1000)
    fr = [1, 0, 0]
    Md = np.zeros((5, 5))
    Kd = np.zeros((5, 5))
    for t in tets:
        Mx, Kx = _exact_local([P[v] for v in t], _sigma_rational(fr, sl, st))
        for a in range(4):
            for b in range(4):
                Md[t[a], t[b]] += Mx[a, b]
                Kd[t[a], t[b]] += Kx[a, b]
    xyz = np.array(P, dtype=float)
    M, K = fem.mass_stiffness(xyz, np.array(tets), np.array([[1.0, 0, 0]] * 2), 0.17, 0.019)
    assert np.allclose(M.toarray(), Md, rtol=1e-13, atol=0)
    assert np.allclose(K.toarray(), Kd, rtol=1e-12, atol=1e-15)
    assert M[0, 4] == 0.0 and K[0, 4] == 0.0


def test_conductivity_tensor_eigenpairs():
    rng = np.random.default_rng(0)
    f = rng.normal(size=(5, 3))
    sig = fem.conductivity_tensors(f, 0.17, 0.019)
    fu = f / np.linalg.norm(f, axis=1, keepdims=True)
    t = np.cross(fu, rng.normal(size=(5, 3)))
    for e in range(5):
        assert np.allclose(sig[e] @ fu[e], 0.17 * fu[e], atol=1e-15)
        assert np.allclose(sig[e] @ t[e], 0.019 * t[e], atol=1e-15)


@pytest.fixture(scope="module")
def jittered():
    m = I.slab_mesh(4.0, 2.0, 1.5, 0.25, jitter=0.15, seed=11, fibre="rotating")
    M, K = fem.mass_stiffness(m.xyz, m.tets, m.fibres, 0.17, 0.019)
    return m, M, K


def test_mass_total_is_volume(jittered):
    m, M, K = jittered
    assert abs(M.sum() - 4.0 * 2.0 * 1.5) < 1e-12


def test_mass_row_sums_are_patch_volumes(jittered):
    # integral of phi_i = sum over elements containing node i of vol_e / 4
    m, M, K = jittered
    vol, _, _ = fem.tet_geometry(m.xyz, m.tets)
    ref = np.zeros(m.n_nodes)
    np.add.at(ref, m.tets.ravel(), np.repeat(vol / 4.0, 4))
    assert np.allclose(np.asarray(M.sum(axis=1)).ravel(), ref, rtol=1e-13)


def test_stiffness_symmetric_zero_row_sums(jittered):
    m, M, K = jittered
    assert abs(K - K.T).max() < 1e-15 * abs(K).max()
    assert abs(M - M.T).max() < 1e-15 * abs(M).max()
    rs = np.asarray(K.sum(axis=1)).ravel()
    assert np.abs(rs).max() < 1e-14 * np.abs(K).max()


def test_patch_test_affine_field():
    # With a constant conductivity, K applied to an affine field vanishes on every interior
    # row (sigma grad u is constant and the integral of grad phi_i over its patch is 0).
    m = I.slab_mesh(4.0, 2.0, 1.5, 0.25, jitter=0.15, seed=12, fibre="x")
    M, K = fem.mass_stiffness(m.xyz, m.tets, m.fibres, 0.17, 0.019)
    u = 0.3 + 1.7 * m.xyz[:, 0] - 0.4 * m.xyz[:, 1] + 2.2 * m.xyz[:, 2]
    Ku = K @ u
    dims = np.array(m.shape)
    interior = np.all((m.lattice > 0) & (m.lattice < dims - 1), axis=1)
    assert np.abs(Ku[interior]).max() < 1e-13 * np.abs(K).max() * np.abs(u).max()
    assert np.abs(Ku[~interior]).max() > 1e-6


def test_system_matrix_spd_and_pattern():
    w = I.slab_small_ms()
    m = w.mesh
    M, K = fem.mass_stiffness(m.xyz, m.tets, m.fibres, w.sigma_l, w.sigma_t)
    A = fem.system_matrix(M, K, w.chi, w.cm, w.theta, w.dt)
    assert A.nnz == 11601 and M.nnz == 11601 and K.nnz == 11601
    Ad = A.toarray()
    np.linalg.cholesky(Ad)
    ref = w.chi * w.cm * M.toarray() + w.theta * w.dt * K.toarray()
    assert np.allclose(Ad, ref, rtol=1e-15, atol=0)
