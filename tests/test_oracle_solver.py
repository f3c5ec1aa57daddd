"""Pins of the oracle's PCG (Algorithm 1) and theta-scheme (Eq. 2, Table 2)."""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import fem
from oracle.monodomain import rhs
from oracle.pcg import pcg
from paper_2510_12011_b300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def small():
    w = I.slab_small_ms()
    m = w.mesh
    M, K = fem.mass_stiffness(m.xyz, m.tets, m.fibres, w.sigma_l, w.sigma_t)
    return w, M, K


def test_pcg_matches_dense_solve(small):
    w, M, K = small
    A = fem.system_matrix(M, K, w.chi, w.cm, w.theta, w.dt)
    b = I.random_vector(A.shape[0], 5)
    x, it, zn, ok = pcg(A, b, np.zeros_like(b), A.diagonal(), 0.0, 1e-14, 1000)
    xd = np.linalg.solve(A.toarray(), b)
    assert ok and 0 < it < 200
    assert np.abs(x - xd).max() < 1e-10 * np.abs(xd).max()


def test_pcg_residual_below_tolerance(small):
    w, M, K = small
    A = fem.system_matrix(M, K, w.chi, w.cm, w.theta, w.dt)
    d = A.diagonal()
    b = I.random_vector(A.shape[0], 6)
    x0 = I.random_vector(A.shape[0], 7)
    for rtol in (1e-4, 1e-8):
        x, it, zn, ok = pcg(A, b, x0, d, 0.0, rtol, 1000)
        z0 = np.linalg.norm((b - A @ x0) / d)
        # the recursively updated residual passed the test; the true one agrees to rounding
        assert zn / z0 < rtol
        assert np.linalg.norm((b - A @ x) / d) / z0 < 1.01 * rtol + 1e-13


def test_pcg_jacobi_on_diagonal_matrix_is_one_step():
    # Jacobi preconditioning of a diagonal SPD matrix is exact: one iteration solves it.
    dgl = np.linspace(1.0, 50.0, 40)
    A = sp.diags(dgl).tocsr()
    b = I.random_vector(40, 8)
    x, it, zn, ok = pcg(A, b, np.zeros(40), dgl, 0.0, 1e-12, 10)
    assert it == 1 and ok
    assert np.allclose(x, b / dgl, rtol=1e-15)


def test_pcg_zero_residual_and_max_iter(small):
    w, M, K = small
    A = fem.system_matrix(M, K, w.chi, w.cm, w.theta, w.dt)
    d = A.diagonal()
    x_exact = I.random_vector(A.shape[0], 9)
    b = A @ x_exact
    x, it, zn, ok = pcg(A, b, x_exact, d, 0.0, 1e-10, 100)
    # b - A x0 is zero up to rounding; when it is exactly zero no iteration is made
    x, it, zn, ok = pcg(A, np.zeros(A.shape[0]), np.zeros(A.shape[0]), d, 0.0, 1e-10, 100)
    assert it == 0 and ok and zn == 0.0
    x, it, zn, ok = pcg(A, I.random_vector(A.shape[0], 10), np.zeros(A.shape[0]), d, 0.0, 1e-14, 1)
    assert it == 1 and not ok
    x, it, zn, ok = pcg(A, I.random_vector(A.shape[0], 10), np.zeros(A.shape[0]), d, 1e30, 0.0, 5)
    assert it == 0 and ok


def test_pcg_cg_terminates_in_distinct_eigenvalue_count():
    # Preconditioned CG in exact arithmetic stops after as many steps as D^-1 A has distinct
    # eigenvalues.  With u_i = +-1, B = I + c u u^T has unit-plus-c diagonal and two distinct
    # eigenvalues, and so has D^-1 A for A = Dh B Dh.
    n = 30
    rng = np.random.default_rng(1)
    dg = rng.uniform(1.0, 3.0, n)
    u = rng.choice([-1.0, 1.0], size=n)
    B = np.eye(n) + 0.7 * np.outer(u, u)
    Dh = np.diag(np.sqrt(dg))
    A = sp.csr_matrix(Dh @ B @ Dh)
    b = rng.normal(size=n)
    x, it, zn, ok = pcg(A, b, np.zeros(n), A.diagonal(), 0.0, 1e-12, 50)
    assert it == 2 and ok


def _mode(M, K, chi, cm, j):
    lam, vec = sla.eigh(K.toarray(), chi * cm * M.toarray())
    return lam[j], vec[:, j]


@pytest.mark.parametrize("theta", [0.0, 0.5, 2.0 / 3.0, 1.0])
def test_theta_scheme_amplification_factor(small, theta):
    # For K v = lam chi Cm M v and no ionic current, one step of Eq. 2 maps V = v to g v with
    # g = (1 - (1 - theta) dt lam) / (1 + theta dt lam).
    w, M, K = small
    dt = 0.05
    A = fem.system_matrix(M, K, w.chi, w.cm, theta, dt)
    for j in (1, 7, 200):
        lam, v = _mode(M, K, w.chi, w.cm, j)
        b = rhs(M, K, v, np.zeros_like(v), np.zeros_like(v), w.chi, w.cm, theta, dt)
        x, it, _, ok = pcg(A, b, v, A.diagonal(), 0.0, 1e-13, 1000)
        g = (1.0 - (1.0 - theta) * dt * lam) / (1.0 + theta * dt * lam)
        assert ok
        assert np.abs(x - g * v).max() < 1e-9 * np.abs(v).max()


def test_table2_stability_claims(small):
    # Table 2: theta = 0 is conditionally stable, theta >= 1/2 unconditionally stable.
    w, M, K = small
    ref = json.load(open(os.path.join(GOLDEN, "theta_schemes.json")))
    lam_max = _mode(M, K, w.chi, w.cm, -1)[0]
    for s in ref["schemes"]:
        th = s["theta"]
        for dt in (1e-3, 1.0, 1e3):
            g = (1.0 - (1.0 - th) * dt * lam_max) / (1.0 + th * dt * lam_max)
            if s["stability"] == "unconditionally stable":
                assert abs(g) <= 1.0
            elif dt * lam_max > 2.0:
                assert abs(g) > 1.0
