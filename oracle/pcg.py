"""Jacobi-preconditioned conjugate gradients, Algorithm 1 of the paper (Section 2.2).

Oracle code (test infrastructure only).  Readings of the algorithm as printed:
  * the preconditioner M is diag(A) (Jacobi, Section 2.2), so "solve M z = r" is z = r / diag(A);
  * the break test uses z_{k+1}, so z_{k+1} is computed before the test (the printed listing
    tests it before solving for it);
  * the relative test compares ||z_{k+1}||_2 with ||z_0||_2, the norm computed once before the
    loop; the absolute test compares ||z_{k+1}||_2 with eps_a;
  * if z_0 = 0 or ||z_0|| < eps_a, x_0 is returned after zero iterations (the printed loop
    would divide by p^T q = 0 in that case).
Returns the solution, the number of A-products made in the loop, the final ||z|| and whether
a tolerance was met.
"""
import numpy as np


def pcg(A, b, x0, diag, atol, rtol, max_iter):
    x = x0.copy()
    r = b - A @ x
    z = r / diag
    p = z.copy()
    rho = r @ z
    z0_norm = np.sqrt(z @ z)
    if z0_norm == 0.0 or z0_norm < atol:
        return x, 0, z0_norm, True
    z_norm = z0_norm
    for k in range(max_iter):
        q = A @ p
        alpha = rho / (p @ q)
        x = x + alpha * p
        r = r - alpha * q
        z = r / diag
        z_norm = np.sqrt(z @ z)
        if z_norm < atol or z_norm / z0_norm < rtol:
            return x, k + 1, z_norm, True
        rho_next = r @ z
        beta = rho_next / rho
        p = z + beta * p
        rho = rho_next
    return x, max_iter, z_norm, False
