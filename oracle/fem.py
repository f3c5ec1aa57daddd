"""P1 finite elements on tetrahedra (and triangles, for the paper's 2D check).

Oracle code (test infrastructure only).  Section 2.2 of the paper: the monodomain equation
(Eq. 1) is discretised with linear finite elements; M and K are the global mass and stiffness
matrices, sparse n x n, and A = chi*Cm*M + theta*dt*K (definitions following Eq. 3).
The element conductivity is built from the longitudinal and transverse conductivities and the
element fibre f (Section 2.1): sigma_e = sigma_t*I + (sigma_l - sigma_t) * f f^T.
"""
import numpy as np
import scipy.sparse as sp


def tet_geometry(xyz, tets):
    """Volumes and barycentric gradients of every tetrahedron.

    With J = [x1-x0, x2-x0, x3-x0] (columns), x = x0 + J xi and the barycentric coordinates are
    l1..l3 = xi, l0 = 1 - sum(xi).  Hence grad l1..l3 are the rows of inv(J) and
    grad l0 = -(sum of those rows).  Volume = |det J| / 6.
    Returns vol (E,), grads (E, 4, 3), detJ (E,).
    """
    X = xyz[tets]                                          # (E, 4, 3)
    J = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], axis=2)
    detJ = np.linalg.det(J)
    Jinv = np.linalg.inv(J)                                # rows = grad l1..l3
    g = np.empty((tets.shape[0], 4, 3))
    g[:, 1:, :] = Jinv
    g[:, 0, :] = -Jinv.sum(axis=1)
    return np.abs(detJ) / 6.0, g, detJ


def conductivity_tensors(fibres, sigma_l, sigma_t):
    """sigma_e = sigma_t I + (sigma_l - sigma_t) f f^T for each element (S/m).

    sigma_l, sigma_t may be scalars or per-element arrays."""
    f = fibres / np.linalg.norm(fibres, axis=1, keepdims=True)
    sl = np.broadcast_to(np.asarray(sigma_l, dtype=np.float64), (f.shape[0],))
    st = np.broadcast_to(np.asarray(sigma_t, dtype=np.float64), (f.shape[0],))
    eye = np.eye(3)[None, :, :]
    return st[:, None, None] * eye + (sl - st)[:, None, None] * np.einsum("ei,ej->eij", f, f)


def tet_element_matrices(xyz, tets, sigma):
    """Local 4x4 matrices of every tetrahedron.

    Mass:      M_e[i, j] = integral of l_i l_j = vol * (1 + delta_ij) / 20.
    Stiffness: K_e[i, j] = integral of grad l_i . sigma_e grad l_j = vol * g_i^T sigma_e g_j.
    """
    vol, g, _ = tet_geometry(xyz, tets)
    Me = vol[:, None, None] * (np.ones((4, 4)) + np.eye(4))[None] / 20.0
    Ke = vol[:, None, None] * np.einsum("eia,eab,ejb->eij", g, sigma, g)
    return Me, Ke


def tri_element_matrices(xy, tris):
    """P1 triangles with identity conductivity: M_e = area (1 + delta_ij)/12,
    K_e = area * grad l_i . grad l_j (used only by the 2D manufactured solution)."""
    X = xy[tris]
    J = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0]], axis=2)   # (E, 2, 2)
    area = np.abs(np.linalg.det(J)) / 2.0
    Jinv = np.linalg.inv(J)
    g = np.empty((tris.shape[0], 3, 2))
    g[:, 1:, :] = Jinv
    g[:, 0, :] = -Jinv.sum(axis=1)
    Me = area[:, None, None] * (np.ones((3, 3)) + np.eye(3))[None] / 12.0
    Ke = area[:, None, None] * np.einsum("eia,eja->eij", g, g)
    return Me, Ke


def assemble(elems, local, n):
    """Sum local matrices into a global CSR matrix: G[e_i, e_j] += local[e, i, j]."""
    k = elems.shape[1]
    rows = np.repeat(elems, k, axis=1).ravel()
    cols = np.tile(elems, (1, k)).ravel()
    G = sp.coo_matrix((local.ravel(), (rows, cols)), shape=(n, n)).tocsr()
    G.sum_duplicates()
    G.sort_indices()
    return G


def mass_stiffness(xyz, tets, fibres, sigma_l, sigma_t):
    """Global M and K (CSR, FP64) of a tetrahedral mesh."""
    sig = conductivity_tensors(fibres, sigma_l, sigma_t)
    Me, Ke = tet_element_matrices(xyz, tets, sig)
    n = xyz.shape[0]
    return assemble(tets, Me, n), assemble(tets, Ke, n)


def system_matrix(M, K, chi, cm, theta, dt):
    """A = chi*Cm*M + theta*dt*K, stored on the union pattern of M and K."""
    A = (chi * cm) * M + (theta * dt) * K
    A.sort_indices()
    return A


def monodomain_conductivity(il, it, el, et):
    """Monodomain conductivities from intra-/extracellular ones (Listing 1 sets regions up with
    il, it, el, et): per direction the series combination sigma_i sigma_e / (sigma_i + sigma_e)."""
    il, it, el, et = (np.asarray(v, dtype=np.float64) for v in (il, it, el, et))
    return 1.0 / (1.0 / il + 1.0 / el), 1.0 / (1.0 / it + 1.0 / et)
