"""Seeded input generator: sizes, orientation, jitter rule, SplitMix64 reference outputs."""
import numpy as np

from paper_2510_12011_b300 import inputs as I


def test_splitmix64_reference_outputs():
    # SplitMix64 seeded with 0: the first three outputs of the published generator.
    out = I.splitmix64(0, np.arange(3, dtype=np.uint64))
    assert [int(x) for x in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_small_slab_sizes():
    w = I.slab_small_ms()
    m = w.mesh
    assert m.shape == (21, 9, 5)
    assert m.n_nodes == 945 and m.n_tets == 3840
    assert len(w.stimuli[0].nodes) == 27
    assert w.n_steps == 5000


def _volumes(m):
    X = m.xyz[m.tets]
    J = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], axis=2)
    return np.linalg.det(J) / 6.0


def test_positive_orientation_and_total_volume():
    m = I.slab_mesh(4.0, 2.0, 1.0, 0.25, jitter=0.15, seed=7)
    vol = _volumes(m)
    assert vol.min() > 0.0
    assert abs(vol.sum() - 8.0) < 1e-12


def test_jitter_bounds_and_faces():
    m = I.slab_mesh(4.0, 2.0, 1.0, 0.25, jitter=0.15, seed=3)
    d = m.xyz - m.lattice * 0.25
    assert np.abs(d).max() <= 0.15 * 0.25 + 1e-15
    assert np.abs(d).max() > 0.1 * 0.25
    dims = np.array(m.shape)
    on_face = (m.lattice == 0) | (m.lattice == dims - 1)
    assert np.all(d[on_face] == 0.0)
    assert np.all(d[~on_face] != 0.0)


def test_large_slab_shape_only():
    # lattice sizes of the 40x16x6 mm slab at h = 0.2 mm (no mesh is built here)
    nx, ny, nz = (int(round(L / 0.2)) + 1 for L in (40.0, 16.0, 6.0))
    assert (nx, ny, nz) == (201, 81, 31)
    assert nx * ny * nz == 504711
    assert 6 * (nx - 1) * (ny - 1) * (nz - 1) == 2_880_000


def test_rotating_fibres():
    m = I.slab_mesh(2.0, 1.0, 6.0, 0.5, fibre="rotating")
    f = m.fibres
    assert np.allclose(np.linalg.norm(f, axis=1), 1.0)
    assert np.all(f[:, 2] == 0.0)
    zc = m.xyz[m.tets, 2].mean(axis=1)
    ang = np.rad2deg(np.arctan2(f[:, 1], f[:, 0]))
    assert np.allclose(ang, -60.0 + 20.0 * zc)


def test_prolate_shell_volume_conformity_and_fibres():
    """Coarse (h = 1 mm) truncated ellipsoid shell: voxel volume within 3 % of the analytic
    difference of the two ellipsoid caps below z = -30 mm, a conforming mesh (every face shared by
    at most two tetrahedra), unit fibres tangent to the ellipsoid family that turn from about
    -60 deg at the endocardium to +60 deg at the epicardium, stimulus sites on the apical/septal
    endocardium."""
    import numpy as np
    from paper_2510_12011_b300 import inputs as I

    h = 1.0
    m = I.prolate_shell_mesh(h)
    # analytic volume: cap of x^2/a^2 + y^2/a^2 + z^2/c^2 <= 1 from the apex (z = -c) to z_c
    def cap(a, c, zc):
        return np.pi * a * a * ((zc + c) - (zc ** 3 + c ** 3) / (3 * c * c))
    exact = cap(45.0, 80.0, -30.0) - cap(35.0, 70.0, -30.0)
    p = m.xyz[m.tets]
    vol = np.abs(np.einsum("ij,ij->i", p[:, 1] - p[:, 0], np.cross(p[:, 2] - p[:, 0], p[:, 3] - p[:, 0]))).sum() / 6
    assert abs(vol - exact) < 0.03 * exact, (vol, exact)
    faces = np.sort(np.concatenate([m.tets[:, [0, 1, 2]], m.tets[:, [0, 1, 3]], m.tets[:, [0, 2, 3]],
                                    m.tets[:, [1, 2, 3]]]), axis=1)
    _, counts = np.unique(faces, axis=0, return_counts=True)
    assert counts.max() == 2
    f = m.fibres
    assert np.allclose(np.linalg.norm(f, axis=1), 1.0)
    c = p.mean(axis=1)
    a_s, c_s = 35.0 + 10.0 * m.depth, 70.0 + 10.0 * m.depth
    n = np.stack([c[:, 0] / a_s ** 2, c[:, 1] / a_s ** 2, c[:, 2] / c_s ** 2], axis=1)
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    assert np.abs(np.einsum("ij,ij->i", f, n)).max() < 0.2      # tangent (tet vs cell centre)
    r = np.hypot(c[:, 0], c[:, 1])
    ec = np.stack([-c[:, 1], c[:, 0], np.zeros_like(r)], axis=1) / r[:, None]
    ang = np.degrees(np.arcsin(np.clip(np.einsum("ij,ij->i", f, np.cross(n, ec)), -1, 1)))
    assert abs(np.median(ang[m.depth < 0.1]) + 57.0) < 6.0
    assert abs(np.median(ang[m.depth > 0.9]) - 57.0) < 6.0
    sites = I.endocardial_sites(m, 5, 5)
    assert len(sites) == 5
    for s in sites:
        x = m.xyz[s]
        assert s.size > 0 and x[:, 2].max() <= -45.0 + 1.5 + 1e-9 and x[:, 0].max() <= 1.5 + 1e-9
        fe = (x[:, 0] ** 2 + x[:, 1] ** 2) / 35.0 ** 2 + x[:, 2] ** 2 / 70.0 ** 2
        assert fe.min() <= (1.0 + 2.5 / 35.0) ** 2
