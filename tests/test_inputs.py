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
