"""Seeded synthetic inputs for the monodomain hot path.

This module generates *inputs only*: node coordinates, tetrahedral connectivity, per-element
fibre directions, region ids, stimulus node sets and the parameter sets of the workloads.
It holds none of the method's arithmetic (no element matrices, no assembly, no solver, no
ionic model), so both the CUDA path and the FP64 oracle may draw their inputs from it.

Meshes are structured cuboid slabs split into tetrahedra, the geometry the paper uses for
its idealised cube meshes and its N-version benchmark (Section 3.1.2, Table 3; Section 3.3).
Every hexahedral cell is cut into six tetrahedra along its (0,0,0)-(1,1,1) diagonal (the
Kuhn/Freudenthal split: one tetrahedron per ordering of the three axes), which gives a
conforming mesh.  Optional node jitter uses SplitMix64 (Steele, Lea & Flood 2014) as a
counter-based generator: draw number c of seed s is mix(s + (c+1) * 0x9E3779B97F4A7C15).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, counters: np.ndarray) -> np.ndarray:
    """Counter-based SplitMix64: output number ``counters`` of the stream seeded ``seed``."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (counters.astype(np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, counters: np.ndarray) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of SplitMix64 outputs."""
    return (splitmix64(seed, counters) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


# The six tetrahedra of one hex cell, as corner offsets (dx, dy, dz).  Axis ordering
# (a, b, c) walks (0,0,0) -> e_a -> e_a+e_b -> (1,1,1); odd orderings swap the last two
# vertices so that every tetrahedron is positively oriented.
def _kuhn_corners():
    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    even = {(0, 1, 2), (1, 2, 0), (2, 0, 1)}
    out = []
    for p in perms:
        v = [np.zeros(3, dtype=int)]
        for ax in p:
            nxt = v[-1].copy()
            nxt[ax] = 1
            v.append(nxt)
        if p not in even:
            v[2], v[3] = v[3], v[2]
        out.append([tuple(int(c) for c in x) for x in v])
    return out


KUHN_CORNERS = _kuhn_corners()


@dataclass
class Mesh:
    """A tetrahedral mesh: coordinates in mm, 0-based connectivity, unit fibres per element."""
    xyz: np.ndarray          # (n, 3) float64, mm
    tets: np.ndarray         # (n_tets, 4) int32
    fibres: np.ndarray       # (n_tets, 3) float64, unit
    region: np.ndarray       # (n_tets,) int32
    lattice: np.ndarray      # (n, 3) int32 lattice indices (i, j, k) of each node
    shape: tuple             # (nx, ny, nz) nodes per axis
    h: float

    @property
    def n_nodes(self) -> int:
        return self.xyz.shape[0]

    @property
    def n_tets(self) -> int:
        return self.tets.shape[0]


def slab_mesh(lx: float, ly: float, lz: float, h: float, jitter: float = 0.0, seed: int = 0,
              fibre: str = "x") -> Mesh:
    """Cuboid [0,lx]x[0,ly]x[0,lz] (mm) with node spacing h, six tetrahedra per cell.

    jitter: each node coordinate moves by U(-jitter*h, +jitter*h) drawn from SplitMix64 with
    counter 3*node+axis; a coordinate that lies on a face of the box normal to that axis is
    not moved, so the box stays a box.  With jitter <= 0.15 every tetrahedron keeps a positive
    volume (its smallest height, h/sqrt(2), shrinks by at most 0.3*sqrt(2)*h).
    fibre: "x" for (1,0,0) everywhere; "rotating" for f = (cos a, sin a, 0) with the angle a
    going linearly from -60 deg at z=0 to +60 deg at z=lz, taken at the element centroid.
    """
    nx = int(round(lx / h)) + 1
    ny = int(round(ly / h)) + 1
    nz = int(round(lz / h)) + 1
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    lat = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1).astype(np.int32)
    xyz = lat.astype(np.float64) * h
    n = lat.shape[0]
    if jitter > 0.0:
        c = np.arange(3 * n, dtype=np.uint64).reshape(n, 3)
        d = (2.0 * uniform01(seed, c) - 1.0) * (jitter * h)
        dims = np.array([nx, ny, nz])
        on_face = (lat == 0) | (lat == dims - 1)
        d[on_face] = 0.0
        xyz = xyz + d

    def nid(ii, jj, kk):
        return ii + nx * (jj + ny * kk)

    ci, cj, ck = np.meshgrid(np.arange(nx - 1), np.arange(ny - 1), np.arange(nz - 1), indexing="ij")
    # cell order: i fastest, then j, then k
    ci = ci.transpose(2, 1, 0).ravel()
    cj = cj.transpose(2, 1, 0).ravel()
    ck = ck.transpose(2, 1, 0).ravel()
    tets = np.empty((ci.size, 6, 4), dtype=np.int64)
    for t, corners in enumerate(KUHN_CORNERS):
        for v, (dx, dy, dz) in enumerate(corners):
            tets[:, t, v] = nid(ci + dx, cj + dy, ck + dz)
    tets = tets.reshape(-1, 4).astype(np.int32)

    if fibre == "x":
        fib = np.zeros((tets.shape[0], 3))
        fib[:, 0] = 1.0
    elif fibre == "rotating":
        zc = xyz[tets, 2].mean(axis=1)
        a = np.deg2rad(-60.0 + 120.0 * zc / lz)
        fib = np.stack([np.cos(a), np.sin(a), np.zeros_like(a)], axis=1)
    else:
        raise ValueError(f"unknown fibre rule {fibre!r}")
    region = np.zeros(tets.shape[0], dtype=np.int32)
    return Mesh(xyz=xyz, tets=tets, fibres=fib, region=region, lattice=lat,
                shape=(nx, ny, nz), h=h)


def corner_nodes(mesh: Mesh, size_mm: float) -> np.ndarray:
    """Nodes whose unjittered lattice position lies in the corner cube [0, size_mm]^3."""
    lim = size_mm / mesh.h + 1e-9
    sel = np.all(mesh.lattice.astype(np.float64) <= lim, axis=1)
    return np.nonzero(sel)[0].astype(np.int32)


@dataclass
class MSParams:
    """Mitchell-Schaeffer two-variable model, mapped to mV (v = (V - v_min)/(v_max - v_min))."""
    tau_in: float = 0.3
    tau_out: float = 6.0
    tau_open: float = 120.0
    tau_close: float = 150.0
    v_gate: float = 0.13
    v_min: float = -80.0
    v_max: float = 20.0

    def as_array(self) -> np.ndarray:
        return np.array([self.tau_in, self.tau_out, self.tau_open, self.tau_close,
                         self.v_gate, self.v_min, self.v_max], dtype=np.float64)


@dataclass
class Stimulus:
    nodes: np.ndarray
    start: float        # ms
    duration: float     # ms
    intensity: float    # uA/mm^2


@dataclass
class Workload:
    """One monodomain run: mesh, tissue constants, time stepping, solver and stimuli."""
    name: str
    mesh: Mesh
    sigma_l: object           # S/m, a scalar or one value per region
    sigma_t: object           # S/m, a scalar or one value per region
    chi: float                # 1/mm
    cm: float                 # uF/mm^2
    theta: float
    dt: float                 # ms
    t_end: float              # ms
    model: str                # "ms" or "tp06"
    ms: MSParams = field(default_factory=MSParams)
    stimuli: list = field(default_factory=list)
    atol: float = 0.0
    rtol: float = 1e-10
    max_iter: int = 1000
    v_threshold: float = 0.0  # mV, activation threshold
    tp06_cell: int = 2        # ten Tusscher-Panfilov cell type: 0 endo, 1 mid, 2 epi

    @property
    def n_steps(self) -> int:
        return int(round(self.t_end / self.dt))


def slab_small_ms() -> Workload:
    """10x4x2 mm slab at h=0.5 mm (945 nodes, 3840 tets), fibres along x, Mitchell-Schaeffer,
    dt=0.01 ms for 50 ms, 2 ms corner stimulus at 50 uA/cm^2 = 0.5 uA/mm^2, PCG rel tol 1e-10."""
    m = slab_mesh(10.0, 4.0, 2.0, 0.5)
    st = [Stimulus(corner_nodes(m, 1.0), 0.0, 2.0, 0.5)]
    # chi = 1400 /cm = 140 /mm; Cm = 1 uF/cm^2 = 0.01 uF/mm^2
    return Workload("slab10x4x2_h0.5_ms", m, 0.17, 0.019, 140.0, 0.01, 0.5, 0.01, 50.0, "ms",
                    stimuli=st, atol=0.0, rtol=1e-10, max_iter=1000)


def slab_large(model: str = "ms") -> Workload:
    """40x16x6 mm slab at h=0.2 mm (504,711 nodes, 2,880,000 tets), jitter U(+-0.15h) seed 1,
    fibres rotating -60..+60 deg through the depth, dt=0.02 ms for 100 ms, 1 mm corner stimulus
    (2 ms at 0.5 uA/mm^2).  Solver tolerances are the paper's recommended a_tol = r_tol = 1e-5
    with at most 100 iterations (Section 3.2, Listing 1)."""
    m = slab_mesh(40.0, 16.0, 6.0, 0.2, jitter=0.15, seed=1, fibre="rotating")
    st = [Stimulus(corner_nodes(m, 1.0), 0.0, 2.0, 0.5)]
    return Workload(f"slab40x16x6_h0.2_{model}", m, 0.17, 0.019, 140.0, 0.01, 0.5, 0.02, 100.0,
                    model, stimuli=st, atol=1e-5, rtol=1e-5, max_iter=100)


def slab_custom(lx, ly, lz, h, jitter=0.0, seed=0, fibre="x", dt=0.01, model="ms",
                stim_mm=1.0, rtol=1e-10, atol=0.0, max_iter=1000, t_end=10.0) -> Workload:
    """A slab workload of any size with the small-slab tissue constants (used for sweeps)."""
    m = slab_mesh(lx, ly, lz, h, jitter=jitter, seed=seed, fibre=fibre)
    st = [Stimulus(corner_nodes(m, stim_mm), 0.0, 2.0, 0.5)]
    return Workload(f"slab{lx:g}x{ly:g}x{lz:g}_h{h:g}_{model}", m, 0.17, 0.019, 140.0, 0.01, 0.5,
                    dt, t_end, model, stimuli=st, atol=atol, rtol=rtol, max_iter=max_iter)


@dataclass
class Batch:
    """Several independent slab workloads joined into one mesh of disconnected components.

    Region r of the joined mesh is instance r (its conductivities sit at index r of the
    workload's sigma arrays); node_offset[r] is the first node of instance r."""
    workload: Workload
    instances: list
    node_offset: np.ndarray


def join_workloads(parts, name="batch", gap_mm=1.0) -> Batch:
    """Join workloads that share dt, chi, Cm, theta, model and solver settings into one mesh
    (instances placed side by side along x with a gap, so they share no node)."""
    xyz, tets, fib, reg, lat, stims, offs = [], [], [], [], [], [], []
    off, x0 = 0, 0.0
    for r, w in enumerate(parts):
        m = w.mesh
        p = m.xyz.copy()
        p[:, 0] += x0
        x0 = p[:, 0].max() + gap_mm
        xyz.append(p)
        tets.append(m.tets + off)
        fib.append(m.fibres)
        reg.append(np.full(m.n_tets, r, dtype=np.int32))
        lat.append(m.lattice)
        for st in w.stimuli:
            stims.append(Stimulus(np.asarray(st.nodes, dtype=np.int32) + off, st.start, st.duration,
                                  st.intensity))
        offs.append(off)
        off += m.n_nodes
    w0 = parts[0]
    mesh = Mesh(np.concatenate(xyz), np.concatenate(tets).astype(np.int32), np.concatenate(fib),
                np.concatenate(reg), np.concatenate(lat), (0, 0, 0), w0.mesh.h)
    sl = np.array([float(np.atleast_1d(w.sigma_l)[0]) for w in parts])
    st_ = np.array([float(np.atleast_1d(w.sigma_t)[0]) for w in parts])
    w = Workload(name, mesh, sl, st_, w0.chi, w0.cm, w0.theta, w0.dt, w0.t_end, w0.model,
                 ms=w0.ms, stimuli=stims, atol=w0.atol, rtol=w0.rtol, max_iter=w0.max_iter,
                 v_threshold=w0.v_threshold, tp06_cell=w0.tp06_cell)
    return Batch(w, list(parts), np.array(offs, dtype=np.int64))


def batched_slabs(count: int = 64, seed: int = 4, h: float = 0.25, t_end: float = 200.0) -> Batch:
    """Batch of `count` uneven slabs: dims U(10,40) x U(5,16) x U(2,6) mm (rounded to h),
    conductivities log-uniform in 0.5x..2x of the small slab's, fibres along x, Mitchell-
    Schaeffer, dt = 0.01 ms, one 1 mm stimulus around a random boundary node per slab."""
    u = uniform01(seed, np.arange(8 * count, dtype=np.uint64)).reshape(count, 8)
    parts = []
    for i in range(count):
        lx = max(h, round((10.0 + 30.0 * u[i, 0]) / h) * h)
        ly = max(h, round((5.0 + 11.0 * u[i, 1]) / h) * h)
        lz = max(h, round((2.0 + 4.0 * u[i, 2]) / h) * h)
        m = slab_mesh(lx, ly, lz, h)
        dims = np.array(m.shape)
        on_face = np.any((m.lattice == 0) | (m.lattice == dims - 1), axis=1)
        bnodes = np.nonzero(on_face)[0]
        site = bnodes[int(u[i, 3] * bnodes.size) % bnodes.size]
        d = np.abs(m.lattice - m.lattice[site]).max(axis=1) * h
        nodes = np.nonzero(d <= 1.0 + 1e-9)[0].astype(np.int32)
        sl = 0.17 * np.exp(np.log(0.5) + np.log(4.0) * u[i, 4])
        st = 0.019 * np.exp(np.log(0.5) + np.log(4.0) * u[i, 5])
        parts.append(Workload(f"slab{i}", m, sl, st, 140.0, 0.01, 0.5, 0.01, t_end, "ms",
                              stimuli=[Stimulus(nodes, 0.0, 2.0, 0.5)], atol=1e-5, rtol=1e-5,
                              max_iter=100))
    return join_workloads(parts, name=f"batch{count}_slabs_h{h:g}_ms")


def _site_nodes(m: Mesh, site: int, radius_mm: float) -> np.ndarray:
    """Nodes within radius_mm (max-norm on the unjittered lattice) of node `site`."""
    d = np.abs(m.lattice - m.lattice[site]).max(axis=1) * m.h
    return np.nonzero(d <= radius_mm + 1e-9)[0].astype(np.int32)


def _boundary_site(m: Mesh, u: float) -> int:
    dims = np.array(m.shape)
    on_face = np.any((m.lattice == 0) | (m.lattice == dims - 1), axis=1)
    b = np.nonzero(on_face)[0]
    return int(b[int(u * b.size) % b.size])


def surrogate_training_slabs(count: int = 4, seed: int = 21, h: float = 0.25,
                             t_end: float = 600.0) -> list:
    """TP06 (epicardial) slabs that supply the learned surrogate's training pairs.

    Each is 16x8x3 mm at spacing h with jitter U(+-0.15h) (seed + slab index) and fibres
    rotating -60..+60 deg through the depth; both conductivities are scaled by U(0.7, 1.3); an
    S1 (2 ms at 0.5 uA/mm^2) around a seeded boundary site at t = 0 and an S2 (2 ms at
    1.0 uA/mm^2) around another seeded site at U(320, 420) ms, whose premature beat (or block)
    widens the range of states.  dt = 0.02 ms; solver tolerances as in the large slab."""
    u = uniform01(seed, np.arange(6 * count, dtype=np.uint64)).reshape(count, 6)
    out = []
    for i in range(count):
        m = slab_mesh(16.0, 8.0, 3.0, h, jitter=0.15, seed=seed + i, fibre="rotating")
        g = 0.7 + 0.6 * u[i, 0]
        s1 = _site_nodes(m, _boundary_site(m, u[i, 1]), 1.0)
        s2 = _site_nodes(m, _boundary_site(m, u[i, 2]), 1.0)
        t2 = 320.0 + 100.0 * u[i, 3]
        out.append(Workload(f"tp06_train{i}", m, 0.17 * g, 0.019 * g, 140.0, 0.01, 0.5, 0.02, t_end,
                            "tp06", stimuli=[Stimulus(s1, 0.0, 2.0, 0.5), Stimulus(s2, t2, 2.0, 1.0)],
                            atol=1e-5, rtol=1e-5, max_iter=100))
    return out


def surrogate_test_slab(h: float = 0.25, t_end: float = 400.0) -> Workload:
    """A TP06 slab the surrogate never saw: 20x8x3 mm at spacing h, jitter U(+-0.15h) seed 9,
    rotating fibres, nominal conductivities, 1 mm corner S1 (2 ms at 0.5 uA/mm^2), dt = 0.02 ms."""
    m = slab_mesh(20.0, 8.0, 3.0, h, jitter=0.15, seed=9, fibre="rotating")
    return Workload(f"tp06_slab20x8x3_h{h:g}", m, 0.17, 0.019, 140.0, 0.01, 0.5, 0.02, t_end, "tp06",
                    stimuli=[Stimulus(corner_nodes(m, 1.0), 0.0, 2.0, 0.5)], atol=1e-5, rtol=1e-5,
                    max_iter=100)


def prolate_shell_mesh(h: float = 0.35, endo=(35.0, 70.0), wall: float = 10.0, z_cut: float = -30.0) -> Mesh:
    """Truncated prolate-ellipsoid shell (an idealised left ventricle), apex down.

    The endocardium is the ellipsoid x^2/a0^2 + y^2/a0^2 + z^2/c0^2 = 1 (a0, c0 = endo), the
    epicardium the one with semi-axes a0 + wall, c0 + wall; the shell is cut by the plane z = z_cut.
    Lattice cells of spacing h (origin at (-a1, -a1, -c1)) whose centres lie in the shell are kept
    and split into six tetrahedra like the slabs (a voxel mesh: the surfaces are staircases).
    Every element's transmural depth s in [0, 1] solves x^2/(a0 + s w)^2 + y^2/(a0 + s w)^2 +
    z^2/(c0 + s w)^2 = 1 at its cell centre (bisection); the fibre turns from -60 deg at the
    endocardium to +60 deg at the epicardium, f = cos(a) e_c + sin(a) e_l, with e_c the
    circumferential direction and e_l = n x e_c (n the normal of the ellipsoid through the centre).
    Region 0 throughout; `lattice` holds the integer cell coordinates of every node."""
    a0, c0 = endo
    a1, c1 = a0 + wall, c0 + wall
    nx = int(np.ceil(2 * a1 / h))
    nz = int(np.ceil((z_cut + c1) / h))
    cells = []
    for k in range(nz):
        zc = -c1 + (k + 0.5) * h
        j, i = np.meshgrid(np.arange(nx), np.arange(nx), indexing="ij")
        xc = -a1 + (i + 0.5) * h
        yc = -a1 + (j + 0.5) * h
        r2 = xc * xc + yc * yc
        inside = (r2 / a1 ** 2 + zc * zc / c1 ** 2 <= 1.0) & (r2 / a0 ** 2 + zc * zc / c0 ** 2 >= 1.0) & (zc <= z_cut)
        ii, jj = i[inside], j[inside]
        cells.append(np.stack([ii, jj, np.full(ii.size, k)], axis=1))
    cells = np.concatenate(cells).astype(np.int64)
    stride = np.array([1, nx + 1, (nx + 1) * (nx + 1)], dtype=np.int64)
    corner_ids = np.empty((cells.shape[0], 6, 4), dtype=np.int64)
    for t, corners in enumerate(KUHN_CORNERS):
        for v, d in enumerate(corners):
            corner_ids[:, t, v] = (cells + np.array(d)) @ stride
    used, tets = np.unique(corner_ids.reshape(-1), return_inverse=True)
    tets = tets.reshape(-1, 4).astype(np.int32)
    lat = np.stack([used % (nx + 1), (used // (nx + 1)) % (nx + 1), used // ((nx + 1) * (nx + 1))], axis=1)
    xyz = np.stack([-a1 + lat[:, 0] * h, -a1 + lat[:, 1] * h, -c1 + lat[:, 2] * h], axis=1)
    # transmural depth and fibre per cell (shared by its six tetrahedra)
    cc = np.stack([-a1 + (cells[:, 0] + 0.5) * h, -a1 + (cells[:, 1] + 0.5) * h, -c1 + (cells[:, 2] + 0.5) * h], axis=1)
    rr = cc[:, 0] ** 2 + cc[:, 1] ** 2
    lo, hi = np.zeros(len(cc)), np.ones(len(cc))
    for _ in range(40):
        mid = 0.5 * (lo + hi)
        f = rr / (a0 + wall * mid) ** 2 + cc[:, 2] ** 2 / (c0 + wall * mid) ** 2 - 1.0
        lo = np.where(f > 0.0, mid, lo)
        hi = np.where(f > 0.0, hi, mid)
    depth = 0.5 * (lo + hi)
    a_s, c_s = a0 + wall * depth, c0 + wall * depth
    nrm = np.stack([cc[:, 0] / a_s ** 2, cc[:, 1] / a_s ** 2, cc[:, 2] / c_s ** 2], axis=1)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    r = np.sqrt(rr)
    ec = np.where(r[:, None] > 1e-9, np.stack([-cc[:, 1], cc[:, 0], np.zeros_like(r)], axis=1) / np.maximum(r, 1e-9)[:, None],
                  np.array([1.0, 0.0, 0.0]))
    el = np.cross(nrm, ec)
    el /= np.linalg.norm(el, axis=1, keepdims=True)
    ang = np.deg2rad(-60.0 + 120.0 * depth)
    fib_cell = np.cos(ang)[:, None] * ec + np.sin(ang)[:, None] * el
    fib = np.repeat(fib_cell, 6, axis=0)
    region = np.zeros(tets.shape[0], dtype=np.int32)
    m = Mesh(xyz=xyz, tets=tets, fibres=fib, region=region, lattice=lat.astype(np.int32), shape=(nx + 1, nx + 1, nz + 1),
             h=h)
    m.depth = np.repeat(depth, 6)
    return m


def endocardial_sites(m: Mesh, count: int, seed: int, endo=(35.0, 70.0), radius: float = 1.5,
                      z_max: float = -45.0) -> list:
    """`count` node sets (balls of `radius` mm) around seeded nodes of the endocardial surface
    (nodes on or inside the endocardium's outer layer, x^2/a0^2 + y^2/a0^2 + z^2/c0^2 <= (1 +
    h/a0)^2) in the apical region z <= z_max on the septal side x <= 0."""
    a0, c0 = endo
    x = m.xyz
    f = (x[:, 0] ** 2 + x[:, 1] ** 2) / a0 ** 2 + x[:, 2] ** 2 / c0 ** 2
    cand = np.nonzero((f <= (1.0 + m.h / a0) ** 2) & (x[:, 2] <= z_max) & (x[:, 0] <= 0.0))[0]
    u = uniform01(seed, np.arange(count, dtype=np.uint64))
    sites = cand[(u * cand.size).astype(np.int64) % cand.size]
    out = []
    for sidx in sites:
        d = np.linalg.norm(x - x[sidx], axis=1)
        out.append(np.nonzero(d <= radius + 1e-9)[0].astype(np.int32))
    return out


def ellipsoid_tp06(h: float = 0.35, t_end: float = 300.0, seed: int = 5) -> Workload:
    """The truncated prolate-ellipsoid shell (endocardium 35/35/70 mm, 10 mm wall, cut at
    z = -30 mm, 31 % of the height from the apex: about 2.0 M nodes at h = 0.35 mm) with the
    rule-based fibres, TP06 epicardial cells, the small slab's tissue constants, dt = 0.02 ms,
    and five seeded apical/septal endocardial stimulus sites (1.5 mm balls, 2 ms at 1.0 uA/mm^2,
    all at t = 0)."""
    m = prolate_shell_mesh(h)
    st = [Stimulus(nodes, 0.0, 2.0, 1.0) for nodes in endocardial_sites(m, 5, seed)]
    return Workload(f"ellipsoid_h{h:g}_tp06", m, 0.17, 0.019, 140.0, 0.01, 0.5, 0.02, t_end, "tp06",
                    stimuli=st, atol=1e-5, rtol=1e-5, max_iter=100)


def nversion_slab(h: float, t_end: float = 100.0, cell: int = 2) -> Workload:
    """The N-version benchmark slab (Section 3.1.2, Table 3): 20x7x3 mm, fibres along x, spacing
    h (0.5, 0.2 or 0.1 mm), dt = 0.005 ms, chi = 140 /mm, Cm = 0.01 uF/mm^2, sigma_l =
    0.1334177, sigma_t = 0.0173515 S/m, ten Tusscher-Panfilov (cell type `cell`).  The 50 uA/mm^3
    volumetric stimulus enters as 50/chi uA/mm^2 of membrane current; it is applied for 2 ms to
    the nodes of the 1.5 mm corner cube at P1 = (0, 0, 0) (the table gives neither the corner
    region's size nor the duration)."""
    m = slab_mesh(20.0, 7.0, 3.0, h, fibre="x")
    st = [Stimulus(corner_nodes(m, 1.5), 0.0, 2.0, 50.0 / 140.0)]
    w = Workload(f"nversion_h{h:g}", m, 0.1334177, 0.0173515, 140.0, 0.01, 0.5, 0.005, t_end, "tp06",
                 stimuli=st, atol=0.0, rtol=1e-8, max_iter=1000)
    w.tp06_cell = cell
    return w


def diagonal_nodes(m: Mesh, count: int = 11) -> np.ndarray:
    """Nodes nearest to `count` equally spaced points on the diagonal from P1 = (0, 0, 0) to the
    opposite corner P8 (both corners are nodes)."""
    hi = m.xyz.max(axis=0)
    t = np.linspace(0.0, 1.0, count)
    pts = t[:, None] * hi[None, :]
    return np.array([int(np.argmin(np.linalg.norm(m.xyz - p, axis=1))) for p in pts], dtype=np.int64)


def random_vector(n: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Seeded uniform vector for operator tests."""
    return lo + (hi - lo) * uniform01(seed, np.arange(n, dtype=np.uint64))
