"""C-ABI library: loads, exports every declared symbol, host-side assembly and ordering.

Runs without a GPU: only host-only entry points are called here."""
import os
import re

import numpy as np
import pytest

from oracle import fem
from paper_2510_12011_b300 import inputs as I
from paper_2510_12011_b300 import tc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(tc_[a-z0-9_]+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    L = tc.lib()
    declared = _declared()
    assert len(declared) >= 25
    for name in declared:
        assert hasattr(L, name), name
    assert declared <= set(tc.exported_symbols())
    assert L.tc_version().decode().startswith("tc_b300")


@pytest.mark.parametrize("kind", ["small", "jittered_regions"])
def test_host_assembly_matches_oracle(kind):
    if kind == "small":
        w = I.slab_small_ms()
        m = w.mesh
        sl, st, reg = [w.sigma_l], [w.sigma_t], None
        region = np.zeros(m.n_tets, dtype=np.int32)
    else:
        m = I.slab_mesh(3.0, 2.0, 1.0, 0.25, jitter=0.15, seed=5, fibre="rotating")
        region = (m.xyz[m.tets, 0].mean(axis=1) > 1.5).astype(np.int32)
        sl, st, reg = [0.17, 0.4], [0.019, 0.1], region
    mesh = tc.Mesh(m.xyz, m.tets, m.fibres, reg)
    rp, col, mv, kv = mesh.matrices(sl, st)
    M, K = fem.mass_stiffness(m.xyz, m.tets, m.fibres, np.array(sl)[region], np.array(st)[region])
    assert np.array_equal(rp, M.indptr) and np.array_equal(col, M.indices)
    assert np.array_equal(K.indptr, M.indptr) and np.array_equal(K.indices, M.indices)
    assert np.abs(mv - M.data).max() <= 1e-15 * np.abs(M.data).max()
    assert np.abs(kv - K.data).max() <= 2e-15 * np.abs(K.data).max()


def test_host_assembly_exactly_symmetric():
    m = I.slab_mesh(3.0, 2.0, 1.0, 0.25, jitter=0.15, seed=9, fibre="rotating")
    mesh = tc.Mesh.from_inputs(m)
    rp, col, mv, kv = mesh.matrices(0.17, 0.019)
    import scipy.sparse as sp
    Mh = sp.csr_matrix((mv, col, rp))
    Kh = sp.csr_matrix((kv, col, rp))
    assert (Mh != Mh.T).nnz == 0 and (Kh != Kh.T).nnz == 0


def test_ordering_is_bandwidth_reducing_permutation():
    m = I.slab_mesh(6.0, 3.0, 2.0, 0.25, jitter=0.1, seed=2)
    mesh = tc.Mesh.from_inputs(m)
    rp, col, _, _ = mesh.matrices(0.17, 0.019)
    rows = np.repeat(np.arange(m.n_nodes), np.diff(rp))
    shuffled = np.random.default_rng(0).permutation(m.n_nodes)   # scramble, then reorder
    mesh2 = tc.Mesh(m.xyz[shuffled], np.argsort(shuffled)[m.tets], m.fibres)
    perm, sw = mesh2.ordering(1)
    assert np.array_equal(np.sort(perm), np.arange(m.n_nodes))
    inv = np.empty_like(perm)
    inv[perm] = np.arange(perm.size)
    rp2, col2, _, _ = mesh2.matrices(0.17, 0.019)
    rows2 = np.repeat(np.arange(m.n_nodes), np.diff(rp2))
    bw_rcm = np.abs(inv[rows2] - inv[col2]).max()
    bw_scrambled = np.abs(rows2 - col2).max()
    bw_lattice = np.abs(rows - col).max()
    assert bw_rcm <= 1.2 * bw_lattice and bw_rcm < bw_scrambled / 5
    # slice widths are the longest row of each 32-row slice
    deg = np.diff(rp2)[perm]
    pad = np.concatenate([deg, np.zeros((-deg.size) % 32, dtype=deg.dtype)])
    assert np.array_equal(sw, pad.reshape(-1, 32).max(axis=1))


def test_sell_sigma_sorting_reduces_padding():
    m = I.slab_mesh(8.0, 4.0, 2.0, 0.25)
    mesh = tc.Mesh.from_inputs(m)
    _, sw1 = mesh.ordering(1)
    _, sw2 = mesh.ordering(256)
    assert sw2.sum() <= sw1.sum()


def test_mesh_errors():
    m = I.slab_mesh(1.0, 1.0, 1.0, 0.5)
    bad = m.tets.copy()
    bad[3, 2] = m.n_nodes + 5
    with pytest.raises(tc.TcError) as e:
        tc.Mesh(m.xyz, bad)
    assert e.value.status == tc.TC_ERR_MESH and "out of range" in e.value.message
    flat = m.tets.copy()
    flat[0] = [0, 1, 2, 2]
    with pytest.raises(tc.TcError) as e:
        tc.Mesh(m.xyz, flat)
    assert e.value.status == tc.TC_ERR_MESH and "degenerate" in e.value.message
    fib = m.fibres.copy()
    fib[4] = 0.0
    with pytest.raises(tc.TcError) as e:
        tc.Mesh(m.xyz, m.tets, fib)
    assert e.value.status == tc.TC_ERR_MESH
    with pytest.raises(tc.TcError) as e:
        tc.Mesh(m.xyz[:3], m.tets[:0])
    assert e.value.status == tc.TC_ERR_ARG
    reg = np.zeros(m.n_tets, dtype=np.int32)
    reg[0] = 2
    mesh = tc.Mesh(m.xyz, m.tets, None, reg)
    with pytest.raises(tc.TcError) as e:
        mesh.matrices([0.1, 0.1], [0.01, 0.01])
    assert e.value.status == tc.TC_ERR_ARG
    with pytest.raises(tc.TcError) as e:
        mesh.matrices([0.1, 0.1, -1.0], [0.01, 0.01, 0.01])
    assert e.value.status == tc.TC_ERR_ARG


def test_negative_orientation_accepted():
    m = I.slab_mesh(1.0, 1.0, 1.0, 0.5)
    flipped = m.tets[:, [1, 0, 2, 3]]
    a = tc.Mesh(m.xyz, m.tets).matrices(0.17, 0.019)
    b = tc.Mesh(m.xyz, flipped).matrices(0.17, 0.019)
    for x, y in zip(a, b):
        assert np.allclose(x, y, rtol=1e-14, atol=0)


def test_component_layout_of_a_joined_mesh():
    parts = [I.slab_custom(1.0 + i, 1.0, 0.5, 0.25) for i in range(3)]
    b = I.join_workloads(parts)
    mesh = tc.Mesh.from_inputs(b.workload.mesh)
    nc, n_int = mesh.layout_size()
    sizes = [w.mesh.n_nodes for w in parts]
    assert nc == 3 and n_int == sum((s + 31) // 32 * 32 for s in sizes)
    perm, sw = mesh.ordering(1)
    assert np.array_equal(np.sort(perm), np.arange(sum(sizes)))
    assert sw.size == n_int // 32
    # the internal order keeps every component contiguous (in some order of components)
    comp = np.repeat(np.arange(3), sizes)
    k, seen = 0, set()
    while k < perm.size:
        c = comp[perm[k]]
        assert c not in seen
        seen.add(c)
        assert np.all(comp[perm[k:k + sizes[c]]] == c)
        k += sizes[c]
    assert seen == {0, 1, 2}


def test_monodomain_conductivity_from_bidomain_pairs():
    """Listing 1 configures regions with intra-/extracellular conductivities; the monodomain
    value per direction is their series combination.  Pins: equal intra and extra values halve,
    an extracellular value much larger than the intracellular one leaves the intracellular one,
    and the ABI agrees with the oracle; non-positive input is rejected."""
    import numpy as np
    import pytest
    from oracle import fem
    from paper_2510_12011_b300 import tc
    sl, st = tc.monodomain_conductivity([0.2, 0.3], [0.02, 0.05], [0.2, 0.3], [0.02, 0.05])
    assert np.allclose(sl, [0.1, 0.15], rtol=0, atol=1e-15) and np.allclose(st, [0.01, 0.025], rtol=0, atol=1e-15)
    sl, st = tc.monodomain_conductivity([0.17], [0.019], [1e12], [1e12])
    assert abs(sl[0] - 0.17) < 1e-12 and abs(st[0] - 0.019) < 1e-12
    rng = np.random.default_rng(4)
    v = rng.uniform(0.01, 1.0, (4, 9))
    got = tc.monodomain_conductivity(*v)
    ref = fem.monodomain_conductivity(*v)
    assert np.allclose(got[0], ref[0], rtol=1e-15) and np.allclose(got[1], ref[1], rtol=1e-15)
    with pytest.raises(tc.TcError):
        tc.monodomain_conductivity([0.1], [0.0], [0.1], [0.1])


def test_math_tables_match_their_definition():
    """The exp and log tables of the FP64 ionic kernel are the values math_tables.py derives
    from their definitions (2^(j/2048); fl(1/(1 + j/128)) and -ln of it) with mpmath, and the
    exp polynomial's quadratic coefficient is the one it derives."""
    import contextlib
    import io
    import re
    import runpy
    from pathlib import Path
    csrc = Path(__file__).resolve().parents[1] / "paper_2510_12011_b300" / "csrc"
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        runpy.run_path(str(csrc / "math_tables.py"), run_name="__main__")
    gen = buf.getvalue()
    src = (csrc / "ionic_tp06.cuh").read_text() + (csrc / "exp2_table.inc").read_text()

    def vals(text, key):
        i = text.index("{", text.index(key))
        return [float.fromhex(v) for v in re.findall(r"-?0x[0-9a-fA-F.]+p[+-]?\d+", text[i:text.index("}", i)])]
    for name, n in (("kExp2Hi", 2048), ("kExp2Lo", 2048), ("kLogInv", 128), ("kLogHi", 128), ("kLogLo", 128)):
        v = vals(src, f"double {name}[{n}] =")
        assert len(v) == n and v == vals(gen, f"{name} ="), name
    c2 = re.search(r"kExpC2 = (\S+);", src).group(1)
    assert float.fromhex(c2) == float.fromhex(re.search(r"kExpC2 = (\S+);", gen).group(1))
    assert 0.0 < float.fromhex(c2) - 0.5 < 2e-9
    for name in ("kExp2A1", "kExp2A2", "kExp2A3"):
        assert float.fromhex(re.search(name + r" = (0x[0-9a-fA-F.]+p[+-]?\d+)", src).group(1)) == \
            float.fromhex(re.search(name + r" = (0x[0-9a-fA-F.]+p[+-]?\d+)", gen).group(1)), name
