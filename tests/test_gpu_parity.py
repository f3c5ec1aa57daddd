"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Tolerances: |V_gpu - V_oracle| <= 1e-8 mV after 1000 steps and |act_gpu - act_oracle| <= 1e-6 ms
(the accuracy bar of the plain FP64 method); single kernels are held to rounding-level bounds
derived from their sums (reordered sums of at most ~27 products)."""
import numpy as np
import pytest

from oracle import fem
from oracle.monodomain import Monodomain
from oracle.pcg import pcg
from paper_2510_12011_b300 import inputs as I
from paper_2510_12011_b300 import tc

pytestmark = pytest.mark.gpu

V_TOL = 1e-8      # mV
ACT_TOL = 1e-6    # ms


def _sim(w, **kw):
    return tc.from_workload(w, **kw)


def _oracle_mats(m, sl, st):
    return fem.mass_stiffness(m.xyz, m.tets, m.fibres, sl, st)


@pytest.mark.parametrize("kind", ["small", "ragged_regions"])
def test_operators_match_oracle(kind):
    if kind == "small":
        w = I.slab_small_ms()
        sim = _sim(w)
        M, K = _oracle_mats(w.mesh, w.sigma_l, w.sigma_t)
        chi, cm, th, dt = w.chi, w.cm, w.theta, w.dt
    else:
        m = I.slab_mesh(5.25, 2.5, 1.75, 0.25, jitter=0.15, seed=3, fibre="rotating")
        assert m.n_nodes % 32 != 0
        region = (m.xyz[m.tets, 1].mean(axis=1) > 1.0).astype(np.int32)
        sl, st = np.array([0.17, 0.3]), np.array([0.019, 0.05])
        mesh = tc.Mesh(m.xyz, m.tets, m.fibres, region)
        chi, cm, th, dt = 140.0, 0.01, 0.5, 0.02
        sim = tc.Simulation(mesh, sl, st, chi, cm, th, dt)
        M, K = _oracle_mats(m, sl[region], st[region])
    A = fem.system_matrix(M, K, chi, cm, th, dt)
    x = I.random_vector(M.shape[0], 17, -90.0, 30.0)
    for op, ref in ((tc.TC_OP_M, M), (tc.TC_OP_K, K), (tc.TC_OP_A, A)):
        y = sim.apply(op, x)
        bound = 32 * np.finfo(float).eps * (abs(ref) @ np.abs(x))
        assert np.all(np.abs(y - ref @ x) <= bound + 1e-300)


@pytest.fixture(scope="module")
def small_runs():
    w = I.slab_small_ms()
    o = Monodomain(w)
    g = _sim(w)
    o.run(1)
    g.step(1)
    one = (g.read(), g.read(tc.TC_FIELD_STATE), o.V.copy(), o.state[0].copy())
    o.run(999)
    st = g.step(999)
    k1000 = (g.read(), g.read(tc.TC_FIELD_STATE), g.activation_times(0.0), o.V.copy(),
             o.state[0].copy(), o.act.copy(), st, sum(o.iters[1:]))
    o.run(4000)
    g.step(4000)
    k5000 = (g.read(), g.activation_times(0.0), o.V.copy(), o.act.copy())
    return one, k1000, k5000


def test_first_step_matches_oracle(small_runs):
    vg, hg, vo, ho = small_runs[0]
    assert np.abs(vg - vo).max() <= 1e-11
    assert np.abs(hg - ho).max() <= 1e-14


def test_v_after_1000_steps(small_runs):
    vg, hg, ag, vo, ho, ao, st, oiters = small_runs[1]
    assert np.abs(vg - vo).max() <= V_TOL
    assert np.abs(hg - ho).max() <= 1e-10
    assert np.array_equal(ag >= 0, ao >= 0)
    assert np.abs(ag - ao).max() <= ACT_TOL
    assert st["not_converged"] == 0
    # the same stopping decisions as the oracle, up to a handful of borderline steps
    assert abs(st["cg_iterations"] - oiters) <= 5


def test_activation_times_full_run(small_runs):
    vg, ag, vo, ao = small_runs[2]
    assert np.all(ao >= 0) and np.all(ag >= 0)
    assert np.abs(ag - ao).max() <= ACT_TOL
    assert np.abs(vg - vo).max() <= V_TOL


def test_bitwise_determinism():
    w = I.slab_small_ms()
    a, b = _sim(w), _sim(w)
    a.step(300)
    b.step(300)
    assert np.array_equal(a.read(), b.read())
    assert np.array_equal(a.activation_times(), b.activation_times())


def test_checkpoint_restart_bitwise():
    w = I.slab_small_ms()
    ref = _sim(w)
    ref.step(400)
    a = _sim(w)
    a.step(200)
    saved = {f: a.read(f) for f in (tc.TC_FIELD_V, tc.TC_FIELD_V_PREV, tc.TC_FIELD_STATE)}
    k = a.step_index
    b = _sim(w)
    for f, v in saved.items():
        b.write(f, v)
    b.step_index = k
    b.step(200)
    assert np.array_equal(b.read(), ref.read())
    assert b.step_index == 400


@pytest.mark.parametrize("n_tets", [1, 2, 6])
def test_tiny_meshes(n_tets):
    m = I.slab_mesh(0.5, 0.5, 0.5, 0.5)
    keep = m.tets[:n_tets]
    used = np.unique(keep)
    remap = np.full(m.n_nodes, -1)
    remap[used] = np.arange(used.size)
    mesh = I.Mesh(m.xyz[used], remap[keep].astype(np.int32), m.fibres[:n_tets],
                  m.region[:n_tets], m.lattice[used], m.shape, m.h)
    w = I.Workload("tiny", mesh, 0.17, 0.019, 140.0, 0.01, 0.5, 0.01, 1.0, "ms",
                   stimuli=[I.Stimulus(np.array([0], dtype=np.int32), 0.0, 0.5, 2.0)])
    o = Monodomain(w).run(300)
    g = _sim(w)
    g.step(300)
    assert np.abs(g.read() - o.V).max() <= V_TOL
    assert np.abs(g.activation_times() - o.act).max() <= ACT_TOL


@pytest.mark.parametrize("dims", [(2.0, 1.0, 1.0), (3.0, 2.0, 1.0), (4.0, 2.0, 1.5), (5.0, 3.0, 1.5)])
def test_few_slice_meshes(dims):
    """Meshes of 2 to 10 SELL slices (45 to 308 nodes, the last slice ragged): one PCG block whose
    only round of slices is short, so every slice's row product is split over several warps by
    column range (8, 8, 5 and 3 warps per slice) and added back through shared memory."""
    m = I.slab_mesh(*dims, 0.5, jitter=0.15, seed=3)
    w = I.Workload("few_slices", m, 0.17, 0.019, 140.0, 0.01, 0.5, 0.01, 1.0, "ms",
                   stimuli=[I.Stimulus(I.corner_nodes(m, 0.5), 0.0, 0.5, 2.0)],
                   atol=0.0, rtol=1e-10, max_iter=1000)
    o = Monodomain(w).run(300)
    g = _sim(w)
    g.step(300)
    assert np.abs(g.read() - o.V).max() <= V_TOL
    assert np.abs(g.activation_times() - o.act).max() <= ACT_TOL


def test_iteration_cap_and_zero_residual():
    w = I.slab_small_ms()
    g = _sim(w)
    g.set_solver(0.0, 1e-10, 1)
    st = g.step(20)
    assert st["not_converged"] == 20 and st["max_iterations"] == 1 and st["cg_iterations"] == 20
    o = Monodomain(w)
    o.w.max_iter = 1
    o.run(20)
    assert np.abs(g.read() - o.V).max() <= 1e-10
    # resting tissue at 0 mV without stimulus: every term of r_0 is exactly zero, so the
    # PCG returns x_0 after no iteration (the z_0 = 0 case of Algorithm 1) and V stays at rest
    w2 = I.slab_small_ms()
    w2.stimuli = []
    w2.ms.v_min, w2.ms.v_max = 0.0, 100.0
    g2 = _sim(w2)
    st = g2.step(50)
    assert st["cg_iterations"] == 0 and st["not_converged"] == 0 and st["last_z0norm"] == 0.0
    assert np.all(g2.read() == 0.0)
    o2 = Monodomain(w2).run(5)
    assert o2.iters == [0] * 5 and np.all(o2.V == 0.0)


def test_error_codes():
    w = I.slab_small_ms()
    mesh = tc.Mesh.from_inputs(w.mesh)
    sim = tc.Simulation(mesh, w.sigma_l, w.sigma_t, w.chi, w.cm, w.theta, w.dt)
    with pytest.raises(tc.TcError) as e:
        sim.step(1)
    assert e.value.status == tc.TC_ERR_STATE
    with pytest.raises(tc.TcError) as e:
        sim.set_ionic(tc.TC_MODEL_MS, [0.3, 6.0])
    assert e.value.status == tc.TC_ERR_ARG
    sim.set_ionic(tc.TC_MODEL_MS, w.ms.as_array())
    with pytest.raises(tc.TcError) as e:
        sim.add_stimulus([0, 945], 0.0, 1.0, 0.5)
    assert e.value.status == tc.TC_ERR_ARG
    with pytest.raises(tc.TcError) as e:
        sim.read(99)
    assert e.value.status == tc.TC_ERR_ARG
    sim.step(2)
    with pytest.raises(tc.TcError) as e:
        sim.set_activation_threshold(-10.0)
    assert e.value.status == tc.TC_ERR_STATE
    with pytest.raises(tc.TcError) as e:
        sim.activation_times(-10.0)
    assert e.value.status == tc.TC_ERR_STATE
    with pytest.raises(tc.TcError) as e:
        tc.Simulation(mesh, w.sigma_l, w.sigma_t, w.chi, w.cm, 1.5, w.dt)
    assert e.value.status == tc.TC_ERR_ARG
    with pytest.raises(tc.TcError) as e:
        tc.Simulation(mesh, w.sigma_l, w.sigma_t, w.chi, w.cm, w.theta, w.dt, precision=7)
    assert e.value.status == tc.TC_ERR_ARG


def test_barrier_timeout_returns_status_and_context_survives():
    w = I.slab_custom(12.0, 6.0, 3.0, 0.25, t_end=1.0)
    g = _sim(w)
    assert g.size()["n_blocks"] > 8
    g.set_wait_limit(1)
    with pytest.raises(tc.TcError) as e:
        g.step(3)
    assert e.value.status == tc.TC_ERR_TIMEOUT
    g.set_wait_limit(1 << 26)
    g.set_ionic(tc.TC_MODEL_MS, w.ms.as_array())
    g.step(20)
    o = Monodomain(w).run(20)
    assert np.abs(g.read() - o.V).max() <= V_TOL


@pytest.mark.slow
def test_large_slab_full_size_parity():
    # 40x16x6 mm, h = 0.2 mm (504,711 nodes), the bench's launch configuration, parity mode
    w = I.slab_large("ms")
    w.rtol, w.atol, w.max_iter = 1e-10, 0.0, 1000
    g = _sim(w)
    size = g.size()
    assert size["n_nodes"] == 504711 and size["nnz"] == 7371731
    o = Monodomain(w)
    for _ in range(3):
        o.step()
    g.step(3)
    assert np.abs(g.read() - o.V).max() <= V_TOL
    assert np.abs(g.read(tc.TC_FIELD_STATE) - o.state[0]).max() <= 1e-12


@pytest.mark.slow
def test_large_slab_tp06_full_size_parity():
    """The headline workload at full size (504,711 nodes, TP06 epicardial, FP64) in the bench's
    launch configuration, with the solver in parity mode: 120 steps (2.4 ms: through the 2 ms
    stimulus and past it, the corner's upstroke under way), V, every activation time and all 18
    states against the oracle."""
    w = I.slab_large("tp06")
    w.rtol, w.atol, w.max_iter = 1e-10, 0.0, 1000
    g = _sim(w)
    o = Monodomain(w)
    for _ in range(120):
        o.step()
    g.step(120)
    a_g, a_o = g.activation_times(), o.act
    assert (a_o >= 0).sum() > 100 and np.array_equal(a_g >= 0, a_o >= 0)
    assert np.abs(a_g[a_o >= 0] - a_o[a_o >= 0]).max() <= ACT_TOL
    assert np.abs(g.read() - o.V).max() <= V_TOL
    for j in range(18):
        ref = o.state[j]
        got = g.read(tc.TC_FIELD_STATE + j)
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-15), j


@pytest.mark.gpu
@pytest.mark.slow
def test_nversion_activation_converges_with_refinement():
    """N-version slab (Section 3.1.2, Table 3) at the table's spacings 0.5, 0.2 and 0.1 mm, FP64:
    every node activates, activation time grows along the P1-P8 diagonal, and the change from
    0.2 to 0.1 mm is smaller than the change from 0.5 to 0.2 mm (self-convergence)."""
    from paper_2510_12011_b300 import nversion
    res = nversion.study((0.5, 0.2, 0.1), t_end=100.0)
    for r in res:
        assert r["all_activated"]
        act = np.asarray(r["act_ms"])
        assert np.all(np.diff(act) > 0)
    assert res[2]["diff_to_coarser_ms_max"] < res[1]["diff_to_coarser_ms_max"]


@pytest.mark.slow
def test_ellipsoid_full_size_parity():
    """The precision form's and the surrogate's workload at full size (the truncated ellipsoid,
    2,136,691 nodes, 12,075,312 tets, TP06 epicardial, five endocardial stimulus sites), solver in
    parity mode: FP64 against the oracle after 3 steps to the FP64 bar; the FP32 form against the
    same oracle run to FP32 resolution (a value of V near -85 mV is resolved to 8e-6 mV in FP32;
    the CG iterations and the ionic update add rounding of that order per step)."""
    w = I.ellipsoid_tp06(t_end=0.06)
    w.rtol, w.atol, w.max_iter = 1e-10, 0.0, 1000
    mesh = tc.Mesh.from_inputs(w.mesh)
    o = Monodomain(w)
    o.run(3)
    g = tc.from_workload(w, mesh=mesh)
    g.step(3)
    assert np.abs(g.read() - o.V).max() <= V_TOL
    for j in (0, 2, 9, 12, 17):   # Ki, Cai, m, d, r
        assert np.allclose(g.read(tc.TC_FIELD_STATE + j), o.state[j], rtol=1e-12, atol=1e-15), j
    g.close()
    g32 = tc.from_workload(w, precision=tc.TC_FP32, mesh=mesh)
    g32.step(3)
    assert np.abs(g32.read() - o.V).max() <= 1e-3
    assert np.allclose(g32.read(tc.TC_FIELD_STATE + 9), o.state[9], rtol=1e-4, atol=1e-8)
