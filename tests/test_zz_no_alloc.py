"""tc_apply_operator_static: operator products without any device allocation.

It serves callers that cannot allocate device memory while they run; its output must equal
tc_apply_operator's on consecutive calls (the shared static staging keeps the previous call's
contents, so the second call checks that nothing leaks from the first).  Collected last."""
import numpy as np
import pytest

from oracle import fem
from paper_2510_12011_b300 import inputs as I
from paper_2510_12011_b300 import tc

pytestmark = pytest.mark.gpu


def test_static_operator_matches_allocating_entry_point():
    w = I.slab_small_ms()
    sim = tc.from_workload(w)
    m = w.mesh
    M, K = fem.mass_stiffness(m.xyz, m.tets, m.fibres, w.sigma_l, w.sigma_t)
    A = fem.system_matrix(M, K, w.chi, w.cm, w.theta, w.dt)
    for call, seed in enumerate((101, 202)):
        x = I.random_vector(w.mesh.n_nodes, seed, -90.0, 30.0)
        for op, mat in ((tc.TC_OP_M, M), (tc.TC_OP_K, K), (tc.TC_OP_A, A)):
            ref = sim.apply(op, x)
            got = sim.apply_static(op, x)
            # the bound of the operator parity tests: reordered sums of the row's products
            bound = 32 * np.finfo(float).eps * (abs(mat) @ np.abs(x))
            assert np.all(np.abs(got - ref) <= bound), (call, op)


def test_static_operator_rejects_meshes_above_its_limit():
    w = I.slab_custom(24.0, 12.0, 6.0, 0.2, t_end=0.1)   # 121 x 61 x 31 = 228,811 nodes: fits
    sim = tc.from_workload(w)
    x = I.random_vector(w.mesh.n_nodes, 7)
    assert np.array_equal(sim.apply_static(tc.TC_OP_A, x), sim.apply(tc.TC_OP_A, x))
    big = I.slab_custom(30.0, 12.0, 6.0, 0.2, t_end=0.1)  # 151 x 61 x 31 = 285,541 nodes
    sim2 = tc.from_workload(big)
    with pytest.raises(tc.TcError) as e:
        sim2.apply_static(tc.TC_OP_A, np.zeros(big.mesh.n_nodes))
    assert e.value.status == tc.TC_ERR_ARG and "262144" in e.value.message


def test_static_operator_rejects_fp32_simulations_and_wrong_sizes():
    """The documented argument contract: TC_FP64 simulations only, n equal to the node count."""
    w = I.slab_small_ms()
    sim32 = tc.from_workload(w, precision=tc.TC_FP32)
    x = I.random_vector(w.mesh.n_nodes, 11)
    with pytest.raises(tc.TcError) as e:
        sim32.apply_static(tc.TC_OP_A, x)
    assert e.value.status == tc.TC_ERR_ARG and "FP64" in e.value.message
    sim = tc.from_workload(w)
    for bad in (x[:-1], np.concatenate([x, [0.0]])):
        with pytest.raises(tc.TcError) as e:
            sim.apply_static(tc.TC_OP_A, bad)
        assert e.value.status == tc.TC_ERR_ARG
    # a rejected call leaves the entry point usable
    assert np.array_equal(sim.apply_static(tc.TC_OP_A, x), sim.apply(tc.TC_OP_A, x))
