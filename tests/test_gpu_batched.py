"""Batched form: several meshes (disconnected components) in one simulation, each with its
own PCG, stepped by one cooperative launch per step; CUDA-graph replay of the step loop;
launch-shape autotuning.  A batch must reproduce independent runs of its instances."""
import numpy as np
import pytest

from oracle.monodomain import Monodomain
from paper_2510_12011_b300 import inputs as I
from paper_2510_12011_b300 import tc

pytestmark = pytest.mark.gpu


def _small_batch():
    dims = [(3.0, 2.0, 1.0, 0.25, 0.17, 0.019), (2.0, 1.0, 0.75, 0.25, 0.3, 0.05),
            (4.0, 1.5, 1.0, 0.25, 0.1, 0.012), (1.0, 1.0, 0.5, 0.25, 0.2, 0.03)]
    parts = []
    for i, (lx, ly, lz, h, sl, st) in enumerate(dims):
        w = I.slab_custom(lx, ly, lz, h, jitter=0.1, seed=20 + i, rtol=1e-10, t_end=3.0)
        w.sigma_l, w.sigma_t = sl, st
        w.stimuli = [I.Stimulus(w.stimuli[0].nodes, 0.1 * i, 1.5, 0.6)]
        parts.append(w)
    return I.join_workloads(parts)


@pytest.fixture(scope="module")
def batch_run():
    b = _small_batch()
    g = tc.from_workload(b.workload)
    assert g.layout()["n_components"] == 4
    st = g.step(300)
    return b, g, st


def test_batch_matches_oracle_per_instance(batch_run):
    b, g, st = batch_run
    V, act = g.read(), g.activation_times()
    for w, off in zip(b.instances, b.node_offset):
        o = Monodomain(w).run(300)
        n = w.mesh.n_nodes
        assert np.abs(V[off:off + n] - o.V).max() <= 1e-8
        assert np.abs(act[off:off + n] - o.act).max() <= 1e-6
    assert st["not_converged"] == 0


def test_batch_matches_single_runs(batch_run):
    b, g, st = batch_run
    V = g.read()
    total = 0
    for w, off in zip(b.instances, b.node_offset):
        s1 = tc.from_workload(w)
        st1 = s1.step(300)
        total += st1["cg_iterations"]
        assert np.abs(V[off:off + w.mesh.n_nodes] - s1.read()).max() <= 1e-10
    assert st["cg_iterations"] == total   # every instance stops on its own test


def test_graph_replay_equals_direct_launches():
    w = I.slab_small_ms()
    a = tc.from_workload(w)
    a.set_graphs(True)
    b = tc.from_workload(w)
    b.set_graphs(False)
    for n in (95, 31, 64):   # graph groups of 30 plus remainders, across buffer phases
        sa, sb = a.step(n), b.step(n)
        assert sa["cg_iterations"] == sb["cg_iterations"]
    assert np.array_equal(a.read(), b.read())
    assert np.array_equal(a.activation_times(), b.activation_times())
    assert a.step_index == b.step_index == 190


def test_autotune_restores_state_and_picks_a_shape():
    w = I.slab_custom(12.0, 6.0, 3.0, 0.25, t_end=1.0)
    a = tc.from_workload(w)
    a.step(10)
    v10 = a.read()
    res = a.autotune(5)
    assert res["pcg_threads"] in (512, 1024) and res["ms_per_step"] > 0
    assert np.array_equal(a.read(), v10) and a.step_index == 10
    lay = a.layout()
    assert (lay["pcg_threads"], lay["blocks_per_sm"]) == (res["pcg_threads"], res["blocks_per_sm"])
    a.step(20)
    ref = tc.from_workload(w)
    ref.step(30)
    assert np.abs(a.read() - ref.read()).max() <= 1e-9


def test_full_batch_steps_in_fp32():
    # the 64-slab batch (5.3 M nodes): after 3 ms every instance has activated around its own
    # stimulus site, and nowhere else yet
    b = I.batched_slabs(t_end=3.0)
    g = tc.from_workload(b.workload, precision=tc.TC_FP32)
    assert g.layout()["n_components"] == 64
    st = g.step(300)
    assert st["not_converged"] == 0
    act = g.activation_times()
    for w, off in zip(b.instances, b.node_offset):
        nodes = w.stimuli[0].nodes + off
        a = act[off:off + w.mesh.n_nodes]
        assert np.mean(act[nodes] >= 0.0) > 0.5
        assert 0 < np.count_nonzero(a >= 0.0) < a.size
    # sampled against the oracle: the smallest and the median instance of the full batch, each
    # stepped on its own by the FP64 oracle; the FP32 form's bar (activation well within 1 ms)
    v = g.read()
    sizes = [w.mesh.n_nodes for w in b.instances]
    for i in (int(np.argmin(sizes)), int(np.argsort(sizes)[len(sizes) // 2])):
        w, off = b.instances[i], b.node_offset[i]
        o = Monodomain(w).run(300)
        ai = act[off:off + w.mesh.n_nodes]
        both = (ai >= 0) & (o.act >= 0)
        assert both.sum() >= 0.95 * (o.act >= 0).sum() > 0
        assert np.abs(ai[both] - o.act[both]).max() < 0.05
        assert np.abs(v[off:off + w.mesh.n_nodes] - o.V).max() < 5.0


def test_layout_autotuner_over_sell_window_and_launch_shape():
    """The layout autotuner times each SELL window with its best launch shape and keeps the
    fastest; simulations laid out with different windows compute the same solution (up to the
    order of additions)."""
    from paper_2510_12011_b300 import tune
    b = I.batched_slabs(count=6, seed=11, h=0.5, t_end=5.0)
    w = b.workload
    w.rtol, w.atol, w.max_iter = 1e-10, 0.0, 1000
    res = tune.autotune_layout(w, precision=tc.TC_FP64, sigmas=(1, 1024), trial_steps=10)
    assert {t["sell_sigma"] for t in res["trials"]} == {1, 1024}
    assert res["ms_per_step"] == min(t["ms_per_step"] for t in res["trials"])
    assert res["trials"][0]["padded_nnz"] >= res["trials"][1]["padded_nnz"]
    vs = []
    for sg in (1, 1024):
        res["mesh"].set_sell_sigma(sg)
        sim = tc.from_workload(w, precision=tc.TC_FP64, mesh=res["mesh"])
        sim.step(200)
        vs.append(sim.read())
        sim.close()
    assert np.abs(vs[0] - vs[1]).max() <= 1e-9 * max(1.0, np.abs(vs[1]).max())


def test_one_launch_per_step_matches_two_launches():
    """Mitchell-Schaeffer steps run as one persistent launch (the ionic update is the PCG kernel's
    first phase; the barrier words are reset by the last block out): bitwise the same as the ionic
    kernel followed by the PCG kernel, with graphs and with host launches, and one launch per step."""
    import os
    b = I.batched_slabs(count=6, seed=7, t_end=5.0)
    w = b.workload
    runs = {}
    for fuse in ("1", "0"):
        os.environ["TC_FUSE_IONIC"] = fuse
        try:
            sim = tc.from_workload(w, precision=tc.TC_FP32)
        finally:
            os.environ.pop("TC_FUSE_IONIC", None)
        sim.step(100)                      # graphs
        sim.set_profiling(True)
        sim.reset_profile()
        sim.step(7)                        # host launches, counted
        prof = sim.profile()
        runs[fuse] = (sim.read(), sim.activation_times(), prof)
        sim.close()
    assert np.array_equal(runs["1"][0], runs["0"][0]) and np.array_equal(runs["1"][1], runs["0"][1])
    assert runs["1"][2]["ionic_launches"] == 0 and runs["1"][2]["pcg_launches"] == 7
    assert runs["0"][2]["ionic_launches"] == 7 and runs["0"][2]["pcg_launches"] == 7
