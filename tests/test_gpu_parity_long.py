"""Long GPU-vs-oracle parity runs of the FP64 path, through the C ABI, at the bar of the plain
method: |V_gpu - V_oracle| <= 1e-8 mV after 1000 steps and |t_gpu - t_oracle| <= 1e-6 ms on every
activation (and repolarisation) time.

  * TP06 on the 945-node slab over a whole beat (400 ms, 20,000 steps): the FP64 ionic kernel holds
    the concentration logarithms across steps, so its rounding is exercised over the step counts
    where it would accumulate.
  * The N-version slab of Table 3 (Section 3.1.2) at its coarsest spacing, with the volumetric
    stimulus reading, until the far corner P8 has activated.
  * Two conductivity regions (Section 2.1; Listing 1 sets regions) stepped for 1000 steps.
The solver runs in parity mode (rtol 1e-10, atol 0), so the stopping rule is far below the bar."""
import numpy as np
import pytest

from oracle.monodomain import Monodomain
from paper_2510_12011_b300 import inputs as I
from paper_2510_12011_b300 import tc

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

V_TOL = 1e-8      # mV, after 1000 steps
ACT_TOL = 1e-6    # ms


def _parity_mode(w):
    w.rtol, w.atol, w.max_iter = 1e-10, 0.0, 1000
    return w


def _lockstep(w, checkpoints):
    """Run the oracle and the GPU side by side; at every checkpoint (a step count) record
    max |dV| and both runs' activation times."""
    o = Monodomain(w)
    g = tc.from_workload(w)
    out = {}
    done = 0
    for k in checkpoints:
        o.run(k - done)
        st = g.step(k - done)
        done = k
        assert st["not_converged"] == 0
        out[k] = {"dv": float(np.abs(g.read() - o.V).max()), "act_g": g.activation_times(w.v_threshold),
                  "act_o": o.act.copy()}
    return o, g, out


def _same_times(a_g, a_o, tol):
    assert np.array_equal(a_g >= 0, a_o >= 0)
    both = a_o >= 0
    if both.any():
        assert np.abs(a_g[both] - a_o[both]).max() <= tol


@pytest.fixture(scope="module")
def tp06_beat():
    w = _parity_mode(I.slab_small_ms())
    w.model, w.dt, w.tp06_cell, w.t_end = "tp06", 0.02, 2, 400.0
    w.name = "slab10x4x2_h0.5_tp06_beat"
    return w, _lockstep(w, [1000, 5000, 20000])


def test_tp06_fp64_1000_steps(tp06_beat):
    w, (o, g, out) = tp06_beat
    assert out[1000]["dv"] <= V_TOL
    _same_times(out[1000]["act_g"], out[1000]["act_o"], ACT_TOL)
    assert (out[1000]["act_o"] >= 0).sum() > 400      # the wave is crossing the slab


def test_tp06_fp64_full_beat(tp06_beat):
    """V at 100 ms and at the end of the beat, every node's activation, repolarisation (LRT) and
    APD90 against the oracle."""
    w, (o, g, out) = tp06_beat
    assert out[5000]["dv"] <= V_TOL
    assert out[20000]["dv"] <= V_TOL
    _same_times(out[20000]["act_g"], out[20000]["act_o"], ACT_TOL)
    assert np.all(out[20000]["act_o"] >= 0)
    lrt_o, apd_o = o.lrt, o.apd90()
    assert np.all(apd_o > 200.0) and np.all(lrt_o > 0.0)   # every node repolarised
    _same_times(g.repolarisation_times(), lrt_o, ACT_TOL)
    _same_times(g.apd90(), apd_o, ACT_TOL)
    for j in range(18):
        ref = o.state[j]
        got = g.read(tc.TC_FIELD_STATE + j)
        assert np.allclose(got, ref, rtol=1e-9, atol=1e-14), j


def test_nversion_slab_against_oracle():
    """Table 3's slab at dx = 0.5 mm (4,305 nodes, dt = 0.005 ms, TP06 epicardial, the 50 uA/mm^3
    corner stimulus read as 50/chi uA/mm^2 of membrane current for 2 ms): V after 1000 steps,
    then every node's activation time until the far corner P8 has activated (60 ms, 12,000
    steps), with the P1-P8 diagonal called out."""
    w = _parity_mode(I.nversion_slab(0.5, t_end=60.0))
    assert w.mesh.n_nodes == 4305
    o, g, out = _lockstep(w, [1000, w.n_steps])
    assert out[1000]["dv"] <= V_TOL
    a_g, a_o = out[w.n_steps]["act_g"], out[w.n_steps]["act_o"]
    assert np.all(a_o >= 0)                       # the whole slab, P8 included, has activated
    _same_times(a_g, a_o, ACT_TOL)
    d = I.diagonal_nodes(w.mesh, 11)
    assert np.all(np.diff(a_o[d]) > 0)
    assert np.abs(a_g[d] - a_o[d]).max() <= ACT_TOL


def test_two_region_conductivities_against_oracle():
    """A slab with two conductivity regions (y < 2 mm: the small slab's sigma; above: 1.8x along
    and 2.5x across the fibres), Mitchell-Schaeffer, 1000 steps and 30 ms of activation."""
    w = _parity_mode(I.slab_small_ms())
    m = w.mesh
    m.region = (m.xyz[m.tets, 1].mean(axis=1) > 2.0).astype(np.int32)
    assert 0 < m.region.sum() < m.n_tets
    w.sigma_l = np.array([0.17, 0.17 * 1.8])
    w.sigma_t = np.array([0.019, 0.019 * 2.5])
    w.name = "slab10x4x2_h0.5_ms_two_regions"
    o, g, out = _lockstep(w, [1000, 3000])
    assert out[1000]["dv"] <= V_TOL
    for k in (1000, 3000):
        _same_times(out[k]["act_g"], out[k]["act_o"], ACT_TOL)
    assert (out[3000]["act_o"] >= 0).sum() > 0.9 * m.n_nodes
    # the faster region activates first at equal distance from the stimulus
    ref = Monodomain(_parity_mode(I.slab_small_ms())).run(3000).act
    assert (out[3000]["act_o"] != ref).any()
