"""Pins of the oracle's ionic model, stimulus, activation capture and manufactured solutions."""
import numpy as np
import pytest
from scipy.integrate import solve_ivp

from oracle import ionic, mms
from oracle.monodomain import Monodomain, capture, stimulus_current
from paper_2510_12011_b300 import inputs as I

P = I.MSParams()
CM = 0.01


def test_ms_rest_is_equilibrium():
    V, h = ionic.ms_rest(4, P)
    h2, i_ion = ionic.ms_step(V, h, 0.01, CM, P)
    assert np.all(i_ion == 0.0) and np.all(h2 == 1.0)


def test_ms_gate_rush_larsen_closed_forms():
    # below the gate threshold h relaxes to 1 with tau_open, above it decays with tau_close;
    # Rush-Larsen is exact for a frozen V: h_n = h_inf + (h_0 - h_inf) exp(-n dt / tau).
    dt, n = 0.02, 500
    V = np.array([-79.0, -70.0, 0.0, 15.0])   # v = 0.01, 0.1, 0.8, 0.95
    h = np.full(4, 0.3)
    for _ in range(n):
        h, _ = ionic.ms_step(V, h, dt, CM, P)
    t = n * dt
    ref = np.array([1 - 0.7 * np.exp(-t / P.tau_open)] * 2 + [0.3 * np.exp(-t / P.tau_close)] * 2)
    assert np.allclose(h, ref, rtol=1e-12)


def test_ms_current_hand_values():
    # v = 0.5, h_new = 1 (gate open, tau_open huge effect removed by dt -> 0):
    # J_in = 0.25 * 0.5 / 0.3, J_out = -0.5 / 6, I_ion = -Cm * 100 * (J_in + J_out)
    V = np.array([-30.0])
    h, i_ion = ionic.ms_step(V, np.array([0.0]), 0.0, CM, P)   # dt = 0: h unchanged
    assert h[0] == 0.0 and abs(i_ion[0] - (-CM * 100.0 * (-0.5 / 6.0))) < 1e-15
    h, i_ion = ionic.ms_step(V, np.array([1.0]), 0.0, CM, P)
    j = 0.125 / 0.3 - 0.5 / 6.0
    assert abs(i_ion[0] - (-CM * 100.0 * j)) < 1e-15


def _ms_rhs(t, y, stim, dur):
    v, h = y
    dv = h * v * v * (1 - v) / P.tau_in - v / P.tau_out + (stim / (CM * 100.0) if t < dur else 0.0)
    dh = (1 - h) / P.tau_open if v < P.v_gate else -h / P.tau_close
    return [dv, dh]


def _decoupled_run(dt, t_end):
    """Monodomain with sigma = 0 on every node: each node is a single cell, V^{k+1} =
    V^k + dt (I_stim - I_ion)/Cm (forward Euler), gate by Rush-Larsen."""
    w = I.slab_custom(1.0, 1.0, 1.0, 0.5, dt=dt, rtol=1e-14, t_end=t_end, stim_mm=0.0)
    w.sigma_l = w.sigma_t = 0.0
    w.stimuli = [I.Stimulus(np.array([0], dtype=np.int32), 0.0, 1.0, 0.5)]
    s = Monodomain(w)
    out = []
    for _ in range(w.n_steps):
        s.step()
        out.append(s.V[0])
    return np.array(out), s


def test_single_cell_reduction_converges_first_order():
    # reference: the MS ODE integrated to 1e-11 (scipy LSODA), v -> V
    t_end = 20.0
    ref = solve_ivp(_ms_rhs, (0.0, t_end), [0.0, 1.0], args=(0.5, 1.0), method="LSODA",
                    rtol=1e-11, atol=1e-12, dense_output=True, max_step=0.01)
    errs = []
    for dt in (0.01, 0.005, 0.0025):
        v, s = _decoupled_run(dt, t_end)
        t = dt * np.arange(1, v.size + 1)
        vref = -80.0 + 100.0 * ref.sol(t)[0]
        errs.append(np.abs(v - vref).max())
        assert np.allclose(s.V[1:], -80.0, rtol=0, atol=1e-10)   # unstimulated cells rest
    assert errs[0] < 2.0
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 1.6 < r1 < 2.4 and 1.6 < r2 < 2.4


def test_ms_upper_fixed_point():
    """With the gate held open (tau_close -> infinity) a stimulated cell settles where
    h v (1 - v) / tau_in = v / tau_out with h = 1: v* = (1 + sqrt(1 - 4 tau_in / tau_out)) / 2
    (0.947 for the default constants).  Forward Euler keeps the ODE's fixed points, so the
    decoupled monodomain step reaches V* = V_min + (V_max - V_min) v* to rounding."""
    w = I.slab_custom(1.0, 1.0, 1.0, 0.5, dt=0.01, rtol=1e-14, t_end=60.0, stim_mm=0.0)
    w.sigma_l = w.sigma_t = 0.0
    w.ms = I.MSParams(tau_close=1e12)
    w.stimuli = [I.Stimulus(np.array([0], dtype=np.int32), 0.0, 1.0, 0.5)]
    s = Monodomain(w)
    for _ in range(w.n_steps):
        s.step()
    v_star = (1.0 + np.sqrt(1.0 - 4.0 * P.tau_in / P.tau_out)) / 2.0
    assert abs(v_star - 0.9472135955) < 1e-10
    assert abs(s.V[0] - (-80.0 + 100.0 * v_star)) < 1e-8
    assert np.allclose(s.V[1:], -80.0, rtol=0, atol=1e-10)


def test_stimulus_window():
    nodes = np.array([1, 3], dtype=np.int32)
    st = [I.Stimulus(nodes, 0.5, 2.0, 0.7), I.Stimulus(np.array([3]), 1.0, 0.05, 0.1)]
    dt = 0.01
    on = [k for k in range(400) if stimulus_current(st, k, dt, 5)[1] != 0.0]
    assert on[0] == 50 and on[-1] == 249 and len(on) == 200
    assert abs(stimulus_current(st, 100, dt, 5)[3] - 0.8) < 1e-15
    assert stimulus_current(st, 105, dt, 5)[3] == 0.7


def test_capture_linear_ramps():
    # V(t) = a + b t sampled at t_k: the interpolated crossing of 0 mV is exact for a ramp
    a = np.array([-50.0, -10.0, -3.0, -80.0])
    b = np.array([7.0, 3.0, 30.0, 4.0])
    dt = 0.01
    act = np.full(4, -1.0)
    for k in range(3000):
        capture(act, a + b * k * dt, a + b * (k + 1) * dt, k * dt, dt, 0.0)
    assert np.allclose(act, -a / b, rtol=0, atol=1e-10)
    # exact hit of the threshold at t_{k+1}, and no second capture afterwards
    act = np.full(1, -1.0)
    capture(act, np.array([-1.0]), np.array([0.0]), 0.2, 0.01, 0.0)
    assert act[0] == 0.2 + 0.01
    capture(act, np.array([-1.0]), np.array([5.0]), 0.5, 0.01, 0.0)
    assert act[0] == 0.2 + 0.01


def test_initial_above_threshold_has_time_zero():
    w = I.slab_custom(1.0, 1.0, 1.0, 0.5, t_end=0.1)
    w.v_threshold = -90.0
    s = Monodomain(w)
    assert np.all(s.act == 0.0)


@pytest.mark.parametrize("kind", ["2d", "3d"])
def test_manufactured_solution_second_order(kind):
    # Section 3.1.1: the error against the manufactured solution falls as O(h^2) for P1
    if kind == "2d":
        errs = [mms.mms2d(n, 0.01, 1.0)[0] for n in (11, 21, 41)]
    else:
        errs = [mms.mms3d(I.slab_mesh(1.0, 1.0, 0.25, h), 1.0, 1.0, 0.002, 0.2)[0]
                for h in (0.25, 0.125, 0.0625)]
    r = [errs[i] / errs[i + 1] for i in range(2)]
    assert all(3.4 < x < 4.6 for x in r), (errs, r)


def test_small_slab_wave_speed_ratio():
    # plane-wave conduction speed along/across the fibre ~ sqrt(sigma_l / sigma_t) (sanity band)
    w = I.slab_small_ms()
    s = Monodomain(w).run(3200)
    lat = w.mesh.lattice
    ix = (lat[:, 1] == 0) & (lat[:, 2] == 0) & (lat[:, 0] >= 6) & (lat[:, 0] <= 16)
    iy = (lat[:, 0] == 0) & (lat[:, 2] == 0) & (lat[:, 1] >= 4) & (lat[:, 1] <= 7)
    cx = np.polyfit(s.act[ix], 0.5 * lat[ix, 0], 1)[0]
    cy = np.polyfit(s.act[iy], 0.5 * lat[iy, 1], 1)[0]
    assert np.all(s.act >= 0.0)
    assert 0.85 * np.sqrt(0.17 / 0.019) < cx / cy < 1.15 * np.sqrt(0.17 / 0.019)
    assert max(s.iters) < 1000 and all(s.converged)


def test_repolarisation_capture_on_piecewise_linear_ap():
    # V rises from -85 to +20 mV over 2 ms, then falls at 1.05 mV/ms back to -85 mV.
    # Activation (0 mV) at 2*85/105 ms; 90 % repolarisation level -85 + 0.1*105 = -74.5 mV
    # crossed at 2 + 94.5/1.05 = 92 ms; LRT level -70 mV at 2 + 90/1.05 ms.
    from oracle.monodomain import capture_repolarisation

    def v(t):
        return np.where(t <= 2.0, -85.0 + 52.5 * t, 20.0 - 1.05 * (t - 2.0))

    dt = 0.01
    act = np.full(1, -1.0)
    vpeak = np.full(1, -85.0)
    rep90 = np.full(1, -1.0)
    lrt = np.full(1, -1.0)
    for k in range(12000):
        vo, vn = v(np.array([k * dt])), v(np.array([(k + 1) * dt]))
        before = act.copy()
        capture(act, vo, vn, k * dt, dt, 0.0)
        if before[0] < 0 <= act[0]:
            vpeak[:] = vn
        capture_repolarisation(before, vpeak, rep90, lrt, vo, vn, k * dt, dt, -85.0, -70.0)
    assert abs(act[0] - 170.0 / 105.0) < 1e-9
    assert abs(vpeak[0] - 20.0) < 1e-9
    assert abs(rep90[0] - 92.0) < 1e-9
    assert abs(lrt[0] - (2.0 + 90.0 / 1.05)) < 1e-9
