"""Pins of the oracle's ten Tusscher-Panfilov 2006 model.

The paper names the model (Section 2.2) but prints none of it, so the equations are pinned by
(1) an exact identity of the model: the total membrane charge balance, which ties every current
to its ionic fluxes; (2) the Rush-Larsen closed form of the gates at a frozen potential;
(3) first-order convergence of the split step to an accurate ODE solution; and (4) published
action-potential features of the model (resting potential, overshoot, APD90 ordering and
range of the three cell types) as bands.  The individual rate constants are otherwise
unpinned against the paper."""
import numpy as np
import pytest
from scipy.integrate import solve_ivp

from oracle import tp06 as T


def _ode(cell, v0=-20.0, t_end=500.0):
    V0, u0 = T.rest(1)

    def rhs(t, y):
        dv, du = T.derivatives(np.array([y[0]]), y[1:].reshape(1, 18), cell)
        return np.concatenate([dv, du[0]])

    y0 = np.concatenate([[v0], u0[0]])
    return solve_ivp(rhs, (0.0, t_end), y0, method="LSODA", rtol=1e-11, atol=1e-13,
                     dense_output=True, max_step=0.5)


@pytest.fixture(scope="module")
def aps():
    return {cell: _ode(cell) for cell in (0, 1, 2)}


def _apd90(t, v, v_rest):
    peak = v.max()
    after = (t > t[np.argmax(v)]) & (v < peak - 0.9 * (peak - v_rest))
    return t[np.argmax(after)]


def test_charge_balance_is_conserved(aps):
    # dV/dt = -I_ion and the Na, K, Ca balances carry the same charge: the invariant is exact
    for cell, sol in aps.items():
        ts = np.linspace(0.0, 500.0, 5001)
        Y = sol.sol(ts)
        inv = T.charge_invariant(Y[0], Y[1:].T)
        assert np.abs(inv - inv[0]).max() < 1e-5, cell
        assert Y[0].max() - Y[0].min() > 100.0     # a full action potential was traversed


def test_rest_is_near_equilibrium():
    V, u = T.rest(3)
    i = T.total_current(T.currents(V, u, 2))
    assert np.all(np.abs(i) < 0.01)
    for cell in (0, 1, 2):
        dv, du = T.derivatives(V[:1], u[:1], cell)
        assert abs(dv[0]) < 0.01


def test_action_potential_features(aps):
    ts = np.linspace(0.0, 500.0, 50001)
    apd = {}
    for cell, sol in aps.items():
        v = sol.sol(ts)[0]
        assert 25.0 < v.max() < 45.0
        assert -87.0 < v[-1] < -83.0
        apd[cell] = _apd90(ts, v, T.REST_V)
    assert 250.0 < apd[0] < 330.0 and 250.0 < apd[2] < 330.0
    assert 340.0 < apd[1] < 430.0
    assert apd[1] > apd[2] + 40.0          # mid-myocardial cells: smaller I_Ks, longer AP


def test_rush_larsen_is_exact_for_frozen_voltage():
    # at a frozen V the gate ODE is linear; Rush-Larsen steps reproduce exp(-t/tau) exactly
    V = np.array([-30.0])
    u0 = T.rest(1)[1]
    inf, tau = T.gate_inf_tau(V, u0, 2)
    u = u0.copy()
    dt, n = 0.02, 250
    for _ in range(n):
        un, _ = T.step(V, u, dt, 2)
        # keep the concentrations frozen so that fCass keeps its rate
        un[:, :6] = u0[:, :6]
        u = un
    for g in (T.M, T.H, T.XR1, T.D, T.F, T.S, T.R):
        ref = inf[g] + (u0[:, g] - inf[g]) * np.exp(-n * dt / tau[g])
        assert np.allclose(u[:, g], ref, rtol=1e-12, atol=1e-15), g


def test_split_step_converges_first_order(aps):
    sol = aps[2]
    errs = []
    for dt in (0.02, 0.01, 0.005):
        V, u = T.rest(1)
        V[:] = -20.0
        t_stop = 150.0
        for _ in range(int(round(t_stop / dt))):
            un, i = T.step(V, u, dt, 2)
            V = V - dt * i
            u = un
        errs.append(abs(V[0] - sol.sol(t_stop)[0]))
    assert errs[0] < 1.0
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 1.5 < r1 < 2.6 and 1.5 < r2 < 2.6, errs
