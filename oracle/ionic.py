"""Ionic models of the oracle (test infrastructure only).

Operator splitting (Section 2.2, Eq. 2 and the paragraph after it): the state variables are
advanced first, then I_ion is evaluated at (V^k, u^{k+1}).  Gating variables use the
Rush-Larsen step u^{k+1} = u_inf + (u^k - u_inf) exp(-dt/tau), which is exact for a gate with
constant u_inf and tau over the step; other states use forward Euler as Eq. 2 states.

Mitchell-Schaeffer (Mitchell & Schaeffer 2003) is named by the workloads but not written out in
the paper, and its variable v is dimensionless; the reading taken maps it to mV with the
potential range [v_min, v_max] of the tissue model:
    v = (V - v_min) / (v_max - v_min)
    J_in = h v^2 (1 - v) / tau_in,   J_out = -v / tau_out
    I_ion = -Cm (v_max - v_min) (J_in + J_out)            [uA/mm^2 with Cm in uF/mm^2]
    gate: v <  v_gate -> h_inf = 1, tau = tau_open
          v >= v_gate -> h_inf = 0, tau = tau_close
so that Cm dV/dt = -I_ion reproduces dv/dt = J_in + J_out of the original model.
Resting state: V = v_min, h = 1.
"""
import numpy as np


def ms_rest(n, p):
    """Resting membrane potential and gate of the Mitchell-Schaeffer model."""
    return np.full(n, p.v_min), np.ones(n)


def ms_step(V, h, dt, cm, p):
    """One Rush-Larsen step of the gate, then I_ion(V^k, h^{k+1}).  Returns (h_new, I_ion)."""
    v = (V - p.v_min) / (p.v_max - p.v_min)
    closing = v >= p.v_gate
    h_inf = np.where(closing, 0.0, 1.0)
    tau = np.where(closing, p.tau_close, p.tau_open)
    h_new = h_inf + (h - h_inf) * np.exp(-dt / tau)
    j_in = h_new * v * v * (1.0 - v) / p.tau_in
    j_out = -v / p.tau_out
    i_ion = -cm * (p.v_max - p.v_min) * (j_in + j_out)
    return h_new, i_ion
