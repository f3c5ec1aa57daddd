"""The operator-split monodomain time step (oracle, test infrastructure only).

Per step k -> k+1 (Section 2.2, Eq. 2, Eq. 3 and the definitions after it):
  1. ionic update: u^{k+1} from (V^k, u^k); I_ion = I_ion(V^k, u^{k+1});
  2. b = chi M (Cm V^k - dt I_ion + dt I_stim) - (1 - theta) dt K V^k
     (the printed Eq. 2 carries +(1-theta) dt K V^k; the definition of b printed after Eq. 3,
     and the theta-method itself, give the minus sign used here);
  3. solve A V^{k+1} = b, A = chi Cm M + theta dt K, by Jacobi-PCG (Algorithm 1) from the
     extrapolated guess 2 V^k - V^{k-1} (end of Section 2.2), with V^{-1} = V^0;
  4. activation times (Section 2.1): the first time V becomes >= threshold (0 mV), linearly
     interpolated inside the step: t_k + dt (thr - V^k) / (V^{k+1} - V^k); a node starting at
     or above the threshold has time 0; never activated -> -1.
Stimuli (Section 2.1): stimulus s adds its intensity to I_stim on its nodes for the steps
k with k0 <= k < k0 + nk, k0 = round(start/dt), nk = round(duration/dt); I_stim is taken at t_k.
"""
import numpy as np

from . import fem, ionic, tp06
from .pcg import pcg


def rhs(M, K, V, i_ion, i_stim, chi, cm, theta, dt):
    """b of Eq. 3: chi M (Cm V - dt I_ion + dt I_stim) - (1 - theta) dt K V."""
    return chi * (M @ (cm * V - dt * i_ion + dt * i_stim)) - (1.0 - theta) * dt * (K @ V)


def capture(act, v_old, v_new, t_k, dt, thr):
    """Record first upward crossings of thr between t_k and t_k + dt (in place)."""
    m = (act < 0.0) & (v_old < thr) & (v_new >= thr)
    act[m] = t_k + dt * (thr - v_old[m]) / (v_new[m] - v_old[m])
    return act


def capture_repolarisation(act, vpeak, rep90, lrt, v_old, v_new, t_k, dt, v_rest, lrt_thr):
    """After activation: track the peak, and record the first downward crossings of the 90 %
    repolarisation level v_rest + 0.1 (peak - v_rest) and of the LRT threshold (Section 2.1: back
    below -70 mV with a negative time derivative), linearly interpolated inside the step.
    Nodes activated in this very step only get their peak set."""
    m = act >= 0.0
    vpeak[m] = np.maximum(vpeak[m], v_new[m])
    t90 = v_rest + 0.1 * (vpeak - v_rest)
    c90 = m & (rep90 < 0.0) & (v_old >= t90) & (v_new < t90)
    rep90[c90] = t_k + dt * (v_old[c90] - t90[c90]) / (v_old[c90] - v_new[c90])
    cl = m & (lrt < 0.0) & (v_old >= lrt_thr) & (v_new < lrt_thr)
    lrt[cl] = t_k + dt * (v_old[cl] - lrt_thr) / (v_old[cl] - v_new[cl])


def stimulus_current(stimuli, k, dt, n):
    """Nodal I_stim (uA/mm^2) at step k."""
    i_stim = np.zeros(n)
    for s in stimuli:
        k0 = int(round(s.start / dt))
        nk = int(round(s.duration / dt))
        if k0 <= k < k0 + nk:
            np.add.at(i_stim, np.asarray(s.nodes, dtype=np.int64), s.intensity)
    return i_stim


class Monodomain:
    """FP64 monodomain simulation of one workload (paper inputs: mesh, chi, Cm, sigma, theta,
    dt, ionic model, stimuli, PCG tolerances)."""

    def __init__(self, w, M=None, K=None):
        self.w = w
        mesh = w.mesh
        if M is None or K is None:
            sl = np.atleast_1d(np.asarray(w.sigma_l, dtype=np.float64))
            st = np.atleast_1d(np.asarray(w.sigma_t, dtype=np.float64))
            if sl.size > 1:
                sl, st = sl[mesh.region], st[mesh.region]
            M, K = fem.mass_stiffness(mesh.xyz, mesh.tets, mesh.fibres, sl, st)
        self.M, self.K = M, K
        self.A = fem.system_matrix(M, K, w.chi, w.cm, w.theta, w.dt)
        self.diag = self.A.diagonal()
        n = mesh.n_nodes
        if w.model == "ms":
            self.V, h = ionic.ms_rest(n, w.ms)
            self.state = [h]
        elif w.model == "tp06":
            self.V, u = tp06.rest(n)
            self.state = [u[:, j].copy() for j in range(tp06.N_STATES)]
        else:
            raise ValueError(f"model {w.model!r} not available in the oracle")
        self.V_prev = self.V.copy()
        self.act = np.full(n, -1.0)
        self.act[self.V >= w.v_threshold] = 0.0
        self.v_rest = float(self.V[0])
        self.vpeak = self.V.copy()
        self.rep90 = np.full(n, -1.0)
        self.lrt = np.full(n, -1.0)
        self.lrt_thr = -70.0
        self.k = 0
        self.iters = []
        self.converged = []

    def ionic(self):
        w = self.w
        if w.model == "ms":
            h, i_ion = ionic.ms_step(self.V, self.state[0], w.dt, w.cm, w.ms)
            return [h], i_ion
        if w.model == "tp06":
            # TP06 currents are in pA/pF; times Cm (uF/mm^2) they are uA/mm^2
            u = np.stack(self.state, axis=1)
            un, i_pa = tp06.step(self.V, u, w.dt, w.tp06_cell)
            return [un[:, j].copy() for j in range(tp06.N_STATES)], w.cm * i_pa
        raise ValueError(w.model)

    def step(self):
        w = self.w
        t_k = self.k * w.dt
        self.state, i_ion = self.ionic()
        i_stim = stimulus_current(w.stimuli, self.k, w.dt, self.V.size)
        b = rhs(self.M, self.K, self.V, i_ion, i_stim, w.chi, w.cm, w.theta, w.dt)
        x0 = 2.0 * self.V - self.V_prev
        v_new, it, _, ok = pcg(self.A, b, x0, self.diag, w.atol, w.rtol, w.max_iter)
        was_active = self.act >= 0.0
        capture(self.act, self.V, v_new, t_k, w.dt, w.v_threshold)
        newly = (~was_active) & (self.act >= 0.0)
        self.vpeak[newly] = v_new[newly]
        act_before = np.where(was_active, self.act, -1.0)
        capture_repolarisation(act_before, self.vpeak, self.rep90, self.lrt, self.V, v_new, t_k,
                               w.dt, self.v_rest, self.lrt_thr)
        self.V_prev, self.V = self.V, v_new
        self.k += 1
        self.iters.append(it)
        self.converged.append(ok)

    def apd90(self):
        return np.where((self.rep90 >= 0.0) & (self.act >= 0.0), self.rep90 - self.act, -1.0)

    def run(self, n_steps):
        for _ in range(n_steps):
            self.step()
        return self
