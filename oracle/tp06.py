"""ten Tusscher-Panfilov 2006 human ventricular model (oracle, test infrastructure only).

The paper runs its volume-mesh benchmarks with this model (Section 2.2, Section 3.3) but does not
print it; the equations below restate the model's primary publication (ten Tusscher & Panfilov,
Am J Physiol Heart Circ Physiol 291:H1088, 2006) in the rapid-buffering differential form.
Units: mV, ms, mM, currents in pA/pF.  State vector u (18 entries, V kept apart):
    0 Ki  1 Nai  2 Cai  3 CaSR  4 CaSS  5 Rbar  6 xr1  7 xr2  8 xs  9 m  10 h  11 j
    12 d  13 f  14 f2  15 fCass  16 s  17 r
Cell types: 0 endocardial, 1 mid-myocardial, 2 epicardial.

Time step (operator splitting as Eq. 2 and the paragraph after it read):
  * every rate is evaluated at (V^k, u^k);
  * gates 6..17 advance by Rush-Larsen, u_inf + (u - u_inf) exp(-dt/tau);
  * concentrations 0..4 and Rbar advance by forward Euler;
  * the current returned is I_ion(V^k, u^{k+1}).
The stimulus current is not added to Ki (in tissue it enters through the PDE source).

The f2 gate's time constant is taken in the form
    tau_f2 = 562 exp(-(V+27)^2/240) + 31/(1 + exp((25-V)/10)) + 80/(1 + exp((V+30)/10)),
the one under which the publication's initial state (REST_U, REST_V) is the end-diastolic
state of the epicardial cell paced at a 550 ms cycle: every gate and V return to their
printed values after a beat.  The variant 600 exp(-(V+25)^2/170) + 31/(...) + 16/(...) leaves
f2 at 0.9995 at the end of every diastole (tau ~16 ms at rest) and cannot reproduce the
printed 0.9755 at any cycle length.
"""
import numpy as np

N_STATES = 18
KI, NAI, CAI, CASR, CASS, RBAR, XR1, XR2, XS, M, H, J, D, F, F2, FCASS, S, R = range(18)
GATES = [XR1, XR2, XS, M, H, J, D, F, F2, FCASS, S, R]

# physical constants and cell geometry
R_GAS, T_K, FARADAY = 8314.472, 310.0, 96485.3415
RTF = R_GAS * T_K / FARADAY
CAP, VC, VSR, VSS = 0.185, 0.016404, 0.001094, 0.00005468
KO, NAO, CAO = 5.4, 140.0, 2.0
# conductances and transport
GNA, GK1, GKR, GPK, GPCA, GBNA, GBCA, GCAL = 14.838, 5.405, 0.153, 0.0146, 0.1238, 0.00029, 0.000592, 3.98e-5
GKS = {0: 0.392, 1: 0.098, 2: 0.392}
GTO = {0: 0.073, 1: 0.294, 2: 0.294}
P_KNA, KPCA = 0.03, 0.0005
P_NAK, KM_K, KM_NA = 2.724, 1.0, 40.0
K_NACA, KM_NAI, KM_CA, K_SAT, GAMMA, ALPHA_NACA = 1000.0, 87.5, 1.38, 0.1, 0.35, 2.5
# calcium handling
V_MAXUP, K_UP, V_REL, V_LEAK, V_XFER = 0.006375, 0.00025, 0.102, 0.00036, 0.0038
K1P, K2P, K3, K4, EC, MAXSR, MINSR = 0.15, 0.045, 0.06, 0.005, 1.5, 2.5, 1.0
BUFC, KBUFC, BUFSR, KBUFSR, BUFSS, KBUFSS = 0.2, 0.001, 10.0, 0.3, 0.4, 0.00025

REST_V = -85.23
REST_U = np.array([136.89, 8.604, 0.000126, 3.64, 0.00036, 0.9073, 0.00621, 0.4712, 0.0095,
                   0.00172, 0.7444, 0.7045, 3.373e-5, 0.7888, 0.9755, 0.9953, 0.999998, 2.42e-8])


def rest(n):
    """Resting V and the (n, 18) state array."""
    return np.full(n, REST_V), np.tile(REST_U, (n, 1))


def currents(V, u, cell):
    """All membrane currents (pA/pF) at (V, u); returns a dict."""
    ki, nai, cai, cass = u[:, KI], u[:, NAI], u[:, CAI], u[:, CASS]
    ek = RTF * np.log(KO / ki)
    ena = RTF * np.log(NAO / nai)
    eks = RTF * np.log((KO + P_KNA * NAO) / (ki + P_KNA * nai))
    eca = 0.5 * RTF * np.log(CAO / cai)
    a_k1 = 0.1 / (1.0 + np.exp(0.06 * (V - ek - 200.0)))
    b_k1 = (3.0 * np.exp(0.0002 * (V - ek + 100.0)) + np.exp(0.1 * (V - ek - 10.0))) / \
        (1.0 + np.exp(-0.5 * (V - ek)))
    c = {}
    c["ik1"] = GK1 * np.sqrt(KO / 5.4) * (a_k1 / (a_k1 + b_k1)) * (V - ek)
    c["ito"] = GTO[cell] * u[:, R] * u[:, S] * (V - ek)
    c["ikr"] = GKR * np.sqrt(KO / 5.4) * u[:, XR1] * u[:, XR2] * (V - ek)
    c["iks"] = GKS[cell] * u[:, XS] ** 2 * (V - eks)
    c["ina"] = GNA * u[:, M] ** 3 * u[:, H] * u[:, J] * (V - ena)
    c["ibna"] = GBNA * (V - ena)
    # L-type: GCaL d f f2 fCass 4 (V-15) F^2/(RT) (0.25 CaSS e^x - Cao)/(e^x - 1), x = 2(V-15)F/RT
    x = 2.0 * (V - 15.0) / RTF
    ex = np.exp(x)
    with np.errstate(invalid="ignore", divide="ignore"):
        ghk = np.where(x != 0.0, 4.0 * (V - 15.0) * FARADAY / RTF * (0.25 * cass * ex - CAO) / np.expm1(x),
                       2.0 * FARADAY * (0.25 * cass - CAO))
    c["ical"] = GCAL * u[:, D] * u[:, F] * u[:, F2] * u[:, FCASS] * ghk
    c["ibca"] = GBCA * (V - eca)
    vf = V / RTF
    c["inak"] = P_NAK * KO / (KO + KM_K) * nai / (nai + KM_NA) / \
        (1.0 + 0.1245 * np.exp(-0.1 * vf) + 0.0353 * np.exp(-vf))
    c["inaca"] = K_NACA * (np.exp(GAMMA * vf) * nai ** 3 * CAO - np.exp((GAMMA - 1.0) * vf) * NAO ** 3 * cai * ALPHA_NACA) / \
        ((KM_NAI ** 3 + NAO ** 3) * (KM_CA + CAO) * (1.0 + K_SAT * np.exp((GAMMA - 1.0) * vf)))
    c["ipca"] = GPCA * cai / (KPCA + cai)
    c["ipk"] = GPK * (V - ek) / (1.0 + np.exp((25.0 - V) / 5.98))
    return c


def total_current(c):
    return (c["ik1"] + c["ito"] + c["ikr"] + c["iks"] + c["ina"] + c["ibna"] + c["ical"] +
            c["ibca"] + c["inak"] + c["inaca"] + c["ipca"] + c["ipk"])


def gate_inf_tau(V, u, cell):
    """(inf, tau) of the 12 gates, in the order of GATES."""
    inf, tau = {}, {}
    am = 1.0 / (1.0 + np.exp((-60.0 - V) / 5.0))
    bm = 0.1 / (1.0 + np.exp((V + 35.0) / 5.0)) + 0.1 / (1.0 + np.exp((V - 50.0) / 200.0))
    inf[M] = 1.0 / (1.0 + np.exp((-56.86 - V) / 9.03)) ** 2
    tau[M] = am * bm
    hinf = 1.0 / (1.0 + np.exp((V + 71.55) / 7.43)) ** 2
    lo = V < -40.0
    ah = np.where(lo, 0.057 * np.exp(-(V + 80.0) / 6.8), 0.0)
    bh = np.where(lo, 2.7 * np.exp(0.079 * V) + 3.1e5 * np.exp(0.3485 * V),
                  0.77 / (0.13 * (1.0 + np.exp(-(V + 10.66) / 11.1))))
    inf[H], tau[H] = hinf, 1.0 / (ah + bh)
    aj = np.where(lo, (-2.5428e4 * np.exp(0.2444 * V) - 6.948e-6 * np.exp(-0.04391 * V)) * (V + 37.78) /
                  (1.0 + np.exp(0.311 * (V + 79.23))), 0.0)
    bj = np.where(lo, 0.02424 * np.exp(-0.01052 * V) / (1.0 + np.exp(-0.1378 * (V + 40.14))),
                  0.6 * np.exp(0.057 * V) / (1.0 + np.exp(-0.1 * (V + 32.0))))
    inf[J], tau[J] = hinf, 1.0 / (aj + bj)
    inf[XR1] = 1.0 / (1.0 + np.exp((-26.0 - V) / 7.0))
    tau[XR1] = 450.0 / (1.0 + np.exp((-45.0 - V) / 10.0)) * 6.0 / (1.0 + np.exp((V + 30.0) / 11.5))
    inf[XR2] = 1.0 / (1.0 + np.exp((V + 88.0) / 24.0))
    tau[XR2] = 3.0 / (1.0 + np.exp((-60.0 - V) / 20.0)) * 1.12 / (1.0 + np.exp((V - 60.0) / 20.0))
    inf[XS] = 1.0 / (1.0 + np.exp((-5.0 - V) / 14.0))
    tau[XS] = 1400.0 / np.sqrt(1.0 + np.exp((5.0 - V) / 6.0)) / (1.0 + np.exp((V - 35.0) / 15.0)) + 80.0
    inf[R] = 1.0 / (1.0 + np.exp((20.0 - V) / 6.0))
    tau[R] = 9.5 * np.exp(-(V + 40.0) ** 2 / 1800.0) + 0.8
    if cell == 0:
        inf[S] = 1.0 / (1.0 + np.exp((V + 28.0) / 5.0))
        tau[S] = 1000.0 * np.exp(-(V + 67.0) ** 2 / 1000.0) + 8.0
    else:
        inf[S] = 1.0 / (1.0 + np.exp((V + 20.0) / 5.0))
        tau[S] = 85.0 * np.exp(-(V + 45.0) ** 2 / 320.0) + 5.0 / (1.0 + np.exp((V - 20.0) / 5.0)) + 3.0
    inf[D] = 1.0 / (1.0 + np.exp((-8.0 - V) / 7.5))
    tau[D] = (1.4 / (1.0 + np.exp((-35.0 - V) / 13.0)) + 0.25) * 1.4 / (1.0 + np.exp((V + 5.0) / 5.0)) + \
        1.0 / (1.0 + np.exp((50.0 - V) / 20.0))
    inf[F] = 1.0 / (1.0 + np.exp((V + 20.0) / 7.0))
    tau[F] = 1102.5 * np.exp(-(V + 27.0) ** 2 / 225.0) + 200.0 / (1.0 + np.exp((13.0 - V) / 10.0)) + \
        180.0 / (1.0 + np.exp((V + 30.0) / 10.0)) + 20.0
    inf[F2] = 0.67 / (1.0 + np.exp((V + 35.0) / 7.0)) + 0.33
    tau[F2] = 562.0 * np.exp(-(V + 27.0) ** 2 / 240.0) + 31.0 / (1.0 + np.exp((25.0 - V) / 10.0)) + \
        80.0 / (1.0 + np.exp((V + 30.0) / 10.0))
    cs = (u[:, CASS] / 0.05) ** 2
    inf[FCASS] = 0.6 / (1.0 + cs) + 0.4
    tau[FCASS] = 80.0 / (1.0 + cs) + 2.0
    return inf, tau


def concentration_rates(V, u, c):
    """d/dt of Ki, Nai, Cai, CaSR, CaSS, Rbar at (V, u) with currents c (rapid buffering)."""
    cai, casr, cass, rbar = u[:, CAI], u[:, CASR], u[:, CASS], u[:, RBAR]
    kcasr = MAXSR - (MAXSR - MINSR) / (1.0 + (EC / casr) ** 2)
    k1 = K1P / kcasr
    k2 = K2P * kcasr
    o = k1 * cass ** 2 * rbar / (K3 + k1 * cass ** 2)
    i_rel = V_REL * o * (casr - cass)
    i_leak = V_LEAK * (casr - cai)
    i_up = V_MAXUP / (1.0 + K_UP ** 2 / cai ** 2)
    i_xfer = V_XFER * (cass - cai)
    f_i = 1.0 / (1.0 + BUFC * KBUFC / (cai + KBUFC) ** 2)
    f_sr = 1.0 / (1.0 + BUFSR * KBUFSR / (casr + KBUFSR) ** 2)
    f_ss = 1.0 / (1.0 + BUFSS * KBUFSS / (cass + KBUFSS) ** 2)
    d = np.empty((u.shape[0], 6))
    d[:, KI] = -(c["ik1"] + c["ito"] + c["ikr"] + c["iks"] + c["ipk"] - 2.0 * c["inak"]) * CAP / (VC * FARADAY)
    d[:, NAI] = -(c["ina"] + c["ibna"] + 3.0 * c["inak"] + 3.0 * c["inaca"]) * CAP / (VC * FARADAY)
    d[:, CAI] = f_i * ((i_leak - i_up) * VSR / VC + i_xfer -
                       (c["ibca"] + c["ipca"] - 2.0 * c["inaca"]) * CAP / (2.0 * VC * FARADAY))
    d[:, CASR] = f_sr * (i_up - (i_rel + i_leak))
    d[:, CASS] = f_ss * (-c["ical"] * CAP / (2.0 * VSS * FARADAY) + i_rel * VSR / VSS - i_xfer * VC / VSS)
    d[:, RBAR] = -k2 * cass * rbar + K4 * (1.0 - rbar)
    return d


def derivatives(V, u, cell):
    """Continuous right-hand side (dV/dt, du/dt) of the single cell without stimulus."""
    c = currents(V, u, cell)
    du = np.empty_like(u)
    du[:, :6] = concentration_rates(V, u, c)
    inf, tau = gate_inf_tau(V, u, cell)
    for g in GATES:
        du[:, g] = (inf[g] - u[:, g]) / tau[g]
    return -total_current(c), du


def step(V, u, dt, cell):
    """One split step: Rush-Larsen gates and forward-Euler concentrations, both from the rates
    at (V^k, u^k); returns (u^{k+1}, I_ion(V^k, u^{k+1})) with I_ion in pA/pF."""
    c = currents(V, u, cell)
    un = u.copy()
    un[:, :6] = u[:, :6] + dt * concentration_rates(V, u, c)
    inf, tau = gate_inf_tau(V, u, cell)
    for g in GATES:
        un[:, g] = inf[g] + (u[:, g] - inf[g]) * np.exp(-dt / tau[g])
    return un, total_current(currents(V, un, cell))


def charge_invariant(V, u):
    """V - (F/Cap)(Vc (Nai + Ki + 2 Cai_tot) + 2 Vss CaSS_tot + 2 Vsr CaSR_tot): constant along any
    solution of the single-cell equations without stimulus (total charge balance)."""
    cai_t = u[:, CAI] + BUFC * u[:, CAI] / (u[:, CAI] + KBUFC)
    casr_t = u[:, CASR] + BUFSR * u[:, CASR] / (u[:, CASR] + KBUFSR)
    cass_t = u[:, CASS] + BUFSS * u[:, CASS] / (u[:, CASS] + KBUFSS)
    return V - FARADAY / CAP * (VC * (u[:, NAI] + u[:, KI] + 2.0 * cai_t) + 2.0 * VSS * cass_t +
                                2.0 * VSR * casr_t)
