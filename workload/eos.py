"""Equation-of-state inputs.

* Stefan-Boltzmann constant of Sec. 2.3: e_ideal = 3 [2(Nc^2-1) + 7/2 Nc Nf] pi^2/90 T^4.
* A tabulated EOS built from a given speed of sound c_s^2(T) at mu = 0:
  d ln s / d ln T = 1/c_s^2, normalised so that s -> s_SB = 4/3 a T^3 as T -> infinity,
  P(T) = int_0^T s dT', e = T s - P.  The table is an *input* to both the CUDA library and the
  oracle (each interpolates it with its own code); its nodes are uniform in ln e and its
  columns are e, P, c_s^2, T and ln(1/3 - c_s^2), all in fm units.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate, optimize

from .problem import HBARC

NC, NF = 3, 3
A_SB = 3.0 * (2.0 * (NC * NC - 1) + 3.5 * NC * NF) * math.pi ** 2 / 90.0  # = 15.6269...


def cs2_baseline_gev(T_gev):
    """c_s^2(T) = 1/3 - 0.2 exp(-((T - 0.17 GeV)/0.05 GeV)^2) (the 128^3 workload's EOS)."""
    return 1.0 / 3.0 - 0.2 * np.exp(-(((np.asarray(T_gev) - 0.17) / 0.05) ** 2))


def lndelta_baseline_gev(T_gev):
    """ln(1/3 - c_s^2) for the same EOS, exact (no cancellation)."""
    return math.log(0.2) - ((np.asarray(T_gev) - 0.17) / 0.05) ** 2


class TableEOS:
    """Tabulated EOS: arrays e, p, cs2, T, lndelta (fm units), nodes uniform in ln e."""

    def __init__(self, e, p, cs2, T, lndelta):
        self.e = np.ascontiguousarray(e, dtype=np.float64)
        self.p = np.ascontiguousarray(p, dtype=np.float64)
        self.cs2 = np.ascontiguousarray(cs2, dtype=np.float64)
        self.T = np.ascontiguousarray(T, dtype=np.float64)
        self.lndelta = np.ascontiguousarray(lndelta, dtype=np.float64)

    @property
    def n(self):
        return len(self.e)


def build_table(cs2_gev=cs2_baseline_gev, lndelta_gev=lndelta_baseline_gev, n=4096,
                T_lo_gev=1e-3, T_hi_gev=2.0) -> tuple[TableEOS, dict]:
    """Integrate the thermodynamics of a given c_s^2(T) and tabulate it on nodes uniform in ln e.

    Returns (table, dense) where dense holds callables e(T), P(T), s(T) (T in fm^-1) built from
    the high-accuracy ODE solution, for tests of the interpolation.
    """
    T_lo, T_hi = T_lo_gev / HBARC, T_hi_gev / HBARC

    def cs2_fm(T):
        return float(cs2_gev(T * HBARC))

    # g(T_lo) = int_{T_lo}^{inf} (1/cs2 - 3) dT/T ; the integrand vanishes far above 0.17 GeV
    def integrand(lnT):
        T = math.exp(lnT)
        return 1.0 / cs2_fm(T) - 3.0

    pts = [math.log(x / HBARC) for x in (0.05, 0.1, 0.17, 0.25, 0.4)]
    g_lo, _ = integrate.quad(integrand, math.log(T_lo), math.log(5.0 / HBARC), points=pts,
                             epsabs=1e-14, epsrel=1e-13, limit=400)
    lns_lo = math.log(4.0 / 3.0 * A_SB * T_lo ** 3) - g_lo
    n_lo = 1.0 / cs2_fm(T_lo)
    P_lo = T_lo * math.exp(lns_lo) / (n_lo + 1.0)  # power law s ~ T^n below T_lo

    def rhs(x, y):
        T = math.exp(x)
        return [1.0 / cs2_fm(T), T * math.exp(y[0])]

    sol = integrate.solve_ivp(rhs, (math.log(T_lo), math.log(T_hi)), [lns_lo, P_lo], method="DOP853",
                              rtol=1e-13, atol=1e-300, dense_output=True)
    if not sol.success:
        raise RuntimeError("EOS integration failed: " + sol.message)

    def s_of(T):
        return math.exp(sol.sol(math.log(T))[0])

    def P_of(T):
        return float(sol.sol(math.log(T))[1])

    def e_of(T):
        return T * s_of(T) - P_of(T)

    le = np.linspace(math.log(e_of(T_lo)), math.log(e_of(T_hi)), n)
    # invert e(T) at the nodes: a dense log-T grid for the start, then vectorised Newton steps
    # with de/dT = s / c_s^2
    xg = np.linspace(math.log(T_lo), math.log(T_hi), 200001)
    yg = sol.sol(xg)
    Tg = np.exp(xg)
    leg = np.log(Tg * np.exp(yg[0]) - yg[1])
    x = np.interp(le, leg, xg)
    for _ in range(4):
        y = sol.sol(x)
        Tn = np.exp(x)
        s = np.exp(y[0])
        en = Tn * s - y[1]
        c2 = np.array([cs2_fm(t) for t in Tn])
        dedx = Tn * s / c2  # de/dlnT = T de/dT
        x = np.clip(x - (en - np.exp(le)) / dedx, math.log(T_lo), math.log(T_hi))
    T = np.exp(x)
    T[0], T[-1] = T_lo, T_hi
    e = np.array([e_of(t) for t in T])
    p = np.array([P_of(t) for t in T])
    cs2 = np.array([cs2_fm(t) for t in T])
    lnd = np.array([float(lndelta_gev(t * HBARC)) for t in T])
    dense = {"e": e_of, "P": P_of, "s": s_of, "cs2": cs2_fm}
    return TableEOS(e, p, cs2, T, lnd), dense


_CACHE: dict = {}


def baseline_table(n=4096) -> TableEOS:
    """The 128^3 workload's EOS table (cached per process)."""
    if n not in _CACHE:
        _CACHE[n] = build_table(n=n)[0]
    return _CACHE[n]


# ------------------------------------------------------------------ lattice EOS of Sec. 2.3
# Trace anomaly I(T)/T^4 of the Wuppertal-Budapest fit (Sec. 2.3, Eq. traceAnomaly), t = T/0.2 GeV
WB = {"h0": 0.1396, "h1": -0.1800, "h2": 0.0350, "f0": 2.76, "f1": 6.79, "f2": -5.29, "g1": -0.47,
      "g2": 1.04, "alpha": 0.01}


def trace_anomaly(t, p=WB):
    """I/T^4 and d(I/T^4)/dt at t = T / 0.2 GeV (numpy arrays or floats)."""
    t = np.asarray(t, dtype=np.float64)
    den_a = 1.0 + p["alpha"] * t * t
    poly = 1.0 + p["g1"] * t + p["g2"] * t * t
    th = np.tanh(p["f1"] * t + p["f2"])
    F = p["h0"] / den_a + p["f0"] * (th + 1.0) / poly
    dF = (-2.0 * p["alpha"] * t * p["h0"] / den_a ** 2
          + p["f0"] * (p["f1"] * (1.0 - th * th) * poly - (th + 1.0) * (p["g1"] + 2.0 * p["g2"] * t)) / poly ** 2)
    G = np.exp(p["h1"] / t - p["h2"] / (t * t))
    dG = G * (-p["h1"] / (t * t) + 2.0 * p["h2"] / t ** 3)
    return F * G, dF * G + F * dG


def build_lattice_table(n=4096, T_lo_gev=0.02, T_hi_gev=2.0) -> tuple[TableEOS, dict]:
    """The lattice-QCD EOS of Sec. 2.3: P/T^4 = int_0^T (I/T'^4) dT'/T', e = 3P + I, tabulated on
    nodes uniform in ln e.  With s = (e + P)/T and de/dT = 3s + dI/dT, c_s^2 = s/(de/dT) and
    1/3 - c_s^2 = (dI/dT) / (3 de/dT), formed without cancellation.  Returns (table, dense) as
    build_table does (T in fm^-1)."""
    T_lo, T_hi = T_lo_gev / HBARC, T_hi_gev / HBARC
    tsc = HBARC / 0.2  # t = T * tsc for T in fm^-1

    def i_of(T):
        return float(trace_anomaly(T * tsc)[0])

    # y(ln T) = P/T^4 = int_{-inf}^{ln T} i dlnT; below T_lo the integrand is < 1e-3 of i(T_lo)
    y_lo, _ = integrate.quad(lambda x: i_of(math.exp(x)), math.log(1e-3 / HBARC), math.log(T_lo),
                             epsabs=1e-16, epsrel=1e-13, limit=400)
    sol = integrate.solve_ivp(lambda x, y: [i_of(math.exp(x))], (math.log(T_lo), math.log(T_hi)), [y_lo],
                              method="DOP853", rtol=1e-13, atol=1e-300, dense_output=True)
    if not sol.success:
        raise RuntimeError("EOS integration failed: " + sol.message)

    def thermo(T):
        T = np.asarray(T, dtype=np.float64)
        y = sol.sol(np.log(T))[0]
        i, di_dt = trace_anomaly(T * tsc)
        P = T ** 4 * y
        I = T ** 4 * i
        e = 3.0 * P + I
        s = (e + P) / T
        dI = 4.0 * T ** 3 * i + T ** 4 * di_dt * tsc
        de = 3.0 * s + dI
        return e, P, s, s / de, np.log(dI / (3.0 * de))

    le = np.linspace(math.log(float(thermo(T_lo)[0])), math.log(float(thermo(T_hi)[0])), n)
    xg = np.linspace(math.log(T_lo), math.log(T_hi), 200001)
    leg = np.log(thermo(np.exp(xg))[0])
    x = np.interp(le, leg, xg)
    for _ in range(4):  # Newton on e(T) = e_node with de/dlnT = T de/dT = T s / c_s^2
        e, P, s, c2, _ = thermo(np.exp(x))
        x = np.clip(x - (e - np.exp(le)) / (np.exp(x) * s / c2), math.log(T_lo), math.log(T_hi))
    T = np.exp(x)
    T[0], T[-1] = T_lo, T_hi
    e, P, s, c2, lnd = thermo(T)
    dense = {"e": lambda t: float(thermo(t)[0]), "P": lambda t: float(thermo(t)[1]),
             "s": lambda t: float(thermo(t)[2]), "cs2": lambda t: float(thermo(t)[3])}
    return TableEOS(e, P, c2, T, lnd), dense


def lattice_table(n=4096) -> TableEOS:
    """The lattice EOS table (cached per process)."""
    key = ("lattice", n)
    if key not in _CACHE:
        _CACHE[key] = build_lattice_table(n=n)[0]
    return _CACHE[key]


# ------------------------------------------------------------------ zeta/s of Sec. 2.2 (Eq. zetas)
ZETA_PAPER = {"A0": -13.45, "A1": 27.55, "A2": -13.77, "l1": 0.9, "l2": 0.25, "l3": 0.9, "l4": 0.22,
              "s1": 0.025, "s2": 0.13, "s3": 0.0025, "s4": 0.022, "Tc_gev": 0.2}
