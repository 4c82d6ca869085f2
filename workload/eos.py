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
