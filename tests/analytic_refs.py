"""Independent reference solutions used to pin the oracle (derived from the paper's equations).

* Relativistic Riemann problem for a conformal ideal fluid (P = e/3), both sides at rest
  (Sec. 5.1's shock tube): a left rarefaction and a right shock.  Along the rarefaction the
  Riemann invariant artanh(v) + (c_s/(1+c_s^2)) ln e is constant (c_s^2 = 1/3 gives sqrt(3)/4);
  inside the fan (v - c_s)/(1 - v c_s) = x/t.  Across the shock into the resting right state the
  relative velocity satisfies v^2 = (P* - P_R)(e* - e_R)/((e_R + P*)(e* + P_R)) (Taub adiabat).
* Bjorken ODEs of Secs. 5.4-5.5, written from Eqs. (evolutionEd0p1)-(evolutionpi).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate, optimize

CS = 1.0 / math.sqrt(3.0)
K_RAR = CS / (1.0 + CS * CS)  # sqrt(3)/4


class SodSolution:
    def __init__(self, eL, eR):
        self.eL, self.eR = eL, eR
        PR = eR / 3.0

        def v_rar(e):
            return math.tanh(K_RAR * math.log(eL / e))

        def v_shock(e):
            P = e / 3.0
            return math.sqrt((P - PR) * (e - eR) / ((eR + P) * (e + PR)))

        es = optimize.brentq(lambda e: v_rar(e) - v_shock(e), eR * (1 + 1e-12), eL * (1 - 1e-12),
                             xtol=1e-16, rtol=1e-15)
        self.es = es
        self.vs = v_rar(es)
        Ps = es / 3.0
        g2 = 1.0 / (1.0 - self.vs ** 2)
        Ttt = (es + Ps) * g2 - Ps
        Ttx = (es + Ps) * g2 * self.vs
        Txx = (es + Ps) * g2 * self.vs ** 2 + Ps
        self.Vshock = Ttx / (Ttt - eR)
        # second jump condition, kept for the self-check: [T^xx] = V [T^tx]
        self.rh_residual = (Txx - PR) - self.Vshock * Ttx
        self.head = -CS
        self.tail = (self.vs - CS) / (1.0 - self.vs * CS)

    def __call__(self, x, t):
        xi = np.asarray(x, dtype=np.float64) / t
        e = np.empty_like(xi)
        v = np.empty_like(xi)
        left = xi <= self.head
        e[left], v[left] = self.eL, 0.0
        fan = (xi > self.head) & (xi <= self.tail)
        vf = (xi[fan] + CS) / (1.0 + xi[fan] * CS)
        v[fan] = vf
        e[fan] = self.eL * np.exp(-np.arctanh(vf) / K_RAR)
        plat = (xi > self.tail) & (xi <= self.Vshock)
        e[plat], v[plat] = self.es, self.vs
        right = xi > self.Vshock
        e[right], v[right] = self.eR, 0.0
        return e, v


def bjorken_conformal(tau0, e0, pi0, taus, eta_over_s, a_sb, tau_pipi=True):
    """Eqs. (evolutionEd0p1)-(evolutionpi1): de/dtau = -(e+P-pi)/tau,
    tau_pi dpi/dtau + pi = 4/3 eta/tau - (tau_pipi/3 + delta_pipi) pi/tau, P = e/3."""
    def rhs(t, y):
        e, pi = y
        P = e / 3.0
        T = (e / a_sb) ** 0.25
        eta = eta_over_s * (e + P) / T
        tp = 5.0 * eta_over_s / T
        tpp = 10.0 / 7.0 * tp if tau_pipi else 0.0
        return [-(e + P - pi) / t, (4.0 / 3.0 * eta / t - (tpp / 3.0 + 4.0 / 3.0 * tp) * pi / t - pi) / tp]
    r = integrate.solve_ivp(rhs, (tau0, taus[-1]), [e0, pi0], method="DOP853", rtol=1e-13, atol=1e-14,
                            t_eval=taus)
    return r.y
