"""Gubser flow (conformal, boost invariant, radially expanding), used as an initial state and as
the reference solution of the viscous Gubser test (Secs. 5.6-5.7).

In the Weyl-rescaled de Sitter frame the fluid is at rest and the Israel-Stewart equations of
Sec. 2.2 with tau_pipi = 0 and delta_pipi = 4/3 tau_pi reduce to two ODEs in de Sitter time rho
(derived here from the paper's equations; expansion rate 2 tanh rho, shear eigenvalues
-tanh(rho)/3 (twice) and 2 tanh(rho)/3 along eta):

    dT^/drho = T^ (-2/3 + pibar/3) tanh rho
    dpibar/drho = 4/15 tanh rho - 4/3 pibar^2 tanh rho - pibar / tau^_pi,  tau^_pi = 5 (eta/s)/T^

with pibar = pi^{eta eta} tau^2 / (e + P) (the eta-eta component in the local rest frame over
the enthalpy).  With eta/s = 0 this gives the closed form T^ = T^_0 cosh(rho)^(-2/3) of Sec. 5.6.
The coordinate map is sinh rho = -(1 - q^2 tau^2 + q^2 r^2)/(2 q tau) and the flow is
u^r = sinh kappa, kappa = artanh(2 q^2 tau r / (1 + q^2 tau^2 + q^2 r^2)).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate


class GubserSolution:
    def __init__(self, eta_over_s=0.2, T0hat=1.2, q=1.0, rho_range=(-8.0, 8.0)):
        self.eta_over_s = eta_over_s
        self.T0hat = T0hat
        self.q = q

        def rhs(rho, y):
            That, pibar = y
            th = math.tanh(rho)
            dT = That * (-2.0 / 3.0 + pibar / 3.0) * th
            if eta_over_s > 0:
                taupi = 5.0 * eta_over_s / That
                dp = 4.0 / 15.0 * th - 4.0 / 3.0 * pibar * pibar * th - pibar / taupi
            else:
                dp = 0.0
            return [dT, dp]

        y0 = [T0hat, 0.0]  # starts at its Navier-Stokes value pibar = 0 at rho = 0
        self._fwd = integrate.solve_ivp(rhs, (0.0, rho_range[1]), y0, method="DOP853", rtol=1e-12,
                                        atol=1e-14, dense_output=True)
        self._bwd = integrate.solve_ivp(rhs, (0.0, rho_range[0]), y0, method="DOP853", rtol=1e-12,
                                        atol=1e-14, dense_output=True)

    def that_pibar(self, rho):
        rho = np.asarray(rho, dtype=np.float64)
        out = np.empty((2,) + rho.shape)
        pos = rho >= 0
        if np.any(pos):
            out[:, pos] = self._fwd.sol(rho[pos])
        if np.any(~pos):
            out[:, ~pos] = self._bwd.sol(rho[~pos])
        return out[0], out[1]

    def rho_kappa(self, tau, r):
        q = self.q
        rho = np.arcsinh(-(1.0 - q * q * tau * tau + q * q * r * r) / (2.0 * q * tau))
        kappa = np.arctanh(2.0 * q * q * tau * r / (1.0 + q * q * tau * tau + q * q * r * r))
        return rho, kappa

    def state(self, tau, x, y, a_sb):
        """Primaries at proper time tau on points (x, y): e, u^x, u^y and pi^{mu nu} (10 rows)."""
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        r = np.sqrt(x * x + y * y)
        rho, kappa = self.rho_kappa(tau, r)
        That, pibar = self.that_pibar(rho)
        T = That / tau
        e = a_sb * T ** 4
        sk = np.sinh(kappa)
        with np.errstate(invalid="ignore", divide="ignore"):
            cx = np.where(r > 0, x / np.where(r > 0, r, 1.0), 0.0)
            cy = np.where(r > 0, y / np.where(r > 0, r, 1.0), 0.0)
        ux, uy = cx * sk, cy * sk
        ut = np.sqrt(1.0 + ux * ux + uy * uy)
        # pi^{mu nu} = pi_eta [3/2 e_eta e_eta + 1/2 Delta^{mu nu}], pi_eta = pibar (e + P)
        pe = pibar * (4.0 / 3.0) * e
        pi = np.zeros((10,) + e.shape)
        pi[0] = -0.5 * pe * (ux * ux + uy * uy)      # tt
        pi[1] = -0.5 * pe * ut * ux                  # tx
        pi[2] = -0.5 * pe * ut * uy                  # ty
        pi[4] = -0.5 * pe * (1.0 + ux * ux)          # xx
        pi[5] = -0.5 * pe * ux * uy                  # xy
        pi[7] = -0.5 * pe * (1.0 + uy * uy)          # yy
        pi[9] = pe / tau ** 2                        # eta eta
        return {"e": e, "ux": ux, "uy": uy, "ut": ut, "pi": pi, "T": T}
