"""Problem definitions and seeded initial states (inputs only; fm units).

A `Problem` carries the lattice, time step, EOS, transport parametrisations, options and the
initial primaries (e, u^x, u^y, u^eta, pi^{mu nu}, Pi, optional u at tau0 - dtau) on the
physical cells, x fastest then y then eta.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

from .rng import SplitMix64

HBARC = 0.1973269804  # GeV fm


@dataclasses.dataclass
class Problem:
    name: str
    nx: int
    ny: int
    neta: int
    dx: float
    dy: float
    deta: float
    dtau: float
    tau0: float
    nsteps: int
    coords: str = "milne"          # "milne" | "cartesian"
    bc: str = "copy"               # "copy" | "periodic"
    theta: float = 1.0
    eos: object = ("conformal", None)  # ("conformal", a) or workload.eos.TableEOS
    eta_over_s: tuple = ("const", 0.0, 0.0, 1.0)    # (kind, c0, c1, c2), T in fm^-1
    zeta_over_s: tuple = ("const", 0.0, 0.0, 1.0)
    tau_pipi_on: bool = True
    regulate: bool = True
    rho_max: float = 1.0
    xi0: float = 0.1
    e_min: float = 0.0
    tau_relax_min: float = 0.0
    iface: str = "recon"           # "recon" | "invert"
    # initial primaries on physical cells
    e: Optional[np.ndarray] = None        # [cells]
    u: Optional[np.ndarray] = None        # [3, cells]: u^x, u^y, u^eta
    pi: Optional[np.ndarray] = None       # [10, cells]: tt tx ty tn xx xy xn yy yn nn
    Pi: Optional[np.ndarray] = None       # [cells]
    u_prev: Optional[np.ndarray] = None   # [3, cells] at tau0 - dtau

    @property
    def ncells(self) -> int:
        return self.nx * self.ny * self.neta

    def coords_xyz(self):
        """Cell-centre coordinates (x, y, eta) of the physical cells, each shaped [neta, ny, nx]."""
        x = (np.arange(self.nx) - (self.nx - 1) / 2.0) * self.dx
        y = (np.arange(self.ny) - (self.ny - 1) / 2.0) * self.dy
        z = (np.arange(self.neta) - (self.neta - 1) / 2.0) * self.deta
        Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
        return X, Y, Z

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


def conformal_eos():
    from .eos import A_SB
    return ("conformal", A_SB)


# ----------------------------------------------------------------------------- Gubser (C0)
def gubser_problem(nx=32, ny=32, neta=8, dx=0.1, deta=0.1, dtau=0.01, tau0=1.0, nsteps=20,
                   eta_over_s=0.2, T0hat=1.2, q=1.0, theta=1.8, regulate=True) -> Problem:
    """Viscous Gubser flow, conformal EOS, tau_pipi = 0 (Sec. 5.7), pi^{mu nu} on the
    Gubser-symmetric solution that starts from its Navier-Stokes value (0) at rho = 0."""
    from .gubser import GubserSolution
    from .eos import A_SB
    sol = GubserSolution(eta_over_s=eta_over_s, T0hat=T0hat, q=q)
    p = Problem(name=f"gubser_{nx}x{ny}x{neta}", nx=nx, ny=ny, neta=neta, dx=dx, dy=dx, deta=deta,
                dtau=dtau, tau0=tau0, nsteps=nsteps, coords="milne", bc="copy", theta=theta,
                eos=conformal_eos(), eta_over_s=("const", eta_over_s, 0.0, 1.0),
                zeta_over_s=("const", 0.0, 0.0, 1.0), tau_pipi_on=False, regulate=regulate,
                e_min=0.0, tau_relax_min=0.0)
    X, Y, _ = p.coords_xyz()
    st = sol.state(tau0, X.ravel(), Y.ravel(), A_SB)
    stp = sol.state(tau0 - dtau, X.ravel(), Y.ravel(), A_SB)
    p.e = st["e"]
    p.u = np.stack([st["ux"], st["uy"], np.zeros_like(st["ux"])])
    p.pi = st["pi"]
    p.Pi = np.zeros_like(st["e"])
    p.u_prev = np.stack([stp["ux"], stp["uy"], np.zeros_like(stp["ux"])])
    p.gubser = sol  # reference for the semi-analytic comparison
    return p


# ------------------------------------------------------------------- hotspots (128^3 workload)
def hotspot_energy(X, Y, Z, nhot, seed, r_max=6.0, width=0.4, eta_width=1.5, amp_median=30.0,
                   amp_sigma=0.5, e_floor_gev=1e-4):
    """Sum of Gaussian hotspots (GeV/fm^3) times a Gaussian eta profile, plus a floor.

    Centres uniform in the disc r < r_max (r = r_max sqrt(U1), phi = 2 pi U2); amplitudes
    lognormal, A = amp_median exp(amp_sigma Z) with Z ~ N(0,1) by Box-Muller; SplitMix64(seed).
    """
    rng = SplitMix64(seed)
    e = np.zeros_like(X)
    for _ in range(nhot):
        r = r_max * math.sqrt(rng.uniform())
        phi = 2.0 * math.pi * rng.uniform()
        A = amp_median * math.exp(amp_sigma * rng.normal())
        xk, yk = r * math.cos(phi), r * math.sin(phi)
        e += A * np.exp(-((X - xk) ** 2 + (Y - yk) ** 2) / (2.0 * width ** 2))
    e *= np.exp(-Z ** 2 / (2.0 * eta_width ** 2))
    return e + e_floor_gev


def hotspot_problem(nx=128, ny=128, neta=128, dx=0.1, deta=0.1, tau0=0.5, dtau=0.005, nsteps=100,
                    nhot=50, seed=1, eta_over_s=0.08, zeta=True, r_max=6.0, theta=1.0,
                    e_floor_gev=1e-4, eos_table=None) -> Problem:
    """The 128^3 nonconformal viscous workload: tabulated EOS with c_s^2(T) = 1/3 - 0.2
    exp(-((T-0.17)/0.05)^2), eta/s = 0.08, zeta/s = 0.1 exp(-((T-0.17)/0.03)^2), hotspot e,
    u at rest, pi = Pi = 0.  zeta: True / "gauss" (that zeta/s), "paper" (Eq. zetas) or False;
    eos_table: another table (e.g. the lattice EOS of Sec. 2.3)."""
    from .eos import baseline_table
    tab = eos_table if eos_table is not None else baseline_table()
    zs = zeta_coef(zeta)
    p = Problem(name=f"hotspots_{nx}x{ny}x{neta}_s{seed}", nx=nx, ny=ny, neta=neta, dx=dx, dy=dx,
                deta=deta, dtau=dtau, tau0=tau0, nsteps=nsteps, coords="milne", bc="copy",
                theta=theta, eos=tab, eta_over_s=("const", eta_over_s, 0.0, 1.0), zeta_over_s=zs,
                tau_pipi_on=True, regulate=True, e_min=1e-12 * e_floor_gev / HBARC,
                tau_relax_min=dtau)
    X, Y, Z = p.coords_xyz()
    e = hotspot_energy(X, Y, Z, nhot, seed, r_max=r_max, e_floor_gev=e_floor_gev) / HBARC
    p.e = np.ascontiguousarray(e.ravel())
    p.u = np.zeros((3, p.ncells))
    p.pi = np.zeros((10, p.ncells))
    p.Pi = np.zeros(p.ncells)
    return p


# ------------------------------------------------------------------------- Riemann problems
def sod_problem(nx=200, dx=0.1, dt=None, t_end=2.0, e_left_gev=0.0246, e_right_gev=0.0015,
                theta=1.0, axis=0) -> Problem:
    """1D relativistic Sod shock tube (Sec. 5.1): ideal, Cartesian, conformal; membrane at x = 0
    along the chosen axis (0 = x, 1 = y, 2 = eta/z)."""
    dt = dt if dt is not None else dx / 4.0
    n = [1, 1, 1]
    n[axis] = nx
    p = Problem(name=f"sod_{nx}", nx=n[0], ny=n[1], neta=n[2], dx=dx, dy=dx, deta=dx, dtau=dt, tau0=1.0,
                nsteps=int(round(t_end / dt)), coords="cartesian", bc="copy", theta=theta,
                eos=conformal_eos(), regulate=False)
    X, Y, Z = p.coords_xyz()
    xs = [X, Y, Z][axis].ravel()
    p.e = np.where(xs <= 0.0, e_left_gev, e_right_gev) / HBARC
    return p


def sod_diagonal_problem(n=100, dx=0.1, dt=None, t_end=1.5, e_left_gev=0.0246, e_right_gev=0.0015) -> Problem:
    """2D shock tube with the membrane along y = x (Sec. 5.2)."""
    dt = dt if dt is not None else dx / 4.0
    p = Problem(name=f"sod2d_{n}", nx=n, ny=n, neta=1, dx=dx, dy=dx, deta=dx, dtau=dt, tau0=1.0,
                nsteps=int(round(t_end / dt)), coords="cartesian", bc="copy", eos=conformal_eos(),
                regulate=False)
    X, Y, _ = p.coords_xyz()
    p.e = np.where((X - Y).ravel() >= 0.0, e_right_gev, e_left_gev) / HBARC
    return p


def cylinder_problem(n=60, dx=0.2, dt=None, t_end=1.0, R=1.0, e_in_gev=0.0246, e_out_gev=0.0015) -> Problem:
    """Cylindrical explosion (Sec. 5.3)."""
    dt = dt if dt is not None else dx / 4.0
    p = Problem(name=f"cyl_{n}", nx=n, ny=n, neta=1, dx=dx, dy=dx, deta=dx, dtau=dt, tau0=1.0,
                nsteps=int(round(t_end / dt)), coords="cartesian", bc="copy", eos=conformal_eos(),
                regulate=False)
    X, Y, _ = p.coords_xyz()
    p.e = np.where((X ** 2 + Y ** 2).ravel() <= R * R, e_in_gev, e_out_gev) / HBARC
    return p


# ----------------------------------------------------------------------------------- Bjorken
ZETA_PAPER_TC_GEV = 0.2  # T_c of the zeta/s parametrisation of Sec. 2.2 (Eq. zetas)


def zeta_coef(kind):
    """zeta/s inputs: "gauss" = 0.1 exp(-((T - 0.17 GeV)/0.03 GeV)^2) (the 128^3 workload),
    "paper" = Eq. (zetas) with T_c = 200 MeV and normalisation 1, None/False = off."""
    if kind in (True, "gauss"):
        return ("gauss", 0.1, 0.17 / HBARC, 0.03 / HBARC)
    if kind == "paper":
        return ("paper", 1.0, ZETA_PAPER_TC_GEV / HBARC, 1.0)
    return ("const", 0.0, 0.0, 1.0)


def bjorken_problem(T0_gev=0.6, tau0=0.25, dtau=0.005, nsteps=100, eta_over_s=0.2, eos="conformal",
                    zeta=False, n=4, pi_ns=True, tau_pipi_on=True) -> Problem:
    """Transversely homogeneous, boost-invariant flow (Secs. 5.4-5.5) on a small uniform grid.
    eos: "conformal", "table" (the 128^3 workload's c_s^2(T)) or "lattice" (Sec. 2.3)."""
    from .eos import A_SB, baseline_table, lattice_table
    if eos == "conformal":
        eosv = conformal_eos()
    elif eos == "lattice":
        eosv = lattice_table()
    else:
        eosv = baseline_table()
    zs = zeta_coef(zeta)
    p = Problem(name="bjorken", nx=n, ny=n, neta=n, dx=0.1, dy=0.1, deta=0.1, dtau=dtau, tau0=tau0,
                nsteps=nsteps, coords="milne", bc="copy", theta=1.0, eos=eosv,
                eta_over_s=("const", eta_over_s, 0.0, 1.0), zeta_over_s=zs, tau_pipi_on=tau_pipi_on,
                regulate=False, tau_relax_min=0.0)
    T0 = T0_gev / HBARC
    if eos == "conformal":
        e0 = A_SB * T0 ** 4
        s0 = 4.0 / 3.0 * A_SB * T0 ** 3
    else:
        tab = eosv
        lT = np.log(tab.T)
        e0 = float(np.exp(np.interp(math.log(T0), lT, np.log(tab.e))))
        P0 = float(np.interp(math.log(T0), lT, tab.p))
        s0 = (e0 + P0) / T0
    N = p.ncells
    p.e = np.full(N, e0)
    p.u = np.zeros((3, N))
    pi = np.zeros((10, N))
    if pi_ns and eta_over_s > 0:
        eta = eta_over_s * s0
        pibar = 4.0 * eta / (3.0 * tau0)  # pi = -tau^2 pi^{eta eta} at its Navier-Stokes value
        pi[4] = pibar / 2.0               # pi^xx
        pi[7] = pibar / 2.0               # pi^yy
        pi[9] = -pibar / tau0 ** 2        # pi^{eta eta}
    p.pi = pi
    p.Pi = np.zeros(N)
    p.bjorken_s0 = s0
    return p


def batch_shapes(n_events=64, seed=1000, nx_choices=tuple(range(64, 161, 16)), neta_choices=(16, 32, 48, 64),
                 hot_range=(20, 100)):
    """The per-event draws of batch_problems without the fields: (nx = ny, neta, hotspots)."""
    rng = SplitMix64(seed)
    out = []
    for _ in range(n_events):
        n = nx_choices[int(rng.uniform() * len(nx_choices))]
        nz = neta_choices[int(rng.uniform() * len(neta_choices))]
        nhot = hot_range[0] + int(rng.uniform() * (hot_range[1] - hot_range[0] + 1))
        out.append((n, nz, nhot))
    return out


def batch_problems(n_events=64, seed=1000, eta_over_s=0.08, nx_choices=tuple(range(64, 161, 16)),
                   neta_choices=(16, 32, 48, 64), hot_range=(20, 100), events=None, **kw):
    """Events with fluctuating initial conditions and uneven grids: per event nx = ny drawn
    uniformly from nx_choices, neta from neta_choices, the hotspot count uniformly in hot_range,
    hotspot seed = seed + event (all draws from SplitMix64(seed)).  events: build only these
    event indices of the batch (in the given order), e.g. one rank's share."""
    shapes = batch_shapes(n_events, seed, nx_choices, neta_choices, hot_range)
    idx = range(n_events) if events is None else events
    return [hotspot_problem(nx=shapes[ev][0], ny=shapes[ev][0], neta=shapes[ev][1], nhot=shapes[ev][2],
                            seed=seed + ev, eta_over_s=eta_over_s, **kw) for ev in idx]
