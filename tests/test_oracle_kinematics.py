"""Pins of the oracle's generic tensor code against the component listings printed in App. A
(sigma, omega, I1, I3, I4), the expansion rate, Du_mu, and App. B's geometric terms G_pi.

The listings use u_tau, u_x, u_y, u_eta for the contravariant components; inside the sigma
listing "D" is the convective derivative d = u^a d_a (the Christoffel parts are written out);
in I1 the D u_lambda are covariant (Du_tau = du_tau + tau u_eta^2, Du_eta = -tau^2 du^eta
- 2 tau u_tau u_eta).  The oracle computes everything from covariant definitions with explicit
Christoffel symbols, so agreement pins index order, signs and metric factors.
"""
import numpy as np
import pytest

import oracle
from workload.problem import Problem, conformal_eos


def _ctx(coords="milne"):
    p = Problem(name="k", nx=1, ny=1, neta=1, dx=0.1, dy=0.1, deta=0.1, dtau=0.01, tau0=1.0, nsteps=0,
                coords=coords, eos=conformal_eos(), eta_over_s=("const", 0.2, 0, 1))
    p.e = np.ones(1)
    return oracle.Oracle(p)


def _random_point(rng, tau):
    ux, uy, un = rng.uniform(-0.8, 0.8, 3)
    un /= tau
    ut = np.sqrt(1 + ux * ux + uy * uy + tau * tau * un * un)
    u = np.array([ut, ux, uy, un])
    du = rng.normal(size=(4, 4))
    X = rng.normal(size=(4, 4))
    pi = X + X.T
    return u, du, pi


def listing(tau, u, du, pi):
    ut, ux, uy, un = u

    def d(m):
        return sum(u[a] * du[a][m] for a in range(4))

    dut, dux, duy, dun = d(0), d(1), d(2), d(3)
    theta = ut / tau + du[0][0] + du[1][1] + du[2][2] + du[3][3]
    Du_t = dut + tau * un ** 2
    Du_x, Du_y = -dux, -duy
    Du_n = -tau ** 2 * dun - 2 * tau * ut * un
    s = np.zeros((4, 4))
    s[0, 0] = -tau * ut * un ** 2 + du[0][0] - ut * dut + (ut ** 2 - 1) * theta / 3
    s[0, 1] = -tau * un ** 2 * ux / 2 + 0.5 * (du[0][1] - du[1][0]) - 0.5 * (ut * dux + ux * dut) + ut * ux * theta / 3
    s[0, 2] = -tau * un ** 2 * uy / 2 + 0.5 * (du[0][2] - du[2][0]) - 0.5 * (ut * duy + uy * dut) + ut * uy * theta / 3
    s[0, 3] = (-un / (2 * tau) * (2 * ut ** 2 + tau ** 2 * un ** 2) + 0.5 * (du[0][3] - du[3][0] / tau ** 2)
               - 0.5 * (ut * dun + un * dut) + ut * un * theta / 3)
    s[3, 3] = -ut / tau ** 3 * (1 + 2 * un ** 2 * tau ** 2) - du[3][3] / tau ** 2 - un * dun + (1 / tau ** 2 + un ** 2) * theta / 3
    s[1, 3] = -ut * ux * un / tau - 0.5 * (du[1][3] + du[3][1] / tau ** 2) - 0.5 * (ux * dun + un * dux) + ux * un * theta / 3
    s[2, 3] = -ut * uy * un / tau - 0.5 * (du[2][3] + du[3][2] / tau ** 2) - 0.5 * (uy * dun + un * duy) + uy * un * theta / 3
    s[1, 1] = -du[1][1] - ux * dux + (1 + ux ** 2) * theta / 3
    s[2, 2] = -du[2][2] - uy * duy + (1 + uy ** 2) * theta / 3
    s[1, 2] = -0.5 * (du[1][2] + du[2][1]) - 0.5 * (ux * duy + uy * dux) + ux * uy * theta / 3
    for a in range(4):
        for b in range(a):
            s[a, b] = s[b, a]
    # omega^mu_lambda listing
    W = np.zeros((4, 4))
    wtx = 0.5 * (du[0][1] + du[1][0]) + 0.5 * (ux * dut - ut * dux) + 0.5 * tau * un ** 2 * ux
    wty = 0.5 * (du[0][2] + du[2][0]) + 0.5 * (uy * dut - ut * duy) + 0.5 * tau * un ** 2 * uy
    d_t2un = tau ** 2 * dun + 2 * tau * ut * un  # d(tau^2 u_eta)
    wtn = (0.5 * (2 * tau * un + tau ** 2 * du[0][3] + du[3][0]) + 0.5 * (tau ** 2 * un * dut - ut * d_t2un)
           + 0.5 * tau ** 3 * un ** 3)
    wxy = 0.5 * (du[2][1] - du[1][2]) + 0.5 * (uy * dux - ux * duy)
    wxn = 0.5 * (du[3][1] - tau ** 2 * du[1][3]) + 0.5 * (tau ** 2 * un * dux - ux * d_t2un)
    wyn = 0.5 * (du[3][2] - tau ** 2 * du[2][3]) + 0.5 * (tau ** 2 * un * duy - uy * d_t2un)
    W[0, 1] = W[1, 0] = wtx
    W[0, 2] = W[2, 0] = wty
    W[0, 3], W[3, 0] = wtn, wtn / tau ** 2
    W[1, 2], W[2, 1] = wxy, -wxy
    W[1, 3], W[3, 1] = wxn, -wxn / tau ** 2
    W[2, 3], W[3, 2] = wyn, -wyn / tau ** 2
    p = pi
    I1 = {
        (1, 1): 2 * ux * (p[0][1] * Du_t + p[1][1] * Du_x + p[2][1] * Du_y + p[3][1] * Du_n),
        (2, 2): 2 * uy * (p[0][2] * Du_t + p[1][2] * Du_x + p[2][2] * Du_y + p[3][2] * Du_n),
        (1, 2): ((p[0][1] * uy + p[0][2] * ux) * Du_t + (p[1][1] * uy + p[1][2] * ux) * Du_x
                 + (p[2][1] * uy + p[2][2] * ux) * Du_y + (p[3][1] * uy + p[3][2] * ux) * Du_n),
        (1, 3): ((p[0][1] * un + p[0][3] * ux) * Du_t + (p[1][1] * un + p[1][3] * ux) * Du_x
                 + (p[2][1] * un + p[2][3] * ux) * Du_y + (p[3][1] * un + p[3][3] * ux) * Du_n),
        (2, 3): ((p[0][2] * un + p[0][3] * uy) * Du_t + (p[1][2] * un + p[1][3] * uy) * Du_x
                 + (p[2][2] * un + p[2][3] * uy) * Du_y + (p[3][2] * un + p[3][3] * uy) * Du_n),
    }
    I3 = {
        (1, 1): 2 * (p[1][0] * W[1][0] + p[1][2] * W[1][2] + p[1][3] * W[1][3]),
        (2, 2): 2 * (p[2][0] * W[2][0] + p[2][1] * W[2][1] + p[2][3] * W[2][3]),
        (1, 2): (p[1][0] * W[2][0] + p[2][0] * W[1][0] + p[1][1] * W[2][1] + p[2][2] * W[1][2]
                 + p[1][3] * W[2][3] + p[2][3] * W[1][3]),
        (1, 3): (p[1][0] * W[3][0] + p[3][0] * W[1][0] + p[1][1] * W[3][1] + p[1][2] * W[3][2]
                 + p[3][2] * W[1][2] + p[3][3] * W[1][3]),
        (2, 3): (p[2][0] * W[3][0] + p[3][0] * W[2][0] + p[2][1] * W[3][1] + p[3][1] * W[2][1]
                 + p[2][2] * W[3][2] + p[3][3] * W[2][3]),
    }
    g = np.array([1.0, -1.0, -1.0, -tau ** 2])
    ps = float(np.einsum("ab,ab,a,b->", p, s, g, g))
    S = s
    t2 = tau ** 2
    I4 = {
        (1, 1): p[1][0] * S[1][0] - p[1][1] * S[1][1] - p[1][2] * S[1][2] - t2 * p[1][3] * S[1][3] + (1 + ux ** 2) * ps / 3,
        (2, 2): p[2][0] * S[2][0] - p[2][1] * S[2][1] - p[2][2] * S[2][2] - t2 * p[2][3] * S[2][3] + (1 + uy ** 2) * ps / 3,
        (1, 2): (0.5 * (p[1][0] * S[2][0] + p[2][0] * S[1][0]) - 0.5 * (p[1][1] * S[2][1] + p[2][1] * S[1][1])
                 - 0.5 * (p[1][2] * S[2][2] + p[2][2] * S[1][2]) - t2 / 2 * (p[1][3] * S[2][3] + p[2][3] * S[1][3])
                 + ux * uy * ps / 3),
        (1, 3): (0.5 * (p[1][0] * S[3][0] + p[3][0] * S[1][0]) - 0.5 * (p[1][1] * S[3][1] + p[3][1] * S[1][1])
                 - 0.5 * (p[1][2] * S[3][2] + p[3][2] * S[1][2]) - t2 / 2 * (p[1][3] * S[3][3] + p[3][3] * S[1][3])
                 + ux * un * ps / 3),
        (2, 3): (0.5 * (p[2][0] * S[3][0] + p[3][0] * S[2][0]) - 0.5 * (p[2][1] * S[3][1] + p[3][1] * S[2][1])
                 - 0.5 * (p[2][2] * S[3][2] + p[3][2] * S[2][2]) - t2 / 2 * (p[2][3] * S[3][3] + p[3][3] * S[2][3])
                 + uy * un * ps / 3),
    }
    return {"theta": theta, "Du": np.array([Du_t, Du_x, Du_y, Du_n]), "sigma": s, "W": W,
            "I1": I1, "I3": I3, "I4": I4}


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("tau", [0.6, 1.0, 2.3])
def test_tensors_match_appendix_listing(seed, tau):
    o = _ctx()
    rng = np.random.default_rng(seed)
    u, du, pi = _random_point(rng, tau)
    got = o.tensor_terms(tau, u, du, pi)
    ref = listing(tau, u, du, pi)
    tol = 1e-12
    scale = 1.0 + np.abs(du).max()
    assert abs(got["theta"] - ref["theta"]) < tol * scale
    np.testing.assert_allclose(got["Du"], ref["Du"], rtol=0, atol=tol * scale * 10)
    np.testing.assert_allclose(got["sigma"], ref["sigma"], rtol=0, atol=tol * scale * 10)
    g = np.array([1.0, -1.0, -1.0, -tau ** 2])
    om_mixed = got["omega"] * g[None, :]
    np.testing.assert_allclose(om_mixed, ref["W"], rtol=0, atol=tol * scale * 10)
    sc = scale * (1 + np.abs(pi).max()) * 100
    for k in ref["I1"]:
        assert abs(got["I1"][k] - ref["I1"][k]) < tol * sc, ("I1", k)
        assert abs(got["I3"][k] - ref["I3"][k]) < tol * sc, ("I3", k)
        assert abs(got["I4"][k] - ref["I4"][k]) < tol * sc, ("I4", k)


def test_geometric_pi_terms_appendix_b():
    """App. B's G_pi rows, from G^{mu nu} = u^a Gamma^mu_{ab} pi^{b nu} + u^a Gamma^nu_{ab} pi^{b mu}
    divided by -u^tau.  The tau-x and tau-y rows follow the definition (one Christoffel term,
    -tau v_eta pi^{x eta}); the listing's factor 2 there is read as a misprint."""
    o = _ctx()
    rng = np.random.default_rng(7)
    tau = 1.7
    u, du, pi = _random_point(rng, tau)
    G = o.tensor_terms(tau, u, du, pi)["Gpi"]
    vn = u[3] / u[0]
    exp = np.zeros((4, 4))
    exp[0, 0] = -2 * tau * vn * pi[0][3]
    exp[0, 1] = -tau * vn * pi[1][3]
    exp[0, 2] = -tau * vn * pi[2][3]
    exp[0, 3] = -tau * vn * pi[3][3] - (pi[0][3] + vn * pi[0][0]) / tau
    exp[1, 3] = -(pi[1][3] + vn * pi[0][1]) / tau
    exp[2, 3] = -(pi[2][3] + vn * pi[0][2]) / tau
    exp[3, 3] = -2.0 / tau * (pi[3][3] + vn * pi[0][3])
    for a in range(4):
        for b in range(a, 4):
            assert abs(G[a, b] - exp[a, b]) < 1e-13 * (1 + np.abs(pi).max()), (a, b)


def test_expansion_rate_bjorken_and_cartesian():
    o = _ctx()
    u = np.array([1.0, 0, 0, 0])
    for tau in (0.25, 1.0, 3.0):
        t = o.tensor_terms(tau, u, np.zeros((4, 4)), np.zeros((4, 4)))
        assert abs(t["theta"] - 1.0 / tau) < 1e-15
        # Bjorken shear: sigma^{xx} = sigma^{yy} = 1/(3 tau), sigma^{eta eta} = -2/(3 tau^3)
        assert abs(t["sigma"][1, 1] - 1 / (3 * tau)) < 1e-15
        assert abs(t["sigma"][3, 3] + 2 / (3 * tau ** 3)) < 1e-14
    oc = _ctx("cartesian")
    t = oc.tensor_terms(1.0, u, np.zeros((4, 4)), np.zeros((4, 4)))
    assert t["theta"] == 0.0 and np.all(t["sigma"] == 0.0)


def test_sigma_traceless_orthogonal_for_consistent_gradients():
    """With d_a u^tau consistent with u.u = 1, sigma^{mu nu} is traceless and orthogonal to u."""
    o = _ctx()
    rng = np.random.default_rng(11)
    tau = 1.3
    for _ in range(5):
        u, du, _ = _random_point(rng, tau)
        ut, ux, uy, un = u
        for a in range(4):
            du[a][0] = (ux * du[a][1] + uy * du[a][2] + tau ** 2 * un * du[a][3] + (tau * un ** 2 if a == 0 else 0)) / ut
        s = o.tensor_terms(tau, u, du, np.zeros((4, 4)))["sigma"]
        g = np.array([1.0, -1.0, -1.0, -tau ** 2])
        assert abs(np.sum(g * np.diag(s))) < 1e-12 * (1 + np.abs(du).max())
        np.testing.assert_allclose(s @ (g * u), 0.0, atol=1e-12 * (1 + np.abs(du).max()))
