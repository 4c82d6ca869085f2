"""Pins of the FP64 network reference (CPU)."""
import math

import numpy as np

import oracle
from oracle import mlp
from workload.problem import gubser_problem


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = rng.normal(size=mlp.NPARAM) * 0.3
    X = rng.normal(size=(64, 6))
    Y = rng.normal(size=64)
    loss, g = mlp.loss_and_grad(p, X, Y)
    h = 1e-6
    for k in rng.choice(mlp.NPARAM, 80, replace=False):
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (mlp.loss_and_grad(pp, X, Y)[0] - mlp.loss_and_grad(pm, X, Y)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * (1 + abs(fd)), k


def test_bf16_rounding():
    v = np.array([1.0, 1.00390625, 1.001953125, 1.005859375, 1.01171875, -3.0e-3, 0.0])
    r = mlp.bf16_round(v)
    # 7 stored mantissa bits: the spacing at 1 is 2^-7; halfway cases round to the even code
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0
    assert r[3] == 1.0078125 and r[4] == 1.015625
    assert np.all(np.abs(r - v) <= np.abs(v) * 2.0 ** -8 + 1e-300)


def test_conformal_feature_is_the_conformal_root():
    """e_conf/E equals the oracle's conformal inversion (Sec. 2.4 closed form, Pi = 0)."""
    p = gubser_problem(nx=2, ny=2, neta=2)
    o = oracle.Oracle(p)
    rng = np.random.default_rng(1)
    for _ in range(50):
        E = rng.uniform(0.5, 50)
        M = E * rng.uniform(0, 0.95)
        q = np.zeros(15)
        q[0], q[1] = E, M
        st, out = o.invert(1.0, q)
        X, ec = mlp.features(E, M * M, 0.0)
        assert abs(ec * E - out[0]) < 1e-12 * E
        assert abs(X[5] - M / E) < 1e-15 and abs(X[1] - (M / E) ** 2) < 1e-15
        assert abs(X[0] - (math.log(E) - 1) / 6) < 1e-15
