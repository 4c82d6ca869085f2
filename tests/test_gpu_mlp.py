"""The learned root-find start on the GPU: features, gradients against the FP64 reference,
tensor-core inference, Adam, training and the learned inversion inside the stage kernel."""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
from workload.problem import hotspot_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1608_06577_gb300 import build
    build.build()
    oracle.build()


def _torch():
    import torch
    return torch


def _small(seed, n=40, nz=20):
    return hotspot_problem(nx=n, ny=n, neta=nz, nhot=10, seed=seed, r_max=1.2)


def test_features_and_exact_targets_match_reference(baseline_eos):
    torch = _torch()
    from paper_1608_06577_gb300 import KT, KT_MIXED
    p = _small(3)
    kt = KT(p, precision=KT_MIXED)
    kt.set_problem_state()
    kt.step(6)
    cells = torch.arange(0, p.ncells, 7, device="cuda")
    x, y, e = kt.mlp_features(cells)
    s = kt.get_state(fields=("q",))
    q = s["q"][:, cells.cpu().numpy()]
    tau = s["tau"]
    E = q[0] - q[4]
    M2 = (q[1] - q[5]) ** 2 + (q[2] - q[6]) ** 2 + tau ** 2 * (q[3] - q[7]) ** 2
    Xr, ec = omlp.features(E, M2, q[14])
    np.testing.assert_allclose(x.cpu().numpy(), Xr, rtol=2e-5, atol=2e-6)
    o = oracle.Oracle(p)
    ee = np.array([o.invert(tau, q[:, k])[1][0] for k in range(q.shape[1])])
    np.testing.assert_allclose(e.cpu().numpy(), ee, rtol=1e-13)
    yref = 10 * np.log(ee / (E * ec))
    np.testing.assert_allclose(y.cpu().numpy(), yref, atol=5e-5)


def test_gradient_matches_fp64_backprop():
    torch = _torch()
    from paper_1608_06577_gb300.binding import mlp_grad
    rng = np.random.default_rng(0)
    p = (rng.normal(size=omlp.NPARAM) * 0.3).astype(np.float32)
    X = rng.normal(size=(3000, 6)).astype(np.float32)
    Y = rng.normal(size=3000).astype(np.float32)
    g, loss = mlp_grad(torch.as_tensor(p, device="cuda"), torch.as_tensor(X, device="cuda"),
                       torch.as_tensor(Y, device="cuda"), bf16_forward=False)
    lr, gr = omlp.loss_and_grad(p.astype(np.float64), X.astype(np.float64), Y.astype(np.float64))
    g = g.cpu().numpy()
    assert abs(loss.item() - lr) < 1e-5 * lr
    assert np.max(np.abs(g - gr)) < 1e-4 * np.max(np.abs(gr))
    # BF16 forward: gradient of the rounded network, close to the FP32 one
    gb, lb = mlp_grad(torch.as_tensor(p, device="cuda"), torch.as_tensor(X, device="cuda"),
                      torch.as_tensor(Y, device="cuda"), bf16_forward=True)
    yb, _ = omlp.forward(p, X, bf16=True)
    assert abs(lb.item() - np.mean((yb - Y) ** 2)) < 2e-3 * lr
    assert np.max(np.abs(gb.cpu().numpy() - gr)) < 5e-2 * np.max(np.abs(gr))


def test_tensor_core_inference_matches_reference():
    torch = _torch()
    from paper_1608_06577_gb300.binding import mlp_predict
    rng = np.random.default_rng(1)
    p = (rng.normal(size=omlp.NPARAM) * 0.3).astype(np.float32)
    X = rng.normal(size=(1000, 6)).astype(np.float32)  # not a multiple of 32: ragged last warp
    y = mlp_predict(torch.as_tensor(p, device="cuda"), torch.as_tensor(X, device="cuda")).cpu().numpy()
    yb, _ = omlp.forward(p, X, bf16=True)
    yf, _ = omlp.forward(p, X, bf16=False)
    scale = np.max(np.abs(yf))
    assert np.max(np.abs(y - yb)) < 1e-2 * scale   # same rounding points, FP32 accumulation order
    assert np.max(np.abs(y - yf)) < 5e-2 * scale   # BF16 weights and activations vs exact FP64


def test_adam_step_formula():
    torch = _torch()
    from paper_1608_06577_gb300.binding import mlp_adam
    rng = np.random.default_rng(2)
    p0 = rng.normal(size=omlp.NPARAM).astype(np.float32)
    g = rng.normal(size=omlp.NPARAM).astype(np.float32)
    P = torch.as_tensor(p0.copy(), device="cuda")
    m = torch.zeros_like(P)
    v = torch.zeros_like(P)
    mlp_adam(P, torch.as_tensor(g, device="cuda"), m, v, 1, 1e-2)
    mh = 0.1 * g / (1 - 0.9)
    vh = 0.001 * g * g / (1 - 0.999)
    ref = p0 - 1e-2 * mh / (np.sqrt(vh) + 1e-8)
    np.testing.assert_allclose(P.cpu().numpy(), ref, rtol=1e-5, atol=1e-6)


@pytest.fixture(scope="module")
def trained():
    from paper_1608_06577_gb300 import learned
    X, Y = learned.collect(lambda s: _small(s, n=48, nz=24), [2, 5, 6], 200_000, steps=40, every=4)
    params, losses = learned.train(*learned.network_targets(X, Y), epochs=12, batch=4096)
    return params, losses, X, Y


def test_training_reduces_loss(trained):
    from paper_1608_06577_gb300 import learned
    params, losses, X, Y = trained
    mx, rms = learned.evaluate(params, X, Y)
    print("trained network: loss after epoch 1", losses[0], "-> final", losses[-1], "max err", mx, "rms", rms)
    assert losses[-1] < 0.3 * losses[0]
    # rms 1e-2 in y = 10 ln(e/e_conf) is a 1e-3 relative start: two Newton steps reach 1e-10
    assert rms < 1e-2
    # the correction beats the conformal root it corrects (y = 0)
    assert rms < 0.5 * float(Y.double().pow(2).mean().sqrt().item())


def test_learned_inversion_accuracy_and_gain(trained):
    """Mixed precision with the learned start vs the oracle after 40 steps (held-out seed),
    and what it gains over the plain start: Newton steps per cell and stage."""
    from paper_1608_06577_gb300 import KT, KT_MIXED, KT_INV_LEARNED
    params, _, _, _ = trained
    p = _small(4)
    ktl = KT(p, precision=KT_MIXED, inversion=KT_INV_LEARNED, mlp_weights=params.cpu().numpy())
    ktl.set_problem_state()
    ktl.step(40)
    sl = ktl.stats()
    g = ktl.get_state(fields=("e", "u"))
    ktp = KT(p, precision=KT_MIXED)
    ktp.set_problem_state()
    ktp.step(40)
    sp = ktp.stats()
    o = oracle.Oracle(p)
    o.step(40)
    r = o.get_state()
    rel = np.max(np.abs(g["e"] / r["e"] - 1))
    ncs = p.ncells * 2 * 40
    it_l, it_p = sl["newton_iters"] / ncs, sp["newton_iters"] / ncs
    fb = sl["fallbacks"] / ncs
    print(f"learned: rel err e {rel:.2e}, Newton/cell-stage {it_l:.3f} (plain {it_p:.3f}), fallback rate {fb:.2e}")
    assert rel < 1e-4
    assert fb < 0.02
    assert it_l < it_p
