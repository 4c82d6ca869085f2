"""Batched events: one persistent launch per stage advances events with uneven grids; each
event's result is bit-identical to the same event run alone."""
import numpy as np
import pytest

import oracle
from workload.problem import batch_problems, hotspot_problem

pytestmark = pytest.mark.gpu

FIELDS = ("e", "u", "pi", "Pi", "q")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1608_06577_gb300 import build
    build.build()
    oracle.build()


def _events():
    return batch_problems(n_events=5, nx_choices=(20, 36, 52), neta_choices=(6, 12), hot_range=(5, 15), r_max=1.0)


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_equals_single_events_bitwise(precision):
    from paper_1608_06577_gb300 import KT
    probs = _events()
    kb = KT(probs, precision=precision)
    kb.set_problem_state()
    kb.step(7)
    for ev, p in enumerate(probs):
        ks = KT(p, precision=precision)
        ks.set_problem_state()
        ks.step(7)
        a, b = kb.get_state(event=ev), ks.get_state()
        for f in FIELDS:
            assert np.array_equal(a[f], b[f]), (ev, f)


def test_batch_fp64_matches_oracle():
    from paper_1608_06577_gb300 import KT
    probs = _events()
    kb = KT(probs, precision=0)
    kb.set_problem_state()
    kb.step(5)
    for ev in (0, 3):
        o = oracle.Oracle(probs[ev])
        o.step(5)
        r = o.get_state()
        g = kb.get_state(event=ev)
        from test_gpu_parity import field_errors
        r["milne"] = True
        errs = field_errors(g, r)
        bad = {k: v for k, v in errs.items() if not v <= 1e-12}
        assert not bad, (ev, bad)


@pytest.mark.parametrize("pi_fp32", [False, True])
def test_autotuner_reports_and_picks_fastest(pi_fp32):
    """The autotuner times both grid variants of every tile shape as split launches and, where the
    context can run them (FP64 pi storage), as fused launches, and keeps the fastest."""
    from paper_1608_06577_gb300 import KT
    p = hotspot_problem(nx=48, ny=40, neta=16, nhot=8, r_max=1.0)
    k = KT(p, precision=1, pi_fp32=pi_fp32)
    k.set_problem_state()
    k.step(3)
    t = k.tuning()
    ms = np.array(t["candidate_ms"])
    shapes = [(32, 4, 2), (32, 8, 1), (32, 2, 4), (32, 1, 8), (32, 4, 1), (32, 2, 2)]
    timed = np.flatnonzero(ms > 0)
    expect = list(range(12)) + ([] if pi_fp32 else list(range(24, 36)))
    assert len(ms) == 6 * len(shapes) and list(timed) == expect
    best = int(timed[np.argmin(ms[timed])])
    assert t["block"] == shapes[(best % 12) // 2]
    assert t["grid_blocks"] >= 1


@pytest.mark.parametrize("learned", [False, True])
def test_grid_variants_are_bit_identical(learned):
    """Every autotuner candidate runs the same arithmetic on the same tiles: every tile shape, with a
    persistent grid or one block per tile, with the update's inputs read directly or staged in
    shared memory by TMA, as split or fused launches, gives the same state, bit for bit."""
    from paper_1608_06577_gb300 import KT, learned as lm
    p = hotspot_problem(nx=72, ny=56, neta=20, nhot=12, r_max=2.0)
    kw = dict(inversion=1, mlp_weights=lm.init_params(3)) if learned else {}
    shapes = [(32, 4, 2), (32, 8, 1), (32, 2, 4), (32, 1, 8), (32, 4, 1), (32, 2, 2)]
    ref = None
    # shapes (32,4,2), (32,8,1) per tile, (32,4,1), (32,2,2) per tile; then the same staged, fused
    for cand in (0, 3, 8, 11, 12, 15, 20, 23, 24, 27, 32, 35):
        k = KT(p, precision=1, **kw)
        k.set_tuning(cand)
        k.set_problem_state()
        k.step(7)  # two graph replays and one direct step
        assert k.tuning()["block"] == shapes[(cand % 12) // 2]
        st = k.get_state()
        if ref is None:
            ref = st
        else:
            for f in FIELDS:
                assert np.array_equal(st[f], ref[f]), (cand, f)
        del k


def test_sixty_four_event_batch_runs():
    """The 64-event configuration (uneven grids, 3.5e7 cells): one launch per stage, 10 steps,
    finite and inverted everywhere; prints the throughput."""
    import time
    import torch
    from paper_1608_06577_gb300 import KT
    probs = batch_problems(n_events=64)
    cells = sum(p.ncells for p in probs)
    kb = KT(probs, precision=1)
    kb.set_problem_state()
    kb.step(3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    kb.step(12)
    dt = time.perf_counter() - t0
    st = kb.stats()
    print(f"64 events, {cells} cells: {dt / 12 * 1e3:.2f} ms/step, {cells * 12 / dt:.3e} cell updates/s, "
          f"tuning {kb.tuning()['block']}")
    assert st["status"] == 0
    e = kb.get_state(fields=("e",), event=63)["e"]
    assert np.all(np.isfinite(e)) and np.all(e > 0)
