"""Operation count of the scheme per cell and Runge-Kutta stage, from the counting build of the
oracle (kt_oracle.c compiled with the counted scalar of flops.hpp): the algorithmic flops of the
method as the oracle writes it out (generic 4x4 tensors, explicit metric and Christoffel
symbols), broken down into

  rhs        C[q]: reconstruction, speeds, fluxes, kinematics, EOS and transport, sources (Sec. 3.1,
             App. A, App. B) -- one evaluation over all cells, per cell
  inversion  T^{tau mu} -> (e, u^mu) of Sec. 2.4, per call (one per cell and stage)
  regulator  Eq. (regPimunu), per call (one per cell and stage)
  rest       Heun sums (Eqs. step1-finalStep), ghost copies and bookkeeping: the stage total minus
             the three above

TEST AND MEASUREMENT INFRASTRUCTURE ONLY.  Usage: python -m oracle.count_flops [--nz 8]
(a 128 x 128 x nz slab of the 128^3 hotspot workload, one step).
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import FLOP_KINDS, Oracle, read_flops

FLOPS = ("add", "mul", "div", "sqrt", "transcendental")  # the kinds counted as floating-point operations


def _pi16(pi10):
    idx = {(0, 0): 0, (0, 1): 1, (0, 2): 2, (0, 3): 3, (1, 1): 4, (1, 2): 5, (1, 3): 6, (2, 2): 7, (2, 3): 8, (3, 3): 9}
    m = np.empty((4, 4))
    for (a, b), k in idx.items():
        m[a, b] = m[b, a] = pi10[k]
    return m


def breakdown(prob, sample: int = 2000, seed: int = 0) -> dict:
    """Per-cell-stage operation counts by part and kind for `prob`: the third step from its
    initial state, then `sample` cells of the state after it for the per-call parts."""
    o = Oracle(prob, flops=True)
    n = prob.ncells
    o.step(2)  # not counted: pi, Pi and u become non-trivial
    read_flops(reset=True)
    o.step(1)
    step = read_flops()
    o.rhs()
    rhs = read_flops()
    st = o.get_state()
    idx = np.random.default_rng(seed).choice(n, size=min(sample, n), replace=False)
    for i in idx:
        o.invert(st["tau"], st["q"][:, i])
    inv = read_flops()
    P0 = {int(i): o.eos(st["e"][i])[0] for i in idx}
    read_flops(reset=True)
    for i in idx:
        o.regulator_factor(st["tau"], st["e"][i], P0[int(i)], st["u"][:, i], _pi16(st["pi"][:, i]), st["Pi"][i])
    reg = read_flops()
    parts = {"rhs": {k: rhs[k] / n for k in FLOP_KINDS},
             "inversion": {k: inv[k] / len(idx) for k in FLOP_KINDS},
             "regulator": {k: reg[k] / len(idx) for k in FLOP_KINDS}}
    total = {k: step[k] / (2 * n) for k in FLOP_KINDS}
    parts["rest"] = {k: total[k] - sum(parts[p][k] for p in ("rhs", "inversion", "regulator")) for k in FLOP_KINDS}
    parts["stage"] = total
    for p in parts.values():
        p["flops"] = sum(p[k] for k in FLOPS)
    return parts


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nz", type=int, default=8)
    args = ap.parse_args()
    from workload.problem import hotspot_problem
    prob = hotspot_problem(nx=128, ny=128, neta=args.nz)
    res = breakdown(prob)
    print(f"{'part':<10} " + " ".join(f"{k:>14}" for k in FLOP_KINDS + ("flops",)))
    for name, p in res.items():
        print(f"{name:<10} " + " ".join(f"{p[k]:14.1f}" for k in FLOP_KINDS + ("flops",)))
    print(json.dumps({k: round(v["flops"], 1) for k, v in res.items()}))


if __name__ == "__main__":
    main()
