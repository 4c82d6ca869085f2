"""The operation-counting build of the oracle (oracle/flops.hpp, oracle/kt_oracle_flops.cpp):
it must reproduce the plain oracle bit for bit, and its counters must count what the code does."""
import ctypes as C

import numpy as np

import oracle
from oracle.count_flops import breakdown
from workload.problem import hotspot_problem

FIELDS = ("e", "u", "pi", "Pi", "q")


def test_counting_build_reproduces_the_oracle_bitwise():
    p = hotspot_problem(nx=20, ny=16, neta=6, nhot=5, r_max=1.0)
    a, b = oracle.Oracle(p, threads=1), oracle.Oracle(p, flops=True)
    assert a.step(3) == 0 and b.step(3) == 0
    sa, sb = a.get_state(), b.get_state()
    for f in FIELDS:
        assert np.array_equal(sa[f], sb[f]), f


def test_counters_on_the_minmod():
    """minmod(x, min(y, z)) of Sec. 3.1 as the oracle writes it: per two-argument minmod, sgn of
    each argument (one compare for a positive value, two for a negative one), one compare of the
    magnitudes, one add, one multiply and one division by 2."""
    L = oracle.lib(True)
    L.ko_minmod3.restype = C.c_double
    L.ko_minmod3.argtypes = [C.c_double] * 3
    oracle.read_flops(reset=True)
    assert L.ko_minmod3(1.0, 2.0, 3.0) == 1.0
    f = oracle.read_flops()
    assert f == {"add": 2, "mul": 2, "div": 2, "sqrt": 0, "transcendental": 0, "compare": 6}, f
    assert L.ko_minmod3(-1.0, -2.0, -3.0) == -1.0
    f = oracle.read_flops()
    assert f["compare"] == 10 and f["add"] == 2 and f["mul"] == 2 and f["div"] == 2, f


def test_breakdown_adds_up():
    p = hotspot_problem(nx=16, ny=16, neta=4, nhot=4, r_max=1.0)
    r = breakdown(p, sample=50)
    st = r["stage"]
    assert 3000 < st["flops"] < 30000  # kflop-scale per cell and stage
    assert r["rhs"]["flops"] > 0.8 * st["flops"]  # the stencil and sources dominate
    assert r["inversion"]["flops"] > 0 and r["regulator"]["flops"] > 0
    total = sum(r[k]["flops"] for k in ("rhs", "inversion", "regulator", "rest"))
    assert abs(total - st["flops"]) < 1e-6 * st["flops"]
