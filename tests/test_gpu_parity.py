"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

FP64 mode must match the oracle to a max relative error of 1e-12 per field (normalised by
the field's max norm, since pi and Pi cross zero) after 10 steps.
"""
import math

import numpy as np
import pytest

import oracle
from workload.eos import A_SB
from workload.problem import (HBARC, Problem, bjorken_problem, conformal_eos, gubser_problem, hotspot_problem,
                              sod_problem)

pytestmark = pytest.mark.gpu

FIELDS = ("e", "u", "pi", "Pi", "q")


PI_ETA_INDICES = [0, 0, 0, 1, 0, 0, 1, 0, 1, 2]  # eta indices of pi^{tt,tx,ty,tn,xx,xy,xn,yy,yn,nn}
GROUP_FLOOR = 1e-3


def field_errors(g, r, milne=True):
    """Max relative error per field: max|a - b| / max(max|b|, 1e-3 S), where S is the scale of the
    field's tensor in an orthonormal frame (T^{tau mu}: max T^{tau tau}; pi^{mu nu}: max over
    components of |pi^{mu nu}| tau^(number of eta indices); u: max u^tau).  The floor only matters
    for components far below their tensor's size, whose differences are rounding noise of the
    larger components they are computed from."""
    tau = r["tau"] if milne else 1.0
    S_T = np.max(np.abs(r["q"][0]))
    S_pi = max(np.max(np.abs(r["pi"][k])) * tau ** PI_ETA_INDICES[k] for k in range(10))
    S_u = np.max(np.abs(r["u"][0]))
    groups = {"q": [S_T] * 4 + [S_pi * tau ** -PI_ETA_INDICES[k] for k in range(10)] + [0.0],
              "pi": [S_pi * tau ** -PI_ETA_INDICES[k] for k in range(10)],
              "u": [S_u, S_u, S_u, S_u / tau], "e": [0.0], "Pi": [0.0]}
    errs = {}
    for f in FIELDS:
        a, b = np.atleast_2d(g[f]), np.atleast_2d(r[f])
        for k in range(a.shape[0]):
            scale = max(np.max(np.abs(b[k])), GROUP_FLOOR * groups[f][k])
            d = np.max(np.abs(a[k] - b[k]))
            errs[f"{f}[{k}]"] = d / scale if scale > 0 else d
    return errs


def run_pair(p, nsteps, precision=0, pi_fp32=False):
    from paper_1608_06577_gb300 import KT
    kt = KT(p, precision=precision, pi_fp32=pi_fp32)
    kt.set_problem_state()
    kt.step(nsteps)
    g = kt.get_state()
    o = oracle.Oracle(p)
    assert o.step(nsteps) == 0
    r = o.get_state()
    r["milne"] = p.coords == "milne"
    return g, r, kt


def assert_parity(g, r, tol=1e-12):
    errs = field_errors(g, r, r.get("milne", True))
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, bad
    assert abs(g["tau"] - r["tau"]) < 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1608_06577_gb300 import build
    build.build()
    oracle.build()


def test_gubser_c0_fp64_parity_and_physics():
    p = gubser_problem()  # 32x32x8, conformal, eta/s = 0.2, theta = 1.8, 20 steps
    g, r, kt = run_pair(p, 10)
    assert_parity(g, r)
    kt.step(10)
    g = kt.get_state()
    o = oracle.Oracle(p)
    o.step(20)
    assert_parity(g, o.get_state())
    X, Y, _ = p.coords_xyz()
    X, Y = X.ravel(), Y.ravel()
    ref = p.gubser.state(g["tau"], X, Y, A_SB)
    m = (np.abs(Y - 0.05) < 1e-9) & (np.abs(X) <= 1.2) & (np.arange(len(X)) < p.nx * p.ny)
    assert np.max(np.abs(g["e"][m] / ref["e"][m] - 1)) < 0.03


@pytest.mark.parametrize("shape", [(20, 18, 10), (37, 5, 9), (33, 33, 3)])
def test_hotspot_fp64_parity_ragged(shape, baseline_eos):
    nx, ny, nz = shape
    p = hotspot_problem(nx=nx, ny=ny, neta=nz, nhot=12, seed=3, r_max=0.8, eos_table=baseline_eos)
    g, r, _ = run_pair(p, 10)
    assert_parity(g, r)


def test_nonconformal_bjorken_bulk_fp64_parity(baseline_eos):
    p = bjorken_problem(T0_gev=0.22, tau0=0.6, dtau=0.004, nsteps=10, eos="table", zeta=True).replace(
        tau_relax_min=0.005, eos=baseline_eos)
    g, r, _ = run_pair(p, 10)
    assert_parity(g, r)
    assert np.max(np.abs(g["Pi"])) > 1e-3


def test_periodic_cartesian_viscous_parity_and_conservation(baseline_eos):
    n = 12
    p = Problem(name="per", nx=n, ny=n - 2, neta=n - 4, dx=0.2, dy=0.2, deta=0.2, dtau=0.02, tau0=1.0, nsteps=10,
                coords="cartesian", bc="periodic", theta=1.5, eos=baseline_eos, eta_over_s=("const", 0.2, 0, 1),
                zeta_over_s=("gauss", 0.1, 0.17 / HBARC, 0.03 / HBARC), tau_relax_min=0.02)
    X, Y, Z = p.coords_xyz()
    kx, ky, kz = 2 * np.pi / (p.nx * 0.2), 2 * np.pi / (p.ny * 0.2), 2 * np.pi / (p.neta * 0.2)
    p.e = (1.0 / HBARC) * (1 + 0.5 * np.sin(kx * X) * np.cos(ky * Y) + 0.3 * np.sin(kz * Z)).ravel()
    p.u = np.stack([0.2 * np.sin(ky * Y).ravel(), 0.1 * np.cos(kx * X).ravel(), 0.15 * np.sin(kx * X + kz * Z).ravel()])
    g, r, kt = run_pair(p, 10)
    assert_parity(g, r)
    kt2_q0 = np.sum(r["q"][:4], axis=1)
    from paper_1608_06577_gb300 import KT
    k2 = KT(p)
    k2.set_problem_state()
    q0 = np.sum(k2.get_state()["q"][:4], axis=1)
    k2.step(30)
    q1 = np.sum(k2.get_state()["q"][:4], axis=1)
    assert np.max(np.abs(q1 - q0)) < 1e-13 * q0[0]
    assert kt2_q0 is not None


@pytest.mark.parametrize("mode", ["fp64", "mixed", "conformal"])
def test_uniform_fluid_at_rest_is_stationary(mode, baseline_eos):
    """The degenerate state: a uniform fluid at rest with pi = Pi = 0 on a periodic Cartesian grid
    (ragged against the tiles) has every difference, face speed, flux and source equal to zero,
    so C[q] = 0 and the Heun step leaves q unchanged: FP64 keeps every field bit for bit; mixed
    precision keeps q bit for bit and pi = Pi = u^i = 0 exactly, with e and u^tau within an FP32
    ulp or two (its root-find restarts from the FP32 copy of e and stops within its tolerance)."""
    from paper_1608_06577_gb300 import KT, KT_INV_CONFORMAL, KT_MIXED
    p = Problem(name="rest", nx=40, ny=13, neta=9, dx=0.1, dy=0.1, deta=0.1, dtau=0.01, tau0=1.0, nsteps=20,
                coords="cartesian", bc="periodic", theta=1.0, eos=baseline_eos, eta_over_s=("const", 0.2, 0, 1),
                zeta_over_s=("gauss", 0.1, 0.17 / HBARC, 0.03 / HBARC), tau_relax_min=0.01)
    p.e = np.full(p.ncells, 5.0 / HBARC)
    p.u = np.zeros((3, p.ncells))
    p.pi = np.zeros((10, p.ncells))
    p.Pi = np.zeros(p.ncells)
    kw = {"fp64": {}, "mixed": {"precision": KT_MIXED},
          "conformal": {"precision": KT_MIXED, "inversion": KT_INV_CONFORMAL}}[mode]
    kt = KT(p, **kw)
    kt.set_problem_state()
    a = kt.get_state()
    kt.step(20)
    b = kt.get_state()
    assert kt.stats()["status"] == 0
    assert np.array_equal(a["q"], b["q"])
    if mode == "fp64":
        for f in ("e", "u", "pi", "Pi"):
            assert np.array_equal(a[f], b[f]), f
    else:
        assert not np.any(b["pi"]) and not np.any(b["Pi"]) and not np.any(b["u"][1:])
        assert np.max(np.abs(b["e"] / a["e"] - 1)) <= 2.4e-7
        assert np.max(np.abs(b["u"][0] - 1)) <= 2.4e-7


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_sod_fp64_parity(axis):
    p = sod_problem(nx=64, dx=0.1, t_end=0.5, axis=axis)
    g, r, _ = run_pair(p, p.nsteps)
    assert_parity(g, r)


def test_milne_flow_with_u_eta_and_shear(baseline_eos):
    """Hotspots with an initial longitudinal flow and shear stress exercise every source term."""
    p = hotspot_problem(nx=24, ny=20, neta=12, nhot=8, seed=5, r_max=0.8, eos_table=baseline_eos)
    X, Y, Z = p.coords_xyz()
    p.u = np.stack([0.1 * np.tanh(X).ravel(), -0.05 * np.tanh(Y).ravel(), (0.3 * np.tanh(Z) / p.tau0).ravel()])
    rng = np.random.default_rng(1)
    pi = np.zeros((10, p.ncells))
    pi[4] = 0.01 * p.e * (1 + 0.1 * rng.normal(size=p.ncells))
    pi[7] = -pi[4]
    p.pi = pi
    p.Pi = -0.01 * p.e
    p.u_prev = p.u * 0.99
    g, r, _ = run_pair(p, 10)
    assert_parity(g, r)


def test_step_counts_and_graph_paths_agree(baseline_eos):
    """Graph replay (3-step cycles) and direct launches give identical bits."""
    from paper_1608_06577_gb300 import KT
    p = hotspot_problem(nx=20, ny=20, neta=8, nhot=6, seed=9, r_max=0.8, eos_table=baseline_eos)
    a = KT(p, use_graph=True)
    a.set_problem_state()
    a.step(7)
    b = KT(p, use_graph=False)
    b.set_problem_state()
    for _ in range(7):
        b.step(1)
    ga, gb = a.get_state(), b.get_state()
    for f in FIELDS:
        assert np.array_equal(ga[f], gb[f]), f


def test_fp64_division_within_one_ulp():
    """The stencil's FP64 division (Newton-Raphson reciprocal from a single-precision seed, one
    quotient correction) against the correctly rounded a / b: at most one unit in the last place
    over random operands spanning its fast range 2^-125 <= b < 2^125, at the range's edges, and
    for operands outside it (IEEE division there: exact)."""
    import ctypes as C
    import torch
    from paper_1608_06577_gb300 import binding
    L = binding.load_library()
    L.kt_selftest_div.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_longlong, C.c_void_p]
    rng = np.random.default_rng(7)
    n = 1 << 20
    b = np.ldexp(rng.uniform(1.0, 2.0, n), rng.integers(-125, 125, n))
    a = np.ldexp(rng.uniform(1.0, 2.0, n), rng.integers(-500, 500, n)) * rng.choice([-1.0, 1.0], n)
    edges_b = [2.0 ** -125, np.nextafter(2.0 ** -125, 1.0), np.nextafter(2.0 ** 125, 0.0), 1.0,
               np.nextafter(1.0, 2.0), np.nextafter(2.0, 1.0), 3.0, 2.0 ** 125, 2.0 ** 200, 2.0 ** -126,
               -1.5, 1e-300]
    edges_a = [1.0, -1.0, np.nextafter(1.0, 2.0), 1.0 / 3.0, 1e-200, 7.0, 1e100, 0.0, -0.0, 2.5, 4.0, 1e-10]
    a = np.concatenate([a, edges_a])
    b = np.concatenate([b, edges_b])
    ta, tb = torch.as_tensor(a, device="cuda"), torch.as_tensor(b, device="cuda")
    tq = torch.empty_like(ta)
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.kt_selftest_div(C.c_void_p(ta.data_ptr()), C.c_void_p(tb.data_ptr()), C.c_void_p(tq.data_ptr()),
                             a.size, st) == 0
    q = tq.cpu().numpy()
    ref = a / b
    ulp = np.spacing(np.abs(ref))
    err = np.abs(q - ref) / np.where(ref != 0, ulp, 1.0)
    fast = (b >= 2.0 ** -125) & (b < 2.0 ** 125)
    print("vdiv: max error", float(err[fast].max()), "ulp over", int(fast.sum()), "operands")
    assert float(err[fast].max()) <= 1.0
    assert np.array_equal(q[~fast], ref[~fast])


def test_integer_pipe_conversions():
    """The kernels' double -> float conversions done with integer instructions: the rounded one
    (stored FP32 copies of q, e, P0, u) equals IEEE round-to-nearest-even (numpy's float32 cast)
    over random doubles of the float range, exact halfway cases, values that round up into the
    next binade and to infinity, with magnitudes below 2^-126 flushed to zero and non-finite
    inputs giving infinity; the truncating one (features, Newton step lengths, interval guesses)
    equals the mantissa cut to 23 bits."""
    import ctypes as C
    import torch
    from paper_1608_06577_gb300 import binding
    L = binding.load_library()
    L.kt_selftest_cvt.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_longlong, C.c_void_p]
    rng = np.random.default_rng(11)
    n = 1 << 20
    x = np.ldexp(rng.uniform(1.0, 2.0, n), rng.integers(-126, 128, n)) * rng.choice([-1.0, 1.0], n)
    f = rng.uniform(1.0, 2.0, 4096).astype(np.float32).astype(np.float64)
    ulp = np.spacing(f.astype(np.float32)).astype(np.float64)
    ties = np.concatenate([f + 0.5 * ulp, f - 0.5 * np.spacing(f.astype(np.float32) - ulp).astype(np.float64)])
    edges = np.array([0.0, -0.0, 1.0, -1.0, 2.0 ** -126, np.nextafter(2.0 ** -126, 0.0), 2.0 ** -127, 1e-300,
                      3.4028234663852886e38, 3.4028235677973366e38, 1e39, np.inf, -np.inf, np.nan,
                      np.nextafter(2.0, 1.0), 1.9999999403953552, 1.99999997019767761230])
    x = np.concatenate([x, ties, -ties, edges])
    tx = torch.as_tensor(x, device="cuda")
    rn = torch.empty(x.size, dtype=torch.float32, device="cuda")
    rz = torch.empty_like(rn)
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.kt_selftest_cvt(C.c_void_p(tx.data_ptr()), C.c_void_p(rn.data_ptr()), C.c_void_p(rz.data_ptr()),
                             x.size, st) == 0
    rn, rz = rn.cpu().numpy(), rz.cpu().numpy()
    with np.errstate(over="ignore", invalid="ignore"):
        ref = x.astype(np.float32)
    small = np.abs(x) < 2.0 ** -126
    ref[small] = np.copysign(0.0, x[small]).astype(np.float32)
    ref[~np.isfinite(x)] = np.copysign(np.inf, np.nan_to_num(x[~np.isfinite(x)], nan=1.0))
    assert np.array_equal(rn.view(np.uint32), ref.view(np.uint32))
    fin = np.isfinite(x) & (np.abs(x) < 2.0 ** 128)
    b = x[fin].view(np.uint64)
    tr = ((b >> 32) & np.uint64(0x80000000)) | np.where((b & np.uint64(0x7fffffffffffffff)) >= np.uint64(897 << 52),
                                                          (((b & np.uint64(0x7fffffffffffffff)) - np.uint64(896 << 52))
                                                           >> np.uint64(29)) & np.uint64(0x7fffffff), np.uint64(0))
    assert np.array_equal(rz[fin].view(np.uint32), tr.astype(np.uint32))


@pytest.mark.parametrize("precision", [0, 1])
def test_cfl_max_speed_matches_oracle(precision, baseline_eos):
    """The CFL diagnostic kt_stats.max_speed (the largest local speed a of Eq. (ax) over all faces
    of the steps of one kt_step call, eta speeds times tau) against the oracle's record of the
    same steps.  The GPU keeps it in FP32 (FP64 mode rounds once; mixed precision computes the
    speeds in FP32)."""
    from paper_1608_06577_gb300 import KT
    for p in (gubser_problem(nx=24, ny=20, neta=6, nsteps=8),
              hotspot_problem(nx=20, ny=18, neta=10, nhot=6, seed=3, r_max=0.8, eos_table=baseline_eos)):
        kt = KT(p, precision=precision)
        kt.set_problem_state()
        kt.step(8)
        o = oracle.Oracle(p)
        assert o.step(8) == 0
        st = kt.stats()
        a, b = st["max_speed"], o.max_speed()
        print(p.name, "max speed GPU", a, "oracle", b)
        assert 0.0 < b < 1.0
        assert abs(a - b) <= (1e-7 if precision == 0 else 1e-5) * b
        # the state's extrema in kt_stats: e in the stored precision, rounded to float
        e = kt.get_state(fields=("e",))["e"]
        assert st["e_min"] == float(np.float32(e.min())) and st["e_max"] == float(np.float32(e.max()))
        assert st["reg_min"] == float(np.min(kt.diagnostics()["regulation"]))


@pytest.mark.parametrize("mode", ["fp64", "learned", "learned_pi32"])
def test_checkpoint_restart_is_bit_exact(mode, baseline_eos):
    """Sec. 4.3 writes the state out every m steps and continues from it: 10 steps equal 5 steps,
    kt_get_checkpoint, kt_set_checkpoint into a fresh context, and 5 more steps, bit for bit in
    every field (q, e, u, pi, Pi) and in the regulation record, after the regulator has acted."""
    from paper_1608_06577_gb300 import KT, KT_INV_LEARNED, KT_MIXED
    from paper_1608_06577_gb300.learned import init_params
    p = hotspot_problem(nx=24, ny=20, neta=10, nhot=6, seed=9, r_max=0.8, eos_table=baseline_eos)
    kw = {} if mode == "fp64" else {"precision": KT_MIXED, "inversion": KT_INV_LEARNED,
                                    "mlp_weights": init_params(3), "pi_fp32": mode.endswith("pi32")}
    a = KT(p, **kw)
    a.set_problem_state()
    a.step(5)
    tau5, ck = a.get_checkpoint()
    a.step(5)
    ref = a.get_state()
    b = KT(p, **kw)
    b.set_checkpoint(tau5, ck)
    tau_b, ck_b = b.get_checkpoint()
    assert tau_b == tau5 and np.array_equal(ck_b, ck)  # the round trip itself is exact
    b.step(5)
    got = b.get_state()
    for f in FIELDS:
        assert np.array_equal(got[f], ref[f]), f
    assert got["tau"] == ref["tau"]
    assert np.array_equal(b.diagnostics()["regulation"], a.diagnostics()["regulation"])
    assert np.min(a.diagnostics()["regulation"]) < 1.0  # the regulator acted


def test_invalid_state_rejected():
    """kt_set_state refuses non-finite input and states that admit no inversion (host-side
    injection: a bulk pressure Pi = -4e in a cell moving with u^x = 1, so that e + P < 0 and
    E = (e + P) (u^tau)^2 - P < 0)."""
    from paper_1608_06577_gb300 import KT, KTError
    p = gubser_problem(nx=8, ny=8, neta=2)
    kt = KT(p)
    e = p.e.copy()
    e[3] = np.nan
    with pytest.raises(KTError, match="KT_ERR_STATE.*non-finite"):
        kt.set_state(p.tau0, e, p.u, p.pi, p.Pi)
    u = np.zeros((3, p.ncells))
    u[0, 5] = 1.0
    Pi = np.zeros(p.ncells)
    Pi[5] = -4.0 * p.e[5]
    with pytest.raises(KTError, match="KT_ERR_STATE.*eInferred"):
        kt.set_state(p.tau0, p.e, u, None, Pi)
    kt.set_state(p.tau0, p.e, p.u, p.pi, p.Pi)  # the context accepts a valid state afterwards
    kt.step(1)


@pytest.mark.parametrize("pi_fp32", [False, True])
def test_mixed_mode_error_after_100_steps(pi_fp32, baseline_eos):
    """Mixed precision (FP32 reconstruction, fluxes and sources; FP64 Heun accumulation and
    FP64 root-find) against the FP64 oracle after 100 steps: pointwise relative error in e
    <= 1e-4 on every cell; the per-field max-norm errors are reported.  pi_fp32: the storage
    variant with pi^{mu nu} and Pi stored and Heun-summed in FP32 (T^{tau mu} in FP64)."""
    p = hotspot_problem(nx=40, ny=36, neta=20, nhot=10, seed=4, r_max=1.2, eos_table=baseline_eos)
    g, r, _ = run_pair(p, 100, precision=1, pi_fp32=pi_fp32)
    rel_e = np.max(np.abs(g["e"] / r["e"] - 1))
    errs = field_errors(g, r)
    print(f"mixed mode (pi fp32: {pi_fp32}) after 100 steps: max rel err e", rel_e,
          {k: f"{v:.2e}" for k, v in errs.items()})
    assert rel_e < 1e-4
    assert errs["e[0]"] < 1e-4 and errs["q[0]"] < 1e-4


@pytest.mark.parametrize("shape", [(20, 18, 10), (33, 9, 7)])
def test_face_inversion_fp64_parity(shape, baseline_eos):
    """KT_IFACE_INVERT (face velocities from root-finds of the extrapolated states, the literal
    reading of Sec. 3.1) against the oracle with the same option: 1e-12 per field after 10 steps."""
    from dataclasses import replace
    nx, ny, nz = shape
    p = replace(hotspot_problem(nx=nx, ny=ny, neta=nz, nhot=6, seed=9, r_max=1.0, eos_table=baseline_eos),
                iface="invert")
    g, r, _ = run_pair(p, 10)
    assert_parity(g, r)


def test_face_inversion_mixed_error(baseline_eos):
    """Mixed precision with FP32 face root-finds against the FP64 oracle (same option): pointwise
    relative error in e <= 1e-4 after 40 steps; and the option changes the result (it is not the
    default reconstruction)."""
    from dataclasses import replace
    p = replace(hotspot_problem(nx=28, ny=24, neta=12, nhot=8, seed=6, r_max=1.0, eos_table=baseline_eos),
                iface="invert")
    g, r, _ = run_pair(p, 40, precision=1)
    rel_e = np.max(np.abs(g["e"] / r["e"] - 1))
    print("face inversion, mixed, 40 steps: max rel err e", rel_e)
    assert rel_e < 1e-4
    g2, _, _ = run_pair(replace(p, iface="recon"), 40, precision=1)
    assert np.max(np.abs(g2["e"] / g["e"] - 1)) > 1e-8


def test_lattice_eos_and_paper_zeta_fp64_parity():
    """The lattice EOS of Sec. 2.3 with zeta/s of Eq. (zetas) (T_c = 200 MeV): hotspots and the
    nonconformal Bjorken setup of Sec. 5.5, FP64 against the oracle to 1e-12 per field."""
    from workload.eos import lattice_table
    p = hotspot_problem(nx=22, ny=20, neta=8, nhot=6, seed=8, r_max=1.0, eta_over_s=0.2, zeta="paper",
                        eos_table=lattice_table())
    g, r, _ = run_pair(p, 10)
    assert_parity(g, r)
    b = bjorken_problem(T0_gev=0.6, tau0=0.25, dtau=0.004, nsteps=10, eos="lattice", zeta="paper", eta_over_s=0.2)
    g, r, _ = run_pair(b, 10)
    assert_parity(g, r)
    assert r["Pi"][0] > 0


def test_lattice_eos_mixed_error():
    """The same hotspots in mixed precision: pointwise relative error in e <= 1e-4 after 40 steps."""
    from workload.eos import lattice_table
    p = hotspot_problem(nx=22, ny=20, neta=8, nhot=6, seed=8, r_max=1.0, eta_over_s=0.2, zeta="paper",
                        eos_table=lattice_table())
    g, r, _ = run_pair(p, 40, precision=1)
    rel_e = np.max(np.abs(g["e"] / r["e"] - 1))
    print("lattice EOS, mixed, 40 steps: max rel err e", rel_e)
    assert rel_e < 1e-4


@pytest.mark.parametrize("precision", [0, 1])
def test_diagnostics_parity(precision, baseline_eos):
    """kt_get_diagnostics (validity diagnostics of Sec. 7) against the oracle after 6 steps on a
    hotspot grid: FP64 to 1e-11 of each diagnostic's max (the regulation factor is stored in FP32,
    so to 1e-7), mixed precision to 1e-4."""
    from paper_1608_06577_gb300 import KT
    p = hotspot_problem(nx=22, ny=18, neta=8, nhot=6, seed=10, r_max=1.0, eos_table=baseline_eos)
    kt = KT(p, precision=precision)
    kt.set_problem_state()
    kt.step(6)
    g = kt.diagnostics()
    o = oracle.Oracle(p)
    assert o.step(6) == 0
    r = o.diagnostics()
    tol = 1e-11 if precision == 0 else 1e-4
    for k in r:
        scale = max(np.max(np.abs(r[k])), 1e-300)
        err = np.max(np.abs(g[k] - r[k])) / scale
        t = max(tol, 1e-7) if k == "regulation" else tol
        assert err <= t, (k, err)
    assert np.min(g["regulation"]) < 1.0


def test_bounded_wait_times_out_and_context_survives(baseline_eos):
    """Failure detection without a GPU fault: a wait on an mbarrier that nothing arms gives up
    after its poll limit and the host sees KT_ERR_TIMEOUT; the same context then steps normally
    and still matches the oracle."""
    from paper_1608_06577_gb300 import KT
    from paper_1608_06577_gb300.binding import ERRORS
    p = hotspot_problem(nx=20, ny=16, neta=6, nhot=4, seed=2, r_max=0.8, eos_table=baseline_eos)
    kt = KT(p, precision=1)
    kt.set_problem_state()
    rc = kt.L.kt_selftest_wait(kt.ctx, 1000)
    assert rc == -8, ERRORS.get(rc, rc)  # KT_ERR_TIMEOUT
    assert b"gave up" in kt.L.kt_last_error(kt.ctx)
    kt.step(5)
    assert kt.stats()["status"] == 0
    o = oracle.Oracle(p)
    assert o.step(5) == 0
    assert np.max(np.abs(kt.get_state()["e"] / o.get_state()["e"] - 1)) < 1e-4
