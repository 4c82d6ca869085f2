"""ctypes wrapper of the plain FP64 CPU oracle (oracle/kt_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the benchmark's CPU-baseline
leg use it to check the CUDA path.  It shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "libkt_oracle.so")
SRC = os.path.join(HERE, "kt_oracle.c")
FLOPS_LIB = os.path.join(HERE, "libkt_oracle_flops.so")
FLOPS_SRC = os.path.join(HERE, "kt_oracle_flops.cpp")
FLOP_KINDS = ("add", "mul", "div", "sqrt", "transcendental", "compare")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FMA contraction, OpenMP over the (eta, y) rows)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "kt_oracle.h"))):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC",
                               "-shared", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


def build_flops(force: bool = False) -> str:
    """Compile the operation-counting oracle (kt_oracle.c with the counted scalar of flops.hpp in
    place of double; single-threaded, no FMA contraction, so it reproduces the plain oracle)."""
    srcs = [SRC, FLOPS_SRC, os.path.join(HERE, "flops.hpp"), os.path.join(HERE, "kt_oracle.h")]
    if force or not os.path.exists(FLOPS_LIB) or os.path.getmtime(FLOPS_LIB) < max(map(os.path.getmtime, srcs)):
        tmp = FLOPS_LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared",
                               "-Wno-return-type-c-linkage", "-o", tmp, FLOPS_SRC, "-lm"])
        os.replace(tmp, FLOPS_LIB)
    return FLOPS_LIB


class _Params(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("neta", C.c_int),
        ("dx", C.c_double), ("dy", C.c_double), ("deta", C.c_double), ("dtau", C.c_double),
        ("coords", C.c_int), ("bc", C.c_int), ("theta", C.c_double),
        ("eos_kind", C.c_int), ("eos_a", C.c_double), ("eos_n", C.c_int),
        ("eos_e", C.POINTER(C.c_double)), ("eos_p", C.POINTER(C.c_double)),
        ("eos_cs2", C.POINTER(C.c_double)), ("eos_T", C.POINTER(C.c_double)),
        ("eos_lndelta", C.POINTER(C.c_double)),
        ("eta_kind", C.c_int), ("eta_c", C.c_double * 3),
        ("zeta_kind", C.c_int), ("zeta_c", C.c_double * 3),
        ("tau_pipi_on", C.c_int), ("regulate", C.c_int), ("rho_max", C.c_double), ("xi0", C.c_double),
        ("e_min", C.c_double), ("tau_relax_min", C.c_double), ("iface", C.c_int),
    ]


_libs = {}


def lib(flops: bool = False):
    """The plain oracle library, or (flops=True) the operation-counting build of it."""
    if flops not in _libs:
        L = C.CDLL(build_flops() if flops else build())
        dp = C.POINTER(C.c_double)
        L.ko_create.restype = C.c_void_p
        L.ko_create.argtypes = [C.POINTER(_Params)]
        L.ko_free.argtypes = [C.c_void_p]
        L.ko_set_state.argtypes = [C.c_void_p, C.c_double, dp, dp, dp, dp, dp]
        L.ko_set_state_q.argtypes = [C.c_void_p, C.c_double, dp, dp, dp, dp]
        L.ko_coefficients.argtypes = [C.c_void_p, C.c_double, dp]
        L.ko_diagnostics.argtypes = [C.c_void_p, dp]
        L.ko_step.argtypes = [C.c_void_p, C.c_int]
        L.ko_get_state.argtypes = [C.c_void_p, dp, dp, dp, dp, dp, dp]
        L.ko_rhs.argtypes = [C.c_void_p, dp]
        L.ko_set_threads.argtypes = [C.c_int]
        L.ko_max_speed.restype = C.c_double
        L.ko_max_speed.argtypes = [C.c_void_p]
        L.ko_minmod3.restype = C.c_double
        L.ko_minmod3.argtypes = [C.c_double] * 3
        L.ko_eos.argtypes = [C.c_void_p, C.c_double, dp]
        L.ko_invert.argtypes = [C.c_void_p, C.c_double, dp, dp]
        L.ko_tensor_terms.argtypes = [C.c_void_p, C.c_double, dp, dp, dp, dp]
        L.ko_regulator_factor.restype = C.c_double
        L.ko_regulator_factor.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double, dp, dp, C.c_double]
        if flops:
            L.ko_flops_read.argtypes = [C.POINTER(C.c_ulonglong), C.c_int]
        _libs[flops] = L
    return _libs[flops]


def read_flops(reset: bool = True) -> dict:
    """Operation counts of the counting build since the last reset, by kind."""
    out = (C.c_ulonglong * len(FLOP_KINDS))()
    lib(True).ko_flops_read(out, int(reset))
    return dict(zip(FLOP_KINDS, [int(x) for x in out]))


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _kind(k):
    return {"const": 0, "gauss": 1, "paper": 2}[k]


class Oracle:
    """One oracle context for a workload.Problem."""

    def __init__(self, prob, threads: int | None = None, flops: bool = False):
        L = lib(flops)
        self.L = L
        if threads is not None:
            L.ko_set_threads(int(threads))
        self.prob = prob
        p = _Params()
        p.nx, p.ny, p.neta = prob.nx, prob.ny, prob.neta
        p.dx, p.dy, p.deta, p.dtau = prob.dx, prob.dy, prob.deta, prob.dtau
        p.coords = 0 if prob.coords == "milne" else 1
        p.bc = 0 if prob.bc == "copy" else 1
        p.theta = prob.theta
        self._keep = []
        if isinstance(prob.eos, tuple):
            p.eos_kind, p.eos_a = 0, float(prob.eos[1])
        else:
            t = prob.eos
            p.eos_kind, p.eos_n = 1, t.n
            arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (t.e, t.p, t.cs2, t.T, t.lndelta)]
            self._keep += arrs
            p.eos_e, p.eos_p, p.eos_cs2, p.eos_T, p.eos_lndelta = [_ptr(a) for a in arrs]
        p.eta_kind = _kind(prob.eta_over_s[0])
        p.eta_c[:] = [float(x) for x in prob.eta_over_s[1:4]]
        p.zeta_kind = _kind(prob.zeta_over_s[0])
        p.zeta_c[:] = [float(x) for x in prob.zeta_over_s[1:4]]
        p.tau_pipi_on = int(bool(prob.tau_pipi_on))
        p.regulate = int(bool(prob.regulate))
        p.rho_max, p.xi0 = prob.rho_max, prob.xi0
        p.e_min, p.tau_relax_min = prob.e_min, prob.tau_relax_min
        p.iface = 0 if prob.iface == "recon" else 1
        self._params = p
        self.ctx = L.ko_create(C.byref(p))
        if not self.ctx:
            raise ValueError("ko_create failed")
        self.set_state(prob.tau0, prob.e, prob.u, prob.pi, prob.Pi, prob.u_prev)

    def __del__(self):
        try:
            if getattr(self, "ctx", None):
                self.L.ko_free(self.ctx)
                self.ctx = None
        except Exception:
            pass

    def set_state(self, tau, e, u=None, pi=None, Pi=None, u_prev=None):
        conv = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float64)  # noqa: E731
        e, u, pi, Pi, u_prev = map(conv, (e, u, pi, Pi, u_prev))
        self._state_keep = (e, u, pi, Pi, u_prev)
        return self.L.ko_set_state(self.ctx, float(tau), _ptr(e), _ptr(u), _ptr(pi), _ptr(Pi), _ptr(u_prev))

    def set_state_q(self, tau, q, e, u, u_prev=None):
        """Restart from evolved variables: q [15, cells], e [cells], u [4, cells] (with u^tau),
        u_prev [4, cells]."""
        conv = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float64)  # noqa: E731
        q, e, u, u_prev = map(conv, (q, e, u, u_prev))
        self._state_keep = (q, e, u, u_prev)
        return self.L.ko_set_state_q(self.ctx, float(tau), _ptr(q), _ptr(e), _ptr(u), _ptr(u_prev))

    def step(self, n=1) -> int:
        return self.L.ko_step(self.ctx, int(n))

    def max_speed(self) -> float:
        """The CFL diagnostic of the last step() call: the largest local speed a of Eq. (ax) over
        all faces of its stages, eta speeds times tau (Milne)."""
        return float(self.L.ko_max_speed(self.ctx))

    def get_state(self):
        N = self.prob.ncells
        tau = C.c_double()
        e = np.empty(N); u = np.empty((4, N)); pi = np.empty((10, N)); Pi = np.empty(N); q = np.empty((15, N))
        self.L.ko_get_state(self.ctx, C.byref(tau), _ptr(e), _ptr(u), _ptr(pi), _ptr(Pi), _ptr(q))
        return {"tau": tau.value, "e": e, "u": u, "pi": pi, "Pi": Pi, "q": q}

    def rhs(self):
        out = np.empty((15, self.prob.ncells))
        self.L.ko_rhs(self.ctx, _ptr(out))
        return out

    DIAGNOSTICS = ("Kn_theta_pi", "Kn_theta_Pi", "Rinv_pi", "Rinv_Pi", "R2inv_pi", "R2inv_Pi", "regulation")

    def diagnostics(self):
        """The validity diagnostics of Sec. 7 at the current state, as a dict of [cells] arrays."""
        out = np.empty((7, self.prob.ncells))
        self.L.ko_diagnostics(self.ctx, _ptr(out))
        return dict(zip(self.DIAGNOSTICS, out))

    def coefficients(self, T):
        """(eta/s, zeta/s) at temperature T (fm^-1)."""
        out = np.empty(2)
        self.L.ko_coefficients(self.ctx, float(T), _ptr(out))
        return out[0], out[1]

    # single-formula entry points
    def eos(self, e):
        out = np.empty(3)
        self.L.ko_eos(self.ctx, float(e), _ptr(out))
        return out

    def invert(self, tau, q15):
        q15 = np.ascontiguousarray(q15, dtype=np.float64)
        out = np.empty(6)
        st = self.L.ko_invert(self.ctx, float(tau), _ptr(q15), _ptr(out))
        return st, out

    def tensor_terms(self, tau, u4, du16, pi16):
        out = np.empty(101)
        a = [np.ascontiguousarray(x, dtype=np.float64).ravel() for x in (u4, du16, pi16)]
        self.L.ko_tensor_terms(self.ctx, float(tau), _ptr(a[0]), _ptr(a[1]), _ptr(a[2]), _ptr(out))
        names = ["sigma", "omega", "I1", "I3", "I4", "Gpi"]
        d = {"theta": out[0], "Du": out[1:5]}
        for k, nm in enumerate(names):
            d[nm] = out[5 + 16 * k: 5 + 16 * (k + 1)].reshape(4, 4)
        return d

    def regulator_factor(self, tau, e, P0, u4, pi16, Pi):
        a = [np.ascontiguousarray(x, dtype=np.float64).ravel() for x in (u4, pi16)]
        return self.L.ko_regulator_factor(self.ctx, float(tau), float(e), float(P0), _ptr(a[0]), _ptr(a[1]),
                                          float(Pi))


def minmod3(x, y, z) -> float:
    return lib().ko_minmod3(float(x), float(y), float(z))


def set_threads(n: int) -> int:
    return lib().ko_set_threads(int(n))
