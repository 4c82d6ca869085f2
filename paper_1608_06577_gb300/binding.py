"""ctypes binding of libkt (include/kt.h): argument marshalling only.

Device memory comes from torch (the state arena is one torch uint8 tensor) and work is
enqueued on torch's current CUDA stream.  Loading fails loudly when libkt.so is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None

KT_OK = 0
ERRORS = {-1: "KT_ERR_ARG", -2: "KT_ERR_CUDA", -3: "KT_ERR_OOM", -4: "KT_ERR_EOS", -5: "KT_ERR_STATE",
          -6: "KT_ERR_INVERSION", -7: "KT_ERR_NONFINITE", -8: "KT_ERR_TIMEOUT"}
KT_FP64, KT_MIXED = 0, 1
KT_INV_PLAIN, KT_INV_LEARNED, KT_INV_CONFORMAL = 0, 1, 2
KT_STORE_FP64, KT_STORE_PI_FP32 = 0, 1
MLP_NPARAM = 32 * 6 + 32 + 32 * 32 + 32 + 32 + 1


class KTError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("neta", C.c_int)]


class Eos(C.Structure):
    _fields_ = [("kind", C.c_int), ("a", C.c_double), ("n", C.c_int),
                ("e", C.POINTER(C.c_double)), ("p", C.POINTER(C.c_double)), ("cs2", C.POINTER(C.c_double)),
                ("T", C.POINTER(C.c_double)), ("lndelta", C.POINTER(C.c_double))]


class Coef(C.Structure):
    _fields_ = [("kind", C.c_int), ("c0", C.c_double), ("c1", C.c_double), ("c2", C.c_double)]


class Options(C.Structure):
    _fields_ = [("theta_limiter", C.c_double), ("coords", C.c_int), ("bc", C.c_int), ("precision", C.c_int),
                ("inversion", C.c_int), ("tau_pipi_on", C.c_int), ("regulate", C.c_int), ("rho_max", C.c_double),
                ("xi0", C.c_double), ("e_min", C.c_double), ("tau_relax_min", C.c_double),
                ("stream", C.c_void_p), ("arena", C.c_void_p), ("arena_bytes", C.c_size_t),
                ("mlp_weights", C.POINTER(C.c_float)), ("use_graph", C.c_int), ("autotune", C.c_int),
                ("iface", C.c_int), ("pi_storage", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("tau", C.c_double), ("steps", C.c_longlong), ("max_speed", C.c_float), ("status", C.c_uint),
                ("newton_iters", C.c_longlong), ("fallbacks", C.c_longlong), ("regulated", C.c_longlong),
                ("e_min", C.c_double), ("e_max", C.c_double), ("reg_min", C.c_double)]


def lib_path() -> str:
    return os.path.join(HERE, "libkt.so")


def load_library():
    global _LIB
    if _LIB is not None:
        return _LIB
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built; run paper_1608_06577_gb300.build.build() "
                           "(libkt has no CPU fallback)")
    L = C.CDLL(path)
    dp, vp = C.POINTER(C.c_double), C.c_void_p
    L.kt_options_default.argtypes = [C.POINTER(Options)]
    L.kt_state_bytes.argtypes = [C.POINTER(Grid), C.POINTER(Eos), C.POINTER(Options), C.POINTER(C.c_size_t)]
    L.kt_init.argtypes = [C.POINTER(vp), C.POINTER(Grid), C.c_double, C.c_double, C.c_double, C.POINTER(Eos),
                          C.POINTER(Coef), C.POINTER(Coef), C.POINTER(Options)]
    L.kt_set_state.argtypes = [vp, C.c_double, vp, vp, vp, vp, vp, C.c_int]
    L.kt_step.argtypes = [vp, C.c_int]
    L.kt_get_state.argtypes = [vp, dp, vp, vp, vp, vp, vp, C.c_int]
    L.kt_get_stats.argtypes = [vp, C.POINTER(Stats)]
    L.kt_last_error.restype = C.c_char_p
    L.kt_last_error.argtypes = [vp]
    L.kt_free.argtypes = [vp]
    L.kt_free.restype = None
    L.kt_state_bytes_batch.argtypes = [C.c_int, C.POINTER(Grid), C.POINTER(Eos), C.POINTER(Options),
                                       C.POINTER(C.c_size_t)]
    L.kt_init_batch.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(Grid), C.c_double, C.c_double, C.c_double,
                                C.POINTER(Eos), C.POINTER(Coef), C.POINTER(Coef), C.POINTER(Options)]
    L.kt_set_state_event.argtypes = [vp, C.c_int, C.c_double, vp, vp, vp, vp, vp, C.c_int]
    L.kt_get_state_event.argtypes = [vp, C.c_int, dp, vp, vp, vp, vp, vp, C.c_int]
    L.kt_get_tuning.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_float), C.POINTER(C.c_int)]
    L.kt_set_tuning.argtypes = [vp, C.c_int]
    L.kt_time_kernels.argtypes = [vp, C.c_int, C.POINTER(C.c_float), C.POINTER(C.c_int)]
    L.kt_get_diagnostics.argtypes = [vp, C.c_int, vp, C.c_int]
    L.kt_selftest_wait.argtypes = [vp, C.c_uint]
    L.kt_get_checkpoint.argtypes = [vp, C.c_int, dp, vp, C.c_int]
    L.kt_set_checkpoint.argtypes = [vp, C.c_int, C.c_double, vp, C.c_int]
    _LIB = L
    return L


def _dptr(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


def _coef(t):
    kind = {"const": 0, "gauss": 1, "paper": 2}[t[0]]
    return Coef(kind, float(t[1]), float(t[2]), float(t[3]))


class KT:
    """One libkt context for a problem description (a workload.Problem or a compatible object),
    or for a batch: a list of problems that differ only in grid and initial state."""

    def __init__(self, prob, precision: int = KT_FP64, inversion: int = KT_INV_PLAIN, mlp_weights=None,
                 use_graph: bool = True, device_arena: bool = True, autotune: bool = True, pi_fp32: bool = False):
        import torch
        self.torch = torch
        L = load_library()
        probs = list(prob) if isinstance(prob, (list, tuple)) else [prob]
        self.probs = probs
        self.prob = probs[0]
        prob = probs[0]
        self.nev = len(probs)
        self.ncells_ev = [p.nx * p.ny * p.neta for p in probs]
        self.ncells = self.ncells_ev[0]
        grids = (Grid * self.nev)(*[Grid(p.nx, p.ny, p.neta) for p in probs])
        o = Options()
        L.kt_options_default(C.byref(o))
        o.theta_limiter = prob.theta
        o.coords = 0 if prob.coords == "milne" else 1
        o.bc = 0 if prob.bc == "copy" else 1
        o.precision = precision
        o.inversion = inversion
        o.tau_pipi_on = int(bool(prob.tau_pipi_on))
        o.regulate = int(bool(prob.regulate))
        o.iface = 1 if getattr(prob, "iface", "recon") == "invert" else 0
        o.rho_max, o.xi0 = prob.rho_max, prob.xi0
        o.e_min, o.tau_relax_min = prob.e_min, prob.tau_relax_min
        o.use_graph = int(bool(use_graph))
        o.autotune = int(bool(autotune))
        o.pi_storage = KT_STORE_PI_FP32 if pi_fp32 else KT_STORE_FP64
        self.stream = torch.cuda.current_stream()
        o.stream = C.c_void_p(self.stream.cuda_stream)
        self._keep = []
        if mlp_weights is not None:
            w = np.ascontiguousarray(mlp_weights, dtype=np.float32)
            assert w.size == MLP_NPARAM
            self._keep.append(w)
            o.mlp_weights = w.ctypes.data_as(C.POINTER(C.c_float))
        if isinstance(prob.eos, tuple):
            eos = Eos(0, float(prob.eos[1]), 0, None, None, None, None, None)
        else:
            t = prob.eos
            cols = [np.ascontiguousarray(a, dtype=np.float64) for a in (t.e, t.p, t.cs2, t.T, t.lndelta)]
            self._keep += cols
            P = C.POINTER(C.c_double)
            eos = Eos(1, 0.0, t.n, *[a.ctypes.data_as(P) for a in cols])
        if device_arena:
            nb = C.c_size_t()
            rc = L.kt_state_bytes_batch(self.nev, grids, C.byref(eos), C.byref(o), C.byref(nb))
            if rc != KT_OK:
                raise KTError(rc, "kt_state_bytes_batch")
            self.arena = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
            o.arena, o.arena_bytes = C.c_void_p(self.arena.data_ptr()), nb.value
        ce, cz = _coef(prob.eta_over_s), _coef(prob.zeta_over_s)
        ctx = C.c_void_p()
        rc = L.kt_init_batch(C.byref(ctx), self.nev, grids, prob.dx, prob.deta, prob.dtau, C.byref(eos), C.byref(ce),
                             C.byref(cz), C.byref(o))
        if rc != KT_OK:
            raise KTError(rc, "kt_init failed")
        self.ctx = ctx
        self.L = L

    def _check(self, rc, what):
        if rc != KT_OK:
            raise KTError(rc, f"{what}: {self.L.kt_last_error(self.ctx).decode()}")
        return rc

    def __del__(self):
        try:
            if getattr(self, "ctx", None):
                self.L.kt_free(self.ctx)
                self.ctx = None
        except Exception:
            pass

    # ----------------------------------------------------------------------- state
    def set_state(self, tau, e, u=None, pi=None, Pi=None, u_prev=None, event=0):
        """Host numpy arrays (physical cells, x fastest) or CUDA torch tensors."""
        torch = self.torch
        arrs = [e, u, pi, Pi, u_prev]
        on_dev = any(isinstance(a, torch.Tensor) and a.is_cuda for a in arrs if a is not None)
        if on_dev:
            torch.cuda.synchronize()  # inputs produced on torch's streams must be complete
        ptrs = []
        keep = []
        for a in arrs:
            if a is None:
                ptrs.append(None)
            elif on_dev:
                t = a.to(dtype=torch.float64).contiguous()
                keep.append(t)
                ptrs.append(C.c_void_p(t.data_ptr()))
            else:
                h = np.ascontiguousarray(a, dtype=np.float64)
                keep.append(h)
                ptrs.append(_dptr(h))
        rc = self.L.kt_set_state_event(self.ctx, int(event), float(tau), *ptrs, int(on_dev))
        return self._check(rc, "kt_set_state")

    def set_problem_state(self):
        for ev, p in enumerate(self.probs):
            self.set_state(p.tau0, p.e, p.u, p.pi, p.Pi, p.u_prev, event=ev)

    def step(self, n=1, check=True):
        rc = self.L.kt_step(self.ctx, int(n))
        if check:
            self._check(rc, "kt_step")
        return rc

    def get_state(self, fields=("e", "u", "pi", "Pi", "q"), event=0, out=None):
        """Host copies of the fields; `out` may hold preallocated float64 arrays (e.g. views of
        pinned memory) for some of them."""
        N = self.ncells_ev[event]
        given = out or {}
        out = {}
        shapes = {"e": (N,), "u": (4, N), "pi": (10, N), "Pi": (N,), "q": (15, N)}
        for f in ("e", "u", "pi", "Pi", "q"):
            if f in fields and f in given:
                a = given[f]
                if a.dtype != np.float64 or not a.flags.c_contiguous or a.shape != shapes[f]:
                    raise ValueError(f"out[{f!r}] must be a C-contiguous float64 array of shape {shapes[f]}")
                out[f] = a
            else:
                out[f] = np.empty(shapes[f]) if f in fields else None
        tau = C.c_double()
        rc = self.L.kt_get_state_event(self.ctx, int(event), C.byref(tau),
                                       *[_dptr(out[f]) for f in ("e", "u", "pi", "Pi", "q")], 0)
        self._check(rc, "kt_get_state")
        out["tau"] = tau.value
        return out

    def get_state_device(self, e=None, u=None, pi=None, Pi=None, q=None, event=0):
        """Copy into preallocated CUDA float64 tensors (any may be None)."""
        ptr = lambda t: None if t is None else C.c_void_p(t.data_ptr())  # noqa: E731
        self.torch.cuda.synchronize()
        tau = C.c_double()
        rc = self.L.kt_get_state_event(self.ctx, int(event), C.byref(tau), ptr(e), ptr(u), ptr(pi), ptr(Pi), ptr(q), 1)
        self._check(rc, "kt_get_state")
        return tau.value

    CHECKPOINT_ROWS = 41

    def get_checkpoint(self, event=0):
        """(tau, [41, cells] float64 host array): the complete evolved state (kt_get_checkpoint)."""
        buf = np.empty((self.CHECKPOINT_ROWS, self.ncells_ev[event]))
        tau = C.c_double()
        self._check(self.L.kt_get_checkpoint(self.ctx, int(event), C.byref(tau), _dptr(buf), 0), "kt_get_checkpoint")
        return tau.value, buf

    def set_checkpoint(self, tau, buf, event=0):
        """Continue from a checkpoint taken by get_checkpoint (kt_set_checkpoint)."""
        buf = np.ascontiguousarray(buf, dtype=np.float64)
        assert buf.shape == (self.CHECKPOINT_ROWS, self.ncells_ev[event])
        self._check(self.L.kt_set_checkpoint(self.ctx, int(event), float(tau), _dptr(buf), 0), "kt_set_checkpoint")

    def stats(self) -> dict:
        s = Stats()
        self._check(self.L.kt_get_stats(self.ctx, C.byref(s)), "kt_get_stats")
        return {k: getattr(s, k) for k, _ in Stats._fields_}

    def tuning(self) -> dict:
        blk = (C.c_int * 3)()
        grid = C.c_int()
        ms = (C.c_float * 64)()
        n = C.c_int(64)
        self._check(self.L.kt_get_tuning(self.ctx, blk, C.byref(grid), ms, C.byref(n)), "kt_get_tuning")
        return {"block": tuple(blk), "grid_blocks": grid.value, "candidate_ms": list(ms)[:n.value]}

    def set_tuning(self, candidate: int) -> None:
        """Use autotuner candidate `candidate` = 12 v + 2 s + g (layout v, tile shape s, grid variant
        g) from now on (kt_set_tuning)."""
        self._check(self.L.kt_set_tuning(self.ctx, int(candidate)), "kt_set_tuning")

    KERNEL_SLOTS = ("learned_start", "stage1_rhs", "stage1_update", "stage2_rhs", "stage2_update", "tau_advance")
    DIAGNOSTICS = ("Kn_theta_pi", "Kn_theta_Pi", "Rinv_pi", "Rinv_Pi", "R2inv_pi", "R2inv_Pi", "regulation")

    def diagnostics(self, event=0) -> dict:
        """The validity diagnostics of Sec. 7 at the current state (kt_get_diagnostics)."""
        out = np.empty((7, self.ncells_ev[event]))
        self._check(self.L.kt_get_diagnostics(self.ctx, int(event), _dptr(out), 0), "kt_get_diagnostics")
        return dict(zip(self.DIAGNOSTICS, out))

    def time_kernels(self, n_steps: int) -> dict:
        """Advances n_steps steps launch by launch with CUDA events between the launches
        (kt_time_kernels) and returns the average ms per step of each launch slot; in FP64 mode
        and the fused layout the rhs slots hold the fused stage kernels and the update slots are
        0; learned_start is the network's launch (0 without the learned start)."""
        ms = (C.c_float * 6)()
        n = C.c_int(6)
        self._check(self.L.kt_time_kernels(self.ctx, int(n_steps), ms, C.byref(n)), "kt_time_kernels")
        return dict(zip(self.KERNEL_SLOTS, list(ms)[:n.value]))


# ------------------------------------------------------------------ learned root-find start
MLP_PACKED_BYTES = 3396


def _mlp_lib():
    L = load_library()
    if not getattr(L, "_mlp_ready", False):
        vp, ll = C.c_void_p, C.c_longlong
        L.kt_mlp_features.argtypes = [vp, ll, vp, vp, vp, vp]
        L.kt_mlp_predict.argtypes = [vp, vp, ll, vp, vp, C.c_size_t, vp]
        L.kt_mlp_grad.argtypes = [vp, vp, vp, ll, C.c_int, vp, vp, vp]
        L.kt_mlp_adam.argtypes = [vp, vp, vp, vp, C.c_int, C.c_float, vp]
        L.kt_mlp_targets_workspace.argtypes = [ll, C.POINTER(C.c_size_t)]
        L.kt_mlp_targets.argtypes = [vp, vp, ll, vp, vp, vp, vp, C.c_size_t, vp]
        L.kt_mlp_batch.argtypes = [vp, vp, ll, C.c_ulonglong, C.c_int, ll, ll, vp, vp, vp, vp]
        L._mlp_ready = True
    return L


def _p(t):
    return C.c_void_p(t.data_ptr())


def _stream_handle():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def mlp_predict(params, x, scratch=None):
    """Tensor-core inference: params [1313] float32 CUDA, x [n, 6] float32 CUDA -> y [n]."""
    import torch
    L = _mlp_lib()
    n = x.shape[0]
    y = torch.empty(n, dtype=torch.float32, device=x.device)
    if scratch is None:
        scratch = torch.empty(MLP_PACKED_BYTES, dtype=torch.uint8, device=x.device)
    rc = L.kt_mlp_predict(_p(params), _p(x), n, _p(y), _p(scratch), scratch.numel(), _stream_handle())
    if rc != KT_OK:
        raise KTError(rc, "kt_mlp_predict")
    return y


def mlp_grad(params, x, y, bf16_forward=True):
    import torch
    L = _mlp_lib()
    grad = torch.empty(MLP_NPARAM, dtype=torch.float32, device=x.device)
    loss = torch.empty(1, dtype=torch.float32, device=x.device)
    rc = L.kt_mlp_grad(_p(params), _p(x), _p(y), x.shape[0], int(bool(bf16_forward)), _p(grad), _p(loss),
                       _stream_handle())
    if rc != KT_OK:
        raise KTError(rc, "kt_mlp_grad")
    return grad, loss


def mlp_adam(params, grad, m, v, step, lr):
    L = _mlp_lib()
    rc = L.kt_mlp_adam(_p(params), _p(grad), _p(m), _p(v), int(step), float(lr), _stream_handle())
    if rc != KT_OK:
        raise KTError(rc, "kt_mlp_adam")


def mlp_targets(X, Y):
    """The rows the network corrects and their targets z = y / r^2 (kt_mlp_targets), in order."""
    import torch
    L = _mlp_lib()
    n = X.shape[0]
    nb = C.c_size_t()
    if L.kt_mlp_targets_workspace(n, C.byref(nb)) != KT_OK:
        raise KTError(-1, "kt_mlp_targets_workspace")
    ws = torch.empty(nb.value, dtype=torch.uint8, device=X.device)
    xo = torch.empty_like(X)
    zo = torch.empty_like(Y)
    cnt = torch.empty(1, dtype=torch.int64, device=X.device)
    rc = L.kt_mlp_targets(_p(X), _p(Y), n, _p(xo), _p(zo), _p(cnt), _p(ws), nb.value, _stream_handle())
    if rc != KT_OK:
        raise KTError(rc, "kt_mlp_targets")
    k = int(cnt.cpu().item())
    return xo[:k], zo[:k]


def mlp_batch(X, Y, seed, epoch, b, batch, xb, yb, flag):
    """Mini-batch b of a shuffled epoch into xb, yb (kt_mlp_batch); returns the row count."""
    L = _mlp_lib()
    rc = L.kt_mlp_batch(_p(X), _p(Y), X.shape[0], int(seed), int(epoch), int(b), int(batch), _p(xb), _p(yb),
                        _p(flag), _stream_handle())
    if rc != KT_OK:
        raise KTError(rc, "kt_mlp_batch")
    return min(batch, X.shape[0] - b * batch)


def _kt_mlp_features(self, cells, out=None):
    """Training samples at physical cells (CUDA int64 tensor): features [n, 6], target [n],
    exact root e [n] (float64); `out` may hold (x, y, e) tensors to write into (e.g. views of a
    preallocated training set)."""
    import torch
    L = _mlp_lib()
    n = cells.numel()
    cells = cells.to(dtype=torch.int64).contiguous()
    if out is not None:
        x, y, e = out
        assert x.shape == (n, 6) and y.shape == (n,) and e.shape == (n,) and x.is_contiguous()
    else:
        x = torch.empty((n, 6), dtype=torch.float32, device="cuda")
        y = torch.empty(n, dtype=torch.float32, device="cuda")
        e = torch.empty(n, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    self._check(L.kt_mlp_features(self.ctx, n, _p(cells), _p(x), _p(y), _p(e)), "kt_mlp_features")
    return x, y, e


KT.mlp_features = _kt_mlp_features
