"""The C-ABI library loads and exports every symbol that include/*.h declares (no GPU calls)."""
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(kt_[a-z0-9_]+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_1608_06577_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared_symbols()
    for n in ("kt_init", "kt_set_state", "kt_step", "kt_get_state", "kt_free", "kt_get_stats", "kt_last_error"):
        assert n in names, n


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.check_output(["nm", "-D", "--defined-only", libpath]).decode()
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = _declared_symbols() - exported
    assert not missing, missing


def test_library_loads_and_fails_loudly_without_gpu(libpath):
    import ctypes
    from paper_1608_06577_gb300 import binding
    L = binding.load_library()
    o = binding.Options()
    assert L.kt_options_default(ctypes.byref(o)) == 0
    assert o.theta_limiter == 1.0 and o.regulate == 1
    import torch
    if not torch.cuda.is_available():
        g = binding.Grid(4, 4, 4)
        eos = binding.Eos(0, 15.6, 0, None, None, None, None, None)
        z = binding.Coef(0, 0.0, 0.0, 1.0)
        ctx = ctypes.c_void_p()
        rc = L.kt_init(ctypes.byref(ctx), ctypes.byref(g), 0.1, 0.1, 0.01, ctypes.byref(eos), ctypes.byref(z),
                       ctypes.byref(z), None)
        assert rc == -2  # KT_ERR_CUDA: no device, and no CPU fallback


def test_invalid_arguments_rejected(libpath):
    import ctypes
    from paper_1608_06577_gb300 import binding
    L = binding.load_library()
    ctx = ctypes.c_void_p()
    g = binding.Grid(0, 4, 4)
    eos = binding.Eos(0, 15.6, 0, None, None, None, None, None)
    z = binding.Coef(0, 0.0, 0.0, 1.0)
    assert L.kt_init(ctypes.byref(ctx), ctypes.byref(g), 0.1, 0.1, 0.01, ctypes.byref(eos), ctypes.byref(z),
                     ctypes.byref(z), None) == -1
    # options are validated before any device work: FP32 pi storage needs the mixed precision
    o = binding.Options()
    L.kt_options_default(ctypes.byref(o))
    o.pi_storage = 1
    g4 = binding.Grid(4, 4, 4)
    assert L.kt_init(ctypes.byref(ctx), ctypes.byref(g4), 0.1, 0.1, 0.01, ctypes.byref(eos), ctypes.byref(z),
                     ctypes.byref(z), ctypes.byref(o)) == -1
    o.pi_storage = 7
    o.precision = 1
    assert L.kt_init(ctypes.byref(ctx), ctypes.byref(g4), 0.1, 0.1, 0.01, ctypes.byref(eos), ctypes.byref(z),
                     ctypes.byref(z), ctypes.byref(o)) == -1
    # the conformal start (no network) serves the mixed precision only; unknown starts are rejected
    L.kt_options_default(ctypes.byref(o))
    o.inversion = binding.KT_INV_CONFORMAL
    assert L.kt_init(ctypes.byref(ctx), ctypes.byref(g4), 0.1, 0.1, 0.01, ctypes.byref(eos), ctypes.byref(z),
                     ctypes.byref(z), ctypes.byref(o)) == -1
    o.inversion = 3
    o.precision = 1
    assert L.kt_init(ctypes.byref(ctx), ctypes.byref(g4), 0.1, 0.1, 0.01, ctypes.byref(eos), ctypes.byref(z),
                     ctypes.byref(z), ctypes.byref(o)) == -1
    nb = ctypes.c_size_t()
    assert L.kt_state_bytes(ctypes.byref(binding.Grid(128, 128, 128)), None, None, ctypes.byref(nb)) == 0
    assert nb.value > 30 * 132 * 132 * 132 * 8
    # a table EOS adds its per-interval coefficients: a longer table needs more bytes
    sizes = []
    for n in (4096, 16384):
        tab = binding.Eos(1, 0.0, n, None, None, None, None, None)
        b = ctypes.c_size_t()
        assert L.kt_state_bytes(ctypes.byref(binding.Grid(8, 8, 8)), ctypes.byref(tab), None, ctypes.byref(b)) == 0
        sizes.append(b.value)
    assert sizes[1] >= sizes[0] + (16384 - 4096) * 15 * 8  # at least the FP64 coefficients
    short = binding.Eos(1, 0.0, 3, None, None, None, None, None)
    assert L.kt_state_bytes(ctypes.byref(binding.Grid(8, 8, 8)), ctypes.byref(short), None, ctypes.byref(nb)) == -4


def test_network_constants_agree():
    """The gate of the learned start and the parameter count are written in the header, the
    kernels and the Python training driver; they must agree."""
    from paper_1608_06577_gb300 import binding, learned
    hdr = open(os.path.join(ROOT, "include", "kt.h")).read()
    cuh = open(os.path.join(ROOT, "paper_1608_06577_gb300", "csrc", "kt_mlp.cuh")).read()
    gate_h = float(re.search(r"#define KT_MLP_GATE_R2\s+([0-9.eE+-]+)", hdr).group(1))
    gate_k = float(re.search(r"kMlpGateR2\s*=\s*([0-9.eE+-]+)f", cuh).group(1))
    assert gate_h == gate_k == learned.GATE_R2
    npar_h = eval(re.search(r"#define KT_MLP_NPARAM\s+(\([^)]*\))", hdr).group(1))
    assert npar_h == binding.MLP_NPARAM == 1313
