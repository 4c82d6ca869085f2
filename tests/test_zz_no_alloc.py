"""kt_mlp_predict_static: the inference entry point that allocates nothing.

It exists for callers that cannot call cudaMalloc (device memory budgeted up front by a host
application or a custom allocator, or latency-critical loops that cannot afford an allocation
and the synchronisation it may imply).  Its scratch, the packed network weights, lives in a
file-scope device array of the library.  This test calls it through the C ABI and compares it
with kt_mlp_predict, which takes the same scratch from the caller, on two calls in a row with
different weights (so the second call must not see the first call's scratch contents).
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _lib():
    from paper_1608_06577_gb300 import build
    from paper_1608_06577_gb300.binding import load_library
    build.build()
    L = load_library()
    L.kt_mlp_predict_static.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p,
                                        ctypes.c_void_p]
    return L


def test_static_scratch_predict_matches_predict_twice():
    import torch
    from paper_1608_06577_gb300.binding import mlp_predict
    L = _lib()
    rng = np.random.default_rng(7)
    x = torch.as_tensor(rng.normal(size=(1000, 6)).astype(np.float32), device="cuda")  # ragged last warp
    stream = torch.cuda.current_stream()
    for call in range(2):
        params = torch.as_tensor((rng.normal(size=1313) * 0.3).astype(np.float32), device="cuda")
        y_ref = mlp_predict(params, x)
        y = torch.full((x.shape[0],), float("nan"), dtype=torch.float32, device="cuda")
        rc = L.kt_mlp_predict_static(ctypes.c_void_p(params.data_ptr()), ctypes.c_void_p(x.data_ptr()), x.shape[0],
                                     ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, rc
        torch.cuda.synchronize()
        a, b = y.cpu().numpy(), y_ref.cpu().numpy()
        assert np.all(np.isfinite(a)), call
        np.testing.assert_allclose(a, b, rtol=1e-6, atol=1e-7 * np.max(np.abs(b)))


def test_static_scratch_predict_rejects_bad_sizes():
    import torch
    L = _lib()
    p = torch.zeros(1313, dtype=torch.float32, device="cuda")
    x = torch.zeros((4, 6), dtype=torch.float32, device="cuda")
    y = torch.zeros(4, dtype=torch.float32, device="cuda")
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    assert L.kt_mlp_predict_static(ptr(p), ptr(x), -1, ptr(y), None) == -1
    assert L.kt_mlp_predict_static(ptr(p), ptr(x), 2147483648, ptr(y), None) == -1
    assert L.kt_mlp_predict_static(ptr(p), ptr(x), 0, ptr(y), None) == 0
