"""GB300-native KT + Heun step for 3+1d viscous hydrodynamics (arXiv:1608.06577).

The compute path is libkt.so (hand-written CUDA for sm_103a) behind the C ABI of
include/kt.h; this package only marshals arguments to it.  There is no CPU fallback.
"""
from .binding import (KT, KT_FP64, KT_INV_CONFORMAL, KT_INV_LEARNED, KT_INV_PLAIN, KT_MIXED, KTError, lib_path,  # noqa: F401
                      load_library, mlp_adam, mlp_grad, mlp_predict)
