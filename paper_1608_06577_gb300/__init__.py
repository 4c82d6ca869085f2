"""GB300-native KT + Heun step for 3+1d viscous hydrodynamics (arXiv:1608.06577).

The compute path is libkt.so (hand-written CUDA for sm_103a) behind the C ABI of
include/kt.h; this package only marshals arguments to it.  There is no CPU fallback.
"""
from .binding import KT, KTError, lib_path, load_library  # noqa: F401
