"""GB300 (sm_103a) library for the RPA polarization chi0(q, i omega) in the mixed product basis
and the eps / W step of quasiparticle self-consistent GW (arXiv:2506.03477).

The computation lives in libqsgw.so (C ABI in include/qsgw.h); `native` is a thin ctypes
binding with the same function names. There is no CPU fallback.
"""
from . import native  # noqa: F401
from .native import *  # noqa: F401,F403
