"""ctypes binding for libqsgw.so (include/qsgw.h). Argument marshalling only: every step of
the computation runs in the library's CUDA kernels.

Functions keep the C names. Array arguments may be torch tensors (device or host), numpy
arrays (host) or raw integer addresses. Any status other than QSGW_OK raises QsgwError.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libqsgw.so")

QSGW_OK = 0
QSGW_ERR_ARG = -1
QSGW_ERR_DOMAIN = -2
QSGW_ERR_NOMEM = -3
QSGW_ERR_CUDA = -4
QSGW_ERR_NOT_PD = -5
QSGW_ERR_TIMEOUT = -6
QSGW_ERR_STATE = -7
QSGW_FP64 = 0
QSGW_MIXED_F16X3 = 1
QSGW_MIXED_BF16X3 = QSGW_MIXED_F16X3  # earlier name of the same mode
QSGW_MIXED_TF32X3 = 2  # reserved: rejected with QSGW_ERR_ARG

EXPORTS = [
    "qsgw_chi0_init", "qsgw_chi0_accumulate", "qsgw_chi0_finalize", "qsgw_eps_inv", "qsgw_chi0_reset",
    "qsgw_chi0_sync", "qsgw_chi0_destroy", "qsgw_status_string", "qsgw_synth_z", "qsgw_chi0_accumulate_synthetic",
    "qsgw_chi0_accumulate_batch", "qsgw_chi0_block_noalloc", "qsgw_chi0_accumulate_c64",
    "qsgw_sigx_init", "qsgw_sigx_accumulate", "qsgw_sigx_accumulate_c64", "qsgw_selftest_wait_timeout",
    "qsgw_spectral_init", "qsgw_spectral_accumulate", "qsgw_spectral_finalize", "qsgw_spectral_real_axis",
    "qsgw_sigc_init", "qsgw_sigc_accumulate", "qsgw_sigc_finalize",
    "qsgw_tile_plan_candidates", "qsgw_chi0_autotune", "qsgw_chi0_set_tile_plan",
]


class qsgw_block(ctypes.Structure):
    """C struct qsgw_block (include/qsgw.h)."""
    _fields_ = [("q", ctypes.c_int), ("Z", ctypes.c_void_p), ("ldz", ctypes.c_longlong), ("n_occ", ctypes.c_int),
                ("n_unocc", ctypes.c_int), ("eps_occ", ctypes.c_void_p), ("eps_unocc", ctypes.c_void_p)]


class qsgw_tile_plan(ctypes.Structure):
    """C struct qsgw_tile_plan (include/qsgw.h)."""
    _fields_ = [("tile_cols", ctypes.c_int), ("tail_pieces", ctypes.c_int)]


class QsgwError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {qsgw_status_string(status)} ({status})")


_lib = None
_i, _ll, _d, _p, _u64 = ctypes.c_int, ctypes.c_longlong, ctypes.c_double, ctypes.c_void_p, ctypes.c_ulonglong


def load():
    """Load libqsgw.so; raises if it has not been built (no CPU fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    sig = {
        "qsgw_chi0_init": [P(_p), _i, P(_i), _i, P(_d), _d, _i, _p],
        "qsgw_chi0_accumulate": [_p, _i, _p, _ll, _i, _i, _p, _p, _i, P(_d)],
        "qsgw_chi0_accumulate_c64": [_p, _i, _p, _ll, _i, _i, _p, _p, _i, P(_d)],
        "qsgw_sigx_init": [P(_p), _i, P(_i), _i, _p],
        "qsgw_sigx_accumulate": [_p, _i, _p, _ll, _i, _i, _p],
        "qsgw_sigx_accumulate_c64": [_p, _i, _p, _ll, _i, _i, _p],
        "qsgw_selftest_wait_timeout": [_d, _p],
        "qsgw_spectral_init": [P(_p), _i, _i, P(_d), _i, _p],
        "qsgw_spectral_accumulate": [_p, _p, _ll, _i, _i, _p, _p],
        "qsgw_spectral_finalize": [_p, _p],
        "qsgw_spectral_real_axis": [_p, _p, _i, P(_i), _p],
        "qsgw_sigc_init": [P(_p), _i, _i, _i, P(_d), _i, _p],
        "qsgw_sigc_accumulate": [_p, _p, _ll, _i, _p, _p, _p],
        "qsgw_sigc_finalize": [_p, _p],
        "qsgw_chi0_finalize": [_p, _i, _p],
        "qsgw_eps_inv": [_p, _i, _p, _p, _p, _i, P(_i)],
        "qsgw_chi0_reset": [_p, _i],
        "qsgw_chi0_sync": [_p],
        "qsgw_chi0_destroy": [_p],
        "qsgw_synth_z": [_u64, _i, _i, _i, _i, _i, _d, _p, _ll, _p],
        "qsgw_chi0_accumulate_synthetic": [_p, _i, _u64, _i, _i, _i, _i, P(_i), _p, _p, _d],
        "qsgw_chi0_accumulate_batch": [_p, _i, P(qsgw_block)],
        "qsgw_chi0_block_noalloc": [_p, _ll, _i, _i, _i, _p, _p, _i, P(_d), _d, _p, _p],
        "qsgw_tile_plan_candidates": [_i, P(qsgw_tile_plan), _i],
        "qsgw_chi0_autotune": [_p, _i, P(qsgw_block), _i, P(qsgw_tile_plan), P(ctypes.c_float)],
        "qsgw_chi0_set_tile_plan": [_p, P(qsgw_tile_plan)],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = _i
    lib.qsgw_status_string.argtypes = [_i]
    lib.qsgw_status_string.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _addr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _check(status: int, where: str):
    if status != QSGW_OK:
        raise QsgwError(status, where)


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
    return int(getattr(stream, "cuda_stream", stream))


def qsgw_status_string(status: int) -> str:
    return load().qsgw_status_string(int(status)).decode()


def qsgw_chi0_init(n_pb, omega, spin_factor: float, prec: int = QSGW_FP64, stream=None) -> int:
    n_pb = list(n_pb)
    om = np.ascontiguousarray(omega, dtype=np.float64)
    ctx = _p()
    arr_n = (_i * len(n_pb))(*n_pb)
    arr_o = (_d * om.size)(*om.tolist())
    _check(load().qsgw_chi0_init(ctypes.byref(ctx), len(n_pb), arr_n, om.size, arr_o, float(spin_factor), int(prec),
                                 _stream(stream)), "qsgw_chi0_init")
    return ctx.value


def qsgw_chi0_accumulate(ctx: int, q: int, Z, ldz: int, n_occ: int, n_unocc: int, eps_occ, eps_unocc, omega):
    om = np.ascontiguousarray(omega, dtype=np.float64)
    arr_o = (_d * om.size)(*om.tolist())
    _check(load().qsgw_chi0_accumulate(ctx, q, _addr(Z), int(ldz), int(n_occ), int(n_unocc), _addr(eps_occ),
                                       _addr(eps_unocc), om.size, arr_o), "qsgw_chi0_accumulate")


def qsgw_chi0_accumulate_c64(ctx: int, q: int, Z, ldz: int, n_occ: int, n_unocc: int, eps_occ, eps_unocc, omega):
    """Z in complex64 (mixed-precision contexts only; see include/qsgw.h)."""
    om = np.ascontiguousarray(omega, dtype=np.float64)
    arr_o = (_d * om.size)(*om.tolist())
    _check(load().qsgw_chi0_accumulate_c64(ctx, q, _addr(Z), int(ldz), int(n_occ), int(n_unocc), _addr(eps_occ),
                                           _addr(eps_unocc), om.size, arr_o), "qsgw_chi0_accumulate_c64")


def qsgw_sigx_init(n_qp, prec: int = QSGW_FP64, stream=None) -> int:
    """Context for the exchange self-energy, Eq. (sigx) (see include/qsgw.h)."""
    n_qp = list(n_qp)
    ctx = _p()
    arr = (_i * len(n_qp))(*n_qp)
    _check(load().qsgw_sigx_init(ctypes.byref(ctx), len(n_qp), arr, int(prec), _stream(stream)), "qsgw_sigx_init")
    return ctx.value


def qsgw_sigx_accumulate(ctx: int, q: int, Z, ldz: int, n_occ: int, n_pb: int, v):
    _check(load().qsgw_sigx_accumulate(ctx, q, _addr(Z), int(ldz), int(n_occ), int(n_pb), _addr(v)),
           "qsgw_sigx_accumulate")


def qsgw_sigx_accumulate_c64(ctx: int, q: int, Z, ldz: int, n_occ: int, n_pb: int, v):
    _check(load().qsgw_sigx_accumulate_c64(ctx, q, _addr(Z), int(ldz), int(n_occ), int(n_pb), _addr(v)),
           "qsgw_sigx_accumulate_c64")


def qsgw_spectral_init(n_pb: int, edges, prec: int = QSGW_FP64, stream=None) -> int:
    """Context for the real-axis route (histogram of Delta; see include/qsgw.h)."""
    e = np.ascontiguousarray(edges, dtype=np.float64)
    arr = (_d * e.size)(*e.tolist())
    ctx = _p()
    _check(load().qsgw_spectral_init(ctypes.byref(ctx), int(n_pb), e.size - 1, arr, int(prec), _stream(stream)),
           "qsgw_spectral_init")
    return ctx.value


def qsgw_spectral_accumulate(ctx: int, Z, ldz: int, n_occ: int, n_unocc: int, eps_occ, eps_unocc):
    _check(load().qsgw_spectral_accumulate(ctx, _addr(Z), int(ldz), int(n_occ), int(n_unocc), _addr(eps_occ),
                                           _addr(eps_unocc)), "qsgw_spectral_accumulate")


def qsgw_spectral_finalize(ctx: int, S):
    _check(load().qsgw_spectral_finalize(ctx, _addr(S)), "qsgw_spectral_finalize")


def qsgw_spectral_real_axis(ctx: int, S, bins_out, out):
    b = list(bins_out)
    arr = (_i * len(b))(*b)
    _check(load().qsgw_spectral_real_axis(ctx, _addr(S), len(b), arr, _addr(out)), "qsgw_spectral_real_axis")


def qsgw_sigc_init(n_qp: int, n_pb: int, omega, prec: int = QSGW_FP64, stream=None) -> int:
    """Context for the imaginary-axis correlation self-energy, Eq. (sigci) (see include/qsgw.h)."""
    om = [float(x) for x in omega]
    arr = (_d * len(om))(*om)
    ctx = _p()
    _check(load().qsgw_sigc_init(ctypes.byref(ctx), int(n_qp), int(n_pb), len(om), arr, int(prec), _stream(stream)),
           "qsgw_sigc_init")
    return ctx.value


def qsgw_sigc_accumulate(ctx: int, Z, ldz: int, n_band: int, e_qp, e_band, Wc):
    _check(load().qsgw_sigc_accumulate(ctx, _addr(Z), int(ldz), int(n_band), _addr(e_qp), _addr(e_band), _addr(Wc)),
           "qsgw_sigc_accumulate")


def qsgw_sigc_finalize(ctx: int, I):
    _check(load().qsgw_sigc_finalize(ctx, _addr(I)), "qsgw_sigc_finalize")


def qsgw_selftest_wait_timeout(limit_seconds: float, stream=None) -> int:
    """Returns the raw status (QSGW_ERR_TIMEOUT is the expected outcome; see include/qsgw.h)."""
    return int(load().qsgw_selftest_wait_timeout(float(limit_seconds), _stream(stream)))


def qsgw_chi0_finalize(ctx: int, q: int, chi0):
    _check(load().qsgw_chi0_finalize(ctx, q, _addr(chi0)), "qsgw_chi0_finalize")


def qsgw_eps_inv(ctx: int, q: int, v, W, eps_out=None, correlation_only: bool = False, n_omega: int = 16,
                 raise_not_pd: bool = True) -> np.ndarray:
    info = (_i * 16)()
    st = load().qsgw_eps_inv(ctx, q, _addr(v), _addr(W), _addr(eps_out), int(bool(correlation_only)), info)
    out = np.array(info[:n_omega], dtype=np.int32)
    if st == QSGW_ERR_NOT_PD and not raise_not_pd:
        return out
    _check(st, "qsgw_eps_inv")
    return out


def qsgw_chi0_reset(ctx: int, q: int):
    _check(load().qsgw_chi0_reset(ctx, q), "qsgw_chi0_reset")


def qsgw_chi0_sync(ctx: int):
    _check(load().qsgw_chi0_sync(ctx), "qsgw_chi0_sync")


def qsgw_chi0_destroy(ctx: int):
    _check(load().qsgw_chi0_destroy(ctx), "qsgw_chi0_destroy")


def qsgw_synth_z(seed: int, gen_q: int, k: int, n_pb: int, n_occ: int, n_unocc: int, s_div: float, Z, ldz: int,
                 stream=None):
    _check(load().qsgw_synth_z(int(seed), int(gen_q), int(k), int(n_pb), int(n_occ), int(n_unocc), float(s_div),
                               _addr(Z), int(ldz), _stream(stream)), "qsgw_synth_z")


def qsgw_chi0_accumulate_synthetic(ctx: int, q: int, seed: int, gen_q: int, k_begin: int, k_end: int, n_occ: int,
                                   n_unocc_per_k, eps_occ, eps_unocc, s_div: float):
    nu = list(n_unocc_per_k)
    arr = (_i * len(nu))(*nu)
    _check(load().qsgw_chi0_accumulate_synthetic(ctx, q, int(seed), int(gen_q), int(k_begin), int(k_end), int(n_occ),
                                                 arr, _addr(eps_occ), _addr(eps_unocc), float(s_div)),
           "qsgw_chi0_accumulate_synthetic")


def qsgw_chi0_accumulate_batch(ctx: int, blocks):
    """blocks: iterable of (q, Z, ldz, n_occ, n_unocc, eps_occ, eps_unocc) with device arrays."""
    blocks = list(blocks)
    arr = (qsgw_block * len(blocks))()
    for i, (q, Z, ldz, n_occ, n_unocc, eo, eu) in enumerate(blocks):
        arr[i] = qsgw_block(int(q), _addr(Z), int(ldz), int(n_occ), int(n_unocc), _addr(eo), _addr(eu))
    _check(load().qsgw_chi0_accumulate_batch(ctx, len(blocks), arr), "qsgw_chi0_accumulate_batch")


def _block_array(blocks):
    blocks = list(blocks)
    arr = (qsgw_block * len(blocks))()
    for i, (q, Z, ldz, n_occ, n_unocc, eo, eu) in enumerate(blocks):
        arr[i] = qsgw_block(int(q), _addr(Z), int(ldz), int(n_occ), int(n_unocc), _addr(eo), _addr(eu))
    return arr


def qsgw_tile_plan_candidates(n_omega: int):
    """The tuner's candidate plans for n_omega frequencies, as (tile_cols, tail_pieces) pairs."""
    out = (qsgw_tile_plan * 16)()
    n = load().qsgw_tile_plan_candidates(int(n_omega), out, 16)
    return [(out[i].tile_cols, out[i].tail_pieces) for i in range(n)]


def qsgw_chi0_autotune(ctx: int, blocks, reps: int = 2):
    """Time every candidate plan on these blocks; returns ((tile_cols, tail_pieces), ms per launch)."""
    arr = _block_array(blocks)
    plan, ms = qsgw_tile_plan(), ctypes.c_float()
    _check(load().qsgw_chi0_autotune(ctx, len(arr), arr, int(reps), ctypes.byref(plan), ctypes.byref(ms)),
           "qsgw_chi0_autotune")
    return (plan.tile_cols, plan.tail_pieces), ms.value


def qsgw_chi0_set_tile_plan(ctx: int, plan):
    """plan: (tile_cols, tail_pieces), or None for the tuned / default plan."""
    p = None if plan is None else ctypes.byref(qsgw_tile_plan(int(plan[0]), int(plan[1])))
    _check(load().qsgw_chi0_set_tile_plan(ctx, p), "qsgw_chi0_set_tile_plan")


def qsgw_chi0_block_noalloc(Z, ldz: int, n_pb: int, n_occ: int, n_unocc: int, eps_occ, eps_unocc, omega,
                            spin_factor: float, chi0, stream=None):
    """chi0 of one block of columns into chi0 without any device allocation (see include/qsgw.h)."""
    om = np.ascontiguousarray(omega, dtype=np.float64)
    arr_o = (_d * om.size)(*om.tolist())
    _check(load().qsgw_chi0_block_noalloc(_addr(Z), int(ldz), int(n_pb), int(n_occ), int(n_unocc), _addr(eps_occ),
                                          _addr(eps_unocc), om.size, arr_o, float(spin_factor), _addr(chi0),
                                          _stream(stream)), "qsgw_chi0_block_noalloc")
