"""FP64 CPU oracle for chi0(q, i omega), eps and W, the exchange self-energy, the real-axis
route and the imaginary-axis correlation self-energy (ctypes wrapper around oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the benchmark's
CPU-baseline leg. The CUDA library never imports or links it, and the two share no code.
Parity is pinned in tests/test_oracle_pins.py against closed forms, the paper's resolvent
form of Eq. (polfx), library special cases, brute force and invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_c_int, _c_ll, _c_double = ctypes.c_int, ctypes.c_longlong, ctypes.c_double
_p = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, OpenMP, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", _LIB, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.oracle_weight.restype = _c_double
        lib.oracle_weight.argtypes = [_c_double, _c_double]
        lib.oracle_delta.restype = _c_int
        lib.oracle_delta.argtypes = [_c_int, _c_int, _p, _p, _p]
        lib.oracle_chi0_rows.restype = None
        lib.oracle_chi0_rows.argtypes = [_c_ll, _c_int, _p, _c_int, _p, _p, _c_int, _p, _c_double, _p]
        lib.oracle_eps_w.restype = None
        lib.oracle_eps_w.argtypes = [_c_int, _c_int, _p, _p, _p, _p, _p, _p, _p, _p]
        lib.oracle_cholesky.restype = _c_int
        lib.oracle_cholesky.argtypes = [_c_int, _p, _p]
        lib.oracle_hist_spectral.restype = _c_ll
        lib.oracle_hist_spectral.argtypes = [_c_ll, _c_int, _p, _c_int, _p, _p, _c_int, _p, _p]
        lib.oracle_hilbert_weight.restype = _c_double
        lib.oracle_hilbert_weight.argtypes = [_c_double, _c_double, _c_double]
        lib.oracle_sigx.restype = None
        lib.oracle_sigx.argtypes = [_c_int, _p, _c_int, _c_int, _c_ll, _p, _p, _p]
        lib.oracle_sigc_weights.restype = None
        lib.oracle_sigc_weights.argtypes = [_c_double, _c_int, _p, _p]
        lib.oracle_sigc.restype = None
        lib.oracle_sigc.argtypes = [_c_int, _p, _c_int, _c_int, _p, _p, _p, _c_int, _p, _p, _p]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def weight(delta: float, omega: float) -> float:
    return _load().oracle_weight(float(delta), float(omega))


def delta(eps_occ: np.ndarray, eps_unocc: np.ndarray) -> tuple[np.ndarray, int]:
    """Transition energies of one k-point (r = n*n_unocc + m) and the count of Delta <= 0."""
    eo = np.ascontiguousarray(eps_occ, dtype=np.float64)
    eu = np.ascontiguousarray(eps_unocc, dtype=np.float64)
    out = np.empty(eo.size * eu.size, dtype=np.float64)
    bad = _load().oracle_delta(eo.size, eu.size, _ptr(eo), _ptr(eu), _ptr(out))
    return out, int(bad)


def chi0_rows(ZI: np.ndarray, ZJ: np.ndarray, delta_r: np.ndarray, omega: np.ndarray, spin: float) -> np.ndarray:
    """chi0 entries for row set I (ZI, shape (nI, K)) and column set J (ZJ, shape (nJ, K)).

    Returns out[l, i, j] = s * sum_r w_l(Delta_r) conj(ZI[i, r]) ZJ[j, r]."""
    ZI = np.ascontiguousarray(ZI, dtype=np.complex128)
    ZJ = np.ascontiguousarray(ZJ, dtype=np.complex128)
    d = np.ascontiguousarray(delta_r, dtype=np.float64)
    om = np.ascontiguousarray(omega, dtype=np.float64)
    nI, K = ZI.shape
    nJ = ZJ.shape[0]
    assert ZJ.shape[1] == K and d.size == K
    out = np.empty((om.size, nJ, nI), dtype=np.complex128)
    _load().oracle_chi0_rows(K, nI, _ptr(ZI), nJ, _ptr(ZJ), _ptr(d), om.size, _ptr(om), float(spin), _ptr(out))
    return np.ascontiguousarray(out.transpose(0, 2, 1))


def chi0_full(Zrows: np.ndarray, delta_r: np.ndarray, omega: np.ndarray, spin: float) -> np.ndarray:
    """Full chi0[l, I, J] from Zrows[I, r] = z_{I,r}."""
    return chi0_rows(Zrows, Zrows, delta_r, omega, spin)


def sigx(Zrows: np.ndarray, n_occ, n_pb: int, v: np.ndarray) -> np.ndarray:
    """Exchange self-energy, Eq. (sigx): out[n, m] = -sum_{k,n',mu} conj(Z[n, r]) v[k, mu] Z[m, r]
    with columns r = (k, n', mu), mu fastest; Zrows has shape (n_qp, n_pb * sum(n_occ))."""
    Z = np.ascontiguousarray(Zrows, dtype=np.complex128)
    occ = np.ascontiguousarray(n_occ, dtype=np.int32)
    vv = np.ascontiguousarray(v, dtype=np.float64)
    n_qp, K = Z.shape
    assert K == n_pb * int(occ.sum()) and vv.shape == (occ.size, n_pb)
    out = np.empty((n_qp, n_qp), dtype=np.complex128)  # column-major in C = transposed here
    _load().oracle_sigx(occ.size, _ptr(occ), int(n_pb), int(n_qp), int(K), _ptr(Z), _ptr(vv), _ptr(out))
    return np.ascontiguousarray(out.T)


def hist_spectral(ZI: np.ndarray, ZJ: np.ndarray, delta_r: np.ndarray, edges: np.ndarray):
    """Eq. (impolf) with one bin per column: S[j, i, jj] = sum_{r in bin j} conj(ZI[i, r]) ZJ[jj, r];
    returns (S, number of columns outside every bin)."""
    ZI = np.ascontiguousarray(ZI, dtype=np.complex128)
    ZJ = np.ascontiguousarray(ZJ, dtype=np.complex128)
    d = np.ascontiguousarray(delta_r, dtype=np.float64)
    e = np.ascontiguousarray(edges, dtype=np.float64)
    nI, K = ZI.shape
    nJ = ZJ.shape[0]
    out = np.empty((e.size - 1, nJ, nI), dtype=np.complex128)
    outside = _load().oracle_hist_spectral(K, nI, _ptr(ZI), nJ, _ptr(ZJ), _ptr(d), e.size - 1, _ptr(e), _ptr(out))
    return np.ascontiguousarray(out.transpose(0, 2, 1)), int(outside)


def hilbert_weight(w: float, lo: float, hi: float) -> float:
    """Eq. (hilbert): (1/(hi-lo)) P.V. int_lo^hi [1/(w - D) - 1/(w + D)] dD, uniform density in the bin."""
    return _load().oracle_hilbert_weight(float(w), float(lo), float(hi))


def real_axis_chi0(S: np.ndarray, edges: np.ndarray, bins_out) -> np.ndarray:
    """chi0 on the real axis at the centres of the bins in bins_out, from the spectral weights S
    (Eqs. (impolf), (hilbert)): the Hermitian part sum_j K_j(w) S_j and the anti-Hermitian part
    -pi S_i / (R_i - L_i) (w in bin i)."""
    e = np.asarray(edges, dtype=np.float64)
    out = []
    for i in bins_out:
        w = 0.5 * (e[i] + e[i + 1])
        re = sum(hilbert_weight(w, e[j], e[j + 1]) * S[j] for j in range(S.shape[0]))
        out.append(re - 1j * np.pi / (e[i + 1] - e[i]) * S[i])
    return np.array(out)


def sigc_weights(dE: float, omega: np.ndarray) -> np.ndarray:
    """Integration weights w_i(dE) of Eq. (sigci): sum_i w_i X(i omega_i) ~= (1/pi) int_0^inf
    dE/(dE^2+w^2) X(iw) dw, X constant below omega_0, linear between mesh points and decaying as
    1/w^2 beyond the last (the reading stated in oracle.c)."""
    om = np.ascontiguousarray(omega, dtype=np.float64)
    w = np.empty(om.size, dtype=np.float64)
    _load().oracle_sigc_weights(float(dE), int(om.size), _ptr(om), _ptr(w))
    return w


def sigc(Zcols, e_qp: np.ndarray, e_band, omega: np.ndarray, Wc) -> np.ndarray:
    """Eq. (sigci): I[n, m] = -sum_{k,n',i} w_i(e_qp[n] - e_band[k][n']) sum_{mu,nu}
    conj(Z_k[n' n, mu]) Wc_k[i, mu, nu] Z_k[n' m, nu]. Per k: Zcols[k] has shape
    (n_band * n_qp, n_pb) (row r = n' * n_qp + n), e_band[k] shape (n_band,), Wc[k] shape
    (L, n_pb, n_pb) indexed [i, mu, nu]."""
    e_q = np.ascontiguousarray(e_qp, dtype=np.float64)
    om = np.ascontiguousarray(omega, dtype=np.float64)
    n_qp, L = e_q.size, om.size
    n_pb = Zcols[0].shape[1]
    nb = np.array([len(e) for e in e_band], dtype=np.int32)
    for k in range(len(Zcols)):
        assert Zcols[k].shape == (nb[k] * n_qp, n_pb) and Wc[k].shape == (L, n_pb, n_pb)
    Z = np.ascontiguousarray(np.concatenate([np.asarray(z, dtype=np.complex128) for z in Zcols]))
    eb = np.ascontiguousarray(np.concatenate(e_band), dtype=np.float64)
    W = np.ascontiguousarray(np.concatenate([np.asarray(w, dtype=np.complex128).transpose(0, 2, 1) for w in Wc]))
    out = np.empty((n_qp, n_qp), dtype=np.complex128)  # column-major in C = transposed here
    _load().oracle_sigc(len(Zcols), _ptr(nb), int(n_pb), int(n_qp), _ptr(Z), _ptr(e_q), _ptr(eb), int(L), _ptr(om),
                        _ptr(W), _ptr(out))
    return np.ascontiguousarray(out.T)


def eps_w(chi: np.ndarray, v: np.ndarray, want_eps: bool = True, want_wc: bool = True):
    """eps, W, W^c (each [L, N, N], numpy row/col indexing [l, i, j]) and Cholesky info per frequency."""
    L, N, _ = chi.shape
    # the C side is column-major per frequency: element (i, j) at j*N + i, i.e. the transpose in C order
    chi_cm = np.ascontiguousarray(chi.transpose(0, 2, 1), dtype=np.complex128)
    vv = np.ascontiguousarray(v, dtype=np.float64)
    eps = np.empty_like(chi_cm) if want_eps else None
    W = np.empty_like(chi_cm)
    Wc = np.empty_like(chi_cm) if want_wc else None
    info = np.zeros(L, dtype=np.int32)
    work_e = np.empty((N, N), dtype=np.complex128)
    work_l = np.empty((N, N), dtype=np.complex128)
    _load().oracle_eps_w(N, L, _ptr(chi_cm), _ptr(vv), _ptr(eps) if want_eps else None, _ptr(W),
                         _ptr(Wc) if want_wc else None, _ptr(info), _ptr(work_e), _ptr(work_l))
    tr = (lambda a: None if a is None else np.ascontiguousarray(a.transpose(0, 2, 1)))
    return tr(eps), tr(W), tr(Wc), info


def cholesky(A: np.ndarray) -> tuple[np.ndarray, int]:
    """Lower Cholesky factor of one Hermitian matrix (numpy [i, j] indexing) and the info code."""
    N = A.shape[0]
    a_cm = np.ascontiguousarray(A.T, dtype=np.complex128)
    l_cm = np.empty_like(a_cm)
    info = _load().oracle_cholesky(N, _ptr(a_cm), _ptr(l_cm))
    return np.ascontiguousarray(l_cm.T), int(info)
