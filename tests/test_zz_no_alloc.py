"""The allocation-free entry point qsgw_chi0_block_noalloc against the context API.

Some callers cannot call cudaMalloc: their device memory is entirely reserved by another
allocator (a framework's caching pool, a fixed arena), or they must not risk the implicit
device synchronisation of cudaMalloc/cudaFree or an allocation failure at run time. For them
the library computes the chi0 of one block of columns inside one fixed array in its device
image. This file checks, through the C ABI, that three calls in a row (different shapes, so the
later ones run on whatever the earlier left in the shared array) give the same chi0 as
qsgw_chi0_accumulate + qsgw_chi0_finalize on a fresh context and as the FP64 oracle, within the
mixed-precision tolerance the other tests use (1e-6 relative Frobenius per frequency), and that
a call made after cudaDeviceReset (a new context, in which the array may sit at another address)
is still right.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from synthetic import eps_occ, eps_unocc, omega_grid, z_block

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-6


@pytest.fixture(scope="module")
def N():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_03477_gb300 import native
    native.load()
    return native


def _case(q, n_pb, n_occ, n_unocc, L):
    zt = z_block(3, q, 0, n_pb, n_occ, n_unocc, 40.0)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return dev(zt), dev(eps_occ(3, q, 0, n_occ)), dev(eps_unocc(3, q, 0, n_unocc)), omega_grid(L)


def _oracle_chi0(q, n_pb, n_occ, n_unocc, L):
    zt = z_block(3, q, 0, n_pb, n_occ, n_unocc, 40.0)
    d = oracle.delta(eps_occ(3, q, 0, n_occ), eps_unocc(3, q, 0, n_unocc))[0]
    return oracle.chi0_full(np.ascontiguousarray(zt.T), d, omega_grid(L), 2.0)


def _context_chi0(N, Z, eo, eu, n_pb, n_occ, n_unocc, om):
    ctx = N.qsgw_chi0_init([n_pb], om, 2.0, N.QSGW_MIXED_F16X3)
    try:
        N.qsgw_chi0_accumulate(ctx, 0, Z, n_pb, n_occ, n_unocc, eo, eu, om)
        chi = torch.empty((len(om), n_pb, n_pb), dtype=torch.complex128, device="cuda")
        N.qsgw_chi0_finalize(ctx, 0, chi)
    finally:
        N.qsgw_chi0_destroy(ctx)
    return chi.cpu().numpy()


def test_noalloc_two_calls_match_context_path(N):
    # (q, n_pb, n_occ, n_unocc, L); the last is the corner the header promises always fits
    cases = [(0, 200, 9, 61, 12), (1, 130, 5, 13, 16), (2, 256, 48, 64, 16)]
    inputs = [_case(*c) for c in cases]
    outs = []
    for (q, n_pb, n_occ, n_unocc, L), (Z, eo, eu, om) in zip(cases, inputs):  # calls in a row
        chi = torch.full((L, n_pb, n_pb), float("nan"), dtype=torch.complex128, device="cuda")
        N.qsgw_chi0_block_noalloc(Z, n_pb, n_pb, n_occ, n_unocc, eo, eu, om, 2.0, chi)
        outs.append(chi.cpu().numpy())
    for (q, n_pb, n_occ, n_unocc, L), (Z, eo, eu, om), got in zip(cases, inputs, outs):
        ref = _context_chi0(N, Z, eo, eu, n_pb, n_occ, n_unocc, om)
        exact = _oracle_chi0(q, n_pb, n_occ, n_unocc, L).transpose(0, 2, 1)  # column-major per frequency
        for l in range(L):
            err = np.linalg.norm(got[l] - ref[l]) / np.linalg.norm(ref[l])
            assert err <= TOL, (n_pb, l, err)
            err = np.linalg.norm(got[l] - exact[l]) / np.linalg.norm(exact[l])
            assert err <= TOL, (n_pb, l, err)


def test_noalloc_rejects_sizes_beyond_its_array(N):
    # n_pb = 2000 needs a 128 MiB accumulator alone (64 MiB array): rejected before any work is queued
    Z = torch.zeros((1, 2000), dtype=torch.complex128, device="cuda")
    eo = torch.full((1,), -0.5, dtype=torch.float64, device="cuda")
    eu = torch.full((1,), 0.5, dtype=torch.float64, device="cuda")
    chi = torch.zeros((1, 2000, 2000), dtype=torch.complex128, device="cuda")
    with pytest.raises(N.QsgwError) as err:
        N.qsgw_chi0_block_noalloc(Z, 2000, 2000, 1, 1, eo, eu, [0.1], 2.0, chi)
    assert err.value.status == N.QSGW_ERR_ARG


# Child process: only the library and the CUDA runtime it links (no torch), so cudaDeviceReset ends
# the process's one context. Buffers come from cudaMalloc in the child: the caller of the entry
# point allocates its inputs and outputs, the entry point itself allocates nothing.
_CHILD = r"""
import ctypes, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2506_03477_gb300 import native as N
N.load()
rt = ctypes.CDLL("libcudart.so.13")  # the runtime instance the library already loaded
rt.cudaMalloc.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_size_t]
rt.cudaMemcpy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
rt.cudaFree.argtypes = [ctypes.c_void_p]
data = np.load(sys.argv[2])
zt, eo, eu, om = data["zt"], data["eo"], data["eu"], data["om"]
n_pb, n_occ, n_unocc = zt.shape[1], eo.size, eu.size
out = []
for rep in range(2):
    bufs = []
    def put(a):
        p = ctypes.c_void_p()
        assert rt.cudaMalloc(ctypes.byref(p), a.nbytes) == 0
        assert rt.cudaMemcpy(p, a.ctypes.data, a.nbytes, 1) == 0
        bufs.append(p)
        return p.value
    chi = np.full((om.size, n_pb, n_pb), np.nan, dtype=np.complex128)
    dz, deo, deu, dchi = put(zt), put(eo), put(eu), put(chi)
    N.qsgw_chi0_block_noalloc(dz, n_pb, n_pb, n_occ, n_unocc, deo, deu, om, 2.0, dchi)
    assert rt.cudaMemcpy(chi.ctypes.data, dchi, chi.nbytes, 2) == 0
    out.append(chi)
    for p in bufs:
        rt.cudaFree(p)
    if rep == 0:
        assert rt.cudaDeviceReset() == 0  # a new context for the second call
np.save(sys.argv[3], np.stack(out))
"""


def test_noalloc_after_device_reset(N, tmp_path):
    q, n_pb, n_occ, n_unocc, L = 4, 192, 12, 40, 12
    zt = z_block(3, q, 0, n_pb, n_occ, n_unocc, 40.0)
    np.savez(tmp_path / "in.npz", zt=zt, eo=eps_occ(3, q, 0, n_occ), eu=eps_unocc(3, q, 0, n_unocc), om=omega_grid(L))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _CHILD, root, str(tmp_path / "in.npz"), str(tmp_path / "out.npy")],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    got = np.load(tmp_path / "out.npy")
    exact = _oracle_chi0(q, n_pb, n_occ, n_unocc, L).transpose(0, 2, 1)
    for rep in range(2):
        for l in range(L):
            err = np.linalg.norm(got[rep, l] - exact[l]) / np.linalg.norm(exact[l])
            assert err <= TOL, (rep, l, err)
