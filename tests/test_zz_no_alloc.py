"""The allocation-free entry point qsgw_chi0_block_noalloc against the context API.

Some callers cannot call cudaMalloc: their device memory is entirely reserved by another
allocator (a framework's caching pool, a fixed arena), or they must not risk the implicit
device synchronisation of cudaMalloc/cudaFree or an allocation failure at run time. For them
the library computes the chi0 of one block of columns inside one fixed array in its device
image. This file checks, through the C ABI, that three calls in a row (different shapes, so the
later ones run on whatever the earlier left in the shared array) give the same chi0 as
qsgw_chi0_accumulate + qsgw_chi0_finalize on a fresh context, within the mixed-precision
tolerance the other tests use (1e-6 relative Frobenius per frequency).
"""
import numpy as np
import pytest

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


def _context_chi0(N, Z, eo, eu, n_pb, n_occ, n_unocc, om):
    ctx = N.qsgw_chi0_init([n_pb], om, 2.0, N.QSGW_MIXED_BF16X3)
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
        for l in range(L):
            err = np.linalg.norm(got[l] - ref[l]) / np.linalg.norm(ref[l])
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
