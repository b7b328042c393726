"""Exchange self-energy Sigma^x, Eq. (sigx), on the GPU (FP64 and mixed tensor-core paths) against
the FP64 oracle: rel. Frobenius <= 1e-12 (FP64) and <= 1e-6 (mixed, plus the per-element
Cauchy-Schwarz bound of a semidefinite matrix), on ragged shapes; complex64 input bit-identical;
v <= 0 reported; the chi0 and Sigma^x contexts reject each other's calls."""
import numpy as np
import pytest

import oracle
from synthetic import coulomb_v, z_block

from test_gpu_fp64 import _dev, rel_fro

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def N():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_03477_gb300 import native
    native.load()
    return native


def _blocks(n_qp, occ, n_pb, seed=7):
    """Per k-point: Z (column r = n' * n_pb + mu, rows n) as the (K_k, n_qp) array whose memory is the
    column-major n_qp x K_k matrix, and v_mu(k) > 0."""
    return [(z_block(seed, 0, k, n_qp, no, n_pb, 40.0), coulomb_v(seed, k, n_pb)) for k, no in enumerate(occ)]


def _oracle(blocks, occ, n_pb):
    Zrows = np.concatenate([zt.T for zt, _ in blocks], axis=1)
    return oracle.sigx(Zrows, occ, n_pb, np.stack([v for _, v in blocks]))


def _run(N, prec, n_qp, occ, n_pb, blocks, mode="device"):
    ctx = N.qsgw_sigx_init([n_qp], prec)
    keep = []
    try:
        for (zt, v), no in zip(blocks, occ):
            if mode == "device":
                N.qsgw_sigx_accumulate(ctx, 0, _dev(zt), n_qp, no, n_pb, _dev(v))
            elif mode == "host":
                N.qsgw_sigx_accumulate(ctx, 0, np.ascontiguousarray(zt), n_qp, no, n_pb, np.ascontiguousarray(v))
            else:  # complex64 on the device
                z64 = _dev(zt.astype(np.complex64))
                keep.append(z64)
                N.qsgw_sigx_accumulate_c64(ctx, 0, z64, n_qp, no, n_pb, _dev(v))
        out = torch.empty((n_qp, n_qp), dtype=torch.complex128, device="cuda")
        N.qsgw_chi0_finalize(ctx, 0, out)
        return out.cpu().numpy().T  # column-major -> [n, m]
    finally:
        N.qsgw_chi0_destroy(ctx)


def test_sigx_fp64_parity_and_host_staging(N):
    n_qp, occ, n_pb = 90, [3, 5], 70
    blocks = _blocks(n_qp, occ, n_pb)
    ref = _oracle(blocks, occ, n_pb)
    got = _run(N, N.QSGW_FP64, n_qp, occ, n_pb, blocks)
    assert rel_fro(got, ref) <= 1e-12
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.array_equal(_run(N, N.QSGW_FP64, n_qp, occ, n_pb, blocks, mode="host"), got)


@pytest.mark.parametrize("n_qp,occ,n_pb", [(1, [1], 1), (70, [2, 3], 50), (130, [4, 1, 6], 333), (300, [7, 9], 250)])
def test_sigx_mixed_parity_ragged(N, n_qp, occ, n_pb):
    blocks = _blocks(n_qp, occ, n_pb)
    ref = _oracle(blocks, occ, n_pb)
    got = _run(N, N.QSGW_MIXED_F16X3, n_qp, occ, n_pb, blocks)
    assert rel_fro(got, ref) <= 1e-6, rel_fro(got, ref)
    d = np.sqrt(np.abs(np.diag(ref)))
    assert np.all(np.abs(got - ref) <= 1e-6 * np.outer(d, d) + 1e-300)
    assert np.array_equal(got, got.conj().T)
    assert np.array_equal(_run(N, N.QSGW_MIXED_F16X3, n_qp, occ, n_pb, blocks, mode="c64"), got)


def test_sigx_nonpositive_v_is_reported(N):
    n_qp, n_pb = 16, 8
    ctx = N.qsgw_sigx_init([n_qp], N.QSGW_MIXED_F16X3)
    try:
        zt = z_block(3, 0, 0, n_qp, 2, n_pb, 40.0)
        v = coulomb_v(3, 0, n_pb)
        v[5] = 0.0
        N.qsgw_sigx_accumulate(ctx, 0, _dev(zt), n_qp, 2, n_pb, _dev(v))
        out = torch.empty((n_qp, n_qp), dtype=torch.complex128, device="cuda")
        with pytest.raises(N.QsgwError) as e:
            N.qsgw_chi0_finalize(ctx, 0, out)
        assert e.value.status == N.QSGW_ERR_DOMAIN
    finally:
        N.qsgw_chi0_destroy(ctx)


def test_sigx_and_chi0_contexts_reject_each_other(N):
    zt = z_block(3, 0, 0, 32, 2, 8, 40.0)
    v = _dev(coulomb_v(3, 0, 8))
    sx = N.qsgw_sigx_init([32], N.QSGW_FP64)
    cx = N.qsgw_chi0_init([32], [0.1], 2.0, N.QSGW_FP64)
    try:
        with pytest.raises(N.QsgwError) as e:
            N.qsgw_chi0_accumulate(sx, 0, _dev(zt), 32, 2, 8, v, v, [0.0])
        assert e.value.status == N.QSGW_ERR_STATE
        with pytest.raises(N.QsgwError) as e:
            N.qsgw_eps_inv(sx, 0, v, torch.empty((1, 32, 32), dtype=torch.complex128, device="cuda"))
        assert e.value.status == N.QSGW_ERR_STATE
        with pytest.raises(N.QsgwError) as e:
            N.qsgw_sigx_accumulate(cx, 0, _dev(zt), 32, 2, 8, v)
        assert e.value.status == N.QSGW_ERR_STATE
    finally:
        N.qsgw_chi0_destroy(sx)
        N.qsgw_chi0_destroy(cx)


def test_sigx_paper_size_sampled(N):
    """Sigma^x at the benchmark's (InAs)6(GaSb)6 size: n_qp = 428, 16 k-points x 276 occupied x
    3139 product-basis functions (13,861,824 columns), Z drawn on the device one k-point at a
    time, mixed precision. Four sampled rows and columns against the oracle over all columns."""
    from synthetic import z_rows
    n_qp, n_pb, n_occ, n_k, seed = 428, 3139, 276, 16, 1
    rows = np.array([0, 101, 300, 427])
    ctx = N.qsgw_sigx_init([n_qp], N.QSGW_MIXED_F16X3)
    try:
        Z = torch.empty((n_occ * n_pb, n_qp), dtype=torch.complex128, device="cuda")
        for k in range(n_k):
            N.qsgw_synth_z(seed, 7, k, n_qp, n_occ, n_pb, 100.0, Z, n_qp)
            v = _dev(coulomb_v(seed, k, n_pb))
            N.qsgw_sigx_accumulate(ctx, 0, Z, n_qp, n_occ, n_pb, v)
            N.qsgw_chi0_sync(ctx)
        del Z
        out = torch.empty((n_qp, n_qp), dtype=torch.complex128, device="cuda")
        N.qsgw_chi0_finalize(ctx, 0, out)
        got = out.cpu().numpy().T[np.ix_(rows, rows)]
    finally:
        N.qsgw_chi0_destroy(ctx)
    ZR = z_rows(seed, 7, rows, n_k, n_occ, lambda k: n_pb, 100.0)
    ref = oracle.sigx(ZR, [n_occ] * n_k, n_pb, np.stack([coulomb_v(seed, k, n_pb) for k in range(n_k)]))
    assert rel_fro(got, ref) <= 1e-6, rel_fro(got, ref)
    dg = np.sqrt(np.abs(np.diag(ref)))
    assert np.all(np.abs(got - ref) <= 1e-6 * np.outer(dg, dg))
