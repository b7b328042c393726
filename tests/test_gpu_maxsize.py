"""The largest product basis the library accepts (n_pb = 16384, the limit in include/qsgw.h), in
both precisions, against the oracle on sampled full rows (first, last and interior rows against
all 16384 columns). A short K keeps it quick; the point is the index arithmetic at the largest
accumulator (mixed: 2 frequencies x 2 parts x 16384^2 elements, 17 GB) and tile counts."""
import numpy as np
import pytest

import oracle
from synthetic import eps_occ, eps_unocc, z_block

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


@pytest.mark.parametrize("prec_name,tol", [("QSGW_MIXED_F16X3", 1e-6), ("QSGW_FP64", 1e-12)])
def test_max_npb_sampled_rows(N, prec_name, tol):
    n, no, nu, om = 16384, 2, 20, np.array([0.01, 0.3])
    zt = z_block(13, 0, 0, n, no, nu, 2000.0)  # (K, n): the column-major n x K matrix
    eo, eu = eps_occ(13, 0, 0, no), eps_unocc(13, 0, 0, nu)
    ctx = N.qsgw_chi0_init([n], om, 2.0, getattr(N, prec_name))
    try:
        N.qsgw_chi0_accumulate(ctx, 0, _dev(zt), n, no, nu, _dev(eo), _dev(eu), om)
        chi = torch.empty((2, n, n), dtype=torch.complex128, device="cuda")
        N.qsgw_chi0_finalize(ctx, 0, chi)
        rows = np.array([0, 1, 4095, 8191, 12000, n - 2, n - 1])
        # column-major per frequency: element (i, j) at j * n + i, i.e. chi[l, j, i] in torch indexing
        got = chi[:, :, torch.as_tensor(rows, device="cuda")].cpu().numpy().transpose(0, 2, 1)  # [l, row, J]
        del chi
    finally:
        N.qsgw_chi0_destroy(ctx)
    Zr = np.ascontiguousarray(zt.T)
    d = oracle.delta(eo, eu)[0]
    ref = oracle.chi0_rows(Zr[rows], Zr, d, om, 2.0)  # [l, row, J]
    for l in range(2):
        assert rel_fro(got[l], ref[l]) <= tol, (l, rel_fro(got[l], ref[l]))
        assert np.abs(got[l] - ref[l]).max() <= 10 * tol * np.abs(ref[l]).max()
