"""eps^{-1} and W in FP64 accuracy in both precisions (Eqs. (dielectricfunction), (screenedcoulomb),
(wc); Alg. 1 MATINV in double precision). The mixed contexts run the rank-32 updates of the block
sweep on the tensor cores in exact integer digits, the FP64 contexts on DFMA. To isolate the inverse
from the mixed chi0, W is compared with the oracle's eps -> Cholesky inverse -> W applied to the
GPU's own chi0: relative Frobenius and diag W <= 1e-10 per frequency, W^c <= 1e-10 v_max, and W
exactly Hermitian. Sizes cover one pivot block (n <= 32), a ragged last pivot block, one and several
64 x 64 tiles and a ragged last tile."""
import numpy as np
import pytest

import oracle
from synthetic import coulomb_v, eps_occ, eps_unocc, omega_grid, z_block

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


@pytest.mark.parametrize("prec_name", ["QSGW_MIXED_F16X3", "QSGW_FP64"])
@pytest.mark.parametrize("n,L,spin", [(1, 2, 2.0), (31, 3, 2.0), (33, 4, 8.0), (64, 2, 30.0), (100, 5, 60.0),
                                      (130, 3, 200.0), (257, 2, 400.0)])
def test_w_against_oracle_on_the_gpus_own_chi0(N, prec_name, n, L, spin):
    no, nu = 8, 48
    om = omega_grid(L)
    zt = z_block(11, n, 0, n, no, nu, 40.0)
    v = coulomb_v(11, n, n)
    ctx = N.qsgw_chi0_init([n], om, spin, getattr(N, prec_name))
    try:
        N.qsgw_chi0_accumulate(ctx, 0, _dev(zt), n, no, nu, _dev(eps_occ(11, n, 0, no)), _dev(eps_unocc(11, n, 0, nu)), om)
        chi = torch.empty((L, n, n), dtype=torch.complex128, device="cuda")
        N.qsgw_chi0_finalize(ctx, 0, chi)
        W = torch.empty_like(chi)
        Wc = torch.empty_like(chi)
        info = N.qsgw_eps_inv(ctx, 0, _dev(v), W, n_omega=L)
        assert np.all(info == 0)
        N.qsgw_eps_inv(ctx, 0, _dev(v), Wc, correlation_only=True, n_omega=L)
    finally:
        N.qsgw_chi0_destroy(ctx)
    chi = chi.cpu().numpy().transpose(0, 2, 1)
    Wg, Wcg = (x.cpu().numpy().transpose(0, 2, 1) for x in (W, Wc))
    _, Wref, Wcref, info_ref = oracle.eps_w(chi, v)
    assert np.all(info_ref == 0)
    for l in range(L):
        assert rel_fro(Wg[l], Wref[l]) <= 1e-10, (l, rel_fro(Wg[l], Wref[l]))
        d = np.abs(np.diagonal(Wg[l]) - np.diagonal(Wref[l])) / np.abs(np.diagonal(Wref[l]))
        assert d.max() <= 1e-10, (l, d.max())
        assert np.abs(Wcg[l] - Wcref[l]).max() <= 1e-10 * v.max()
        assert np.array_equal(Wg[l], Wg[l].conj().T)
