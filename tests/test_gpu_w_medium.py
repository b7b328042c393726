"""chi0 and W at the benchmark's product-basis size, n_pb = 1500, 12 imaginary frequencies, both
precisions through the C ABI against the FP64 oracle (Eqs. (polfx), (dielectricfunction),
(screenedcoulomb)). One k-point of the medium workload (16,000 columns) with the spin factor
scaled by 64 stands in for all 64 k-points: chi0 then has the magnitude of the full workload, so
eps has its conditioning, which is what the accuracy of W depends on. Bars: plain FP64 chi0
<= 1e-12 and W <= 1e-10 relative Frobenius; mixed chi0 <= 1e-6 relative Frobenius and diag W
<= 1e-6 relative, per frequency. The FP64 eps^{-1} (block sweep with Cholesky pivots) runs in
both precisions, here on 47 pivot blocks with a ragged last one (1500 = 46 * 32 + 28); in the mixed
precision its updates run on the tensor cores, checked at 1e-10 against the oracle's inverse of the
GPU's own chi0."""
import numpy as np
import pytest

import oracle
from synthetic import MEDIUM as W
from synthetic import coulomb_v, eps_occ, eps_unocc, z_block

from test_gpu_fp64 import rel_fro

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N_PB, N_OCC, N_UNOCC = 1500, W.n_occ, 400
SPIN = W.spin * W.n_k  # one k-point standing in for 64


@pytest.fixture(scope="module")
def N():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_03477_gb300 import native
    native.load()
    return native


@pytest.fixture(scope="module")
def case():
    zt = z_block(W.seed, 0, 0, N_PB, N_OCC, N_UNOCC, W.s_div)
    eo, eu = eps_occ(W.seed, 0, 0, N_OCC), eps_unocc(W.seed, 0, 0, N_UNOCC)
    d = oracle.delta(eo, eu)[0]
    v = coulomb_v(W.seed, 0, N_PB)
    chi = oracle.chi0_full(np.ascontiguousarray(zt.T), d, W.omega, SPIN)
    _, Wref, _, info = oracle.eps_w(chi, v, want_eps=False, want_wc=False)
    assert np.all(info == 0)
    return dict(zt=zt, eo=eo, eu=eu, v=v, chi=chi, W=Wref)


@pytest.mark.parametrize("prec_name", ["QSGW_FP64", "QSGW_MIXED_F16X3"])
def test_chi0_and_w_at_npb_1500(N, case, prec_name):
    L = W.n_omega
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    ctx = N.qsgw_chi0_init([N_PB], W.omega, SPIN, getattr(N, prec_name))
    try:
        N.qsgw_chi0_accumulate(ctx, 0, dev(case["zt"]), N_PB, N_OCC, N_UNOCC, dev(case["eo"]), dev(case["eu"]), W.omega)
        chi = torch.empty((L, N_PB, N_PB), dtype=torch.complex128, device="cuda")
        N.qsgw_chi0_finalize(ctx, 0, chi)
        Wg = torch.empty_like(chi)
        info = N.qsgw_eps_inv(ctx, 0, dev(case["v"]), Wg, n_omega=L)
        assert np.all(info == 0)
    finally:
        N.qsgw_chi0_destroy(ctx)
    chi = chi.cpu().numpy().transpose(0, 2, 1)
    Wg = Wg.cpu().numpy().transpose(0, 2, 1)
    fp64 = prec_name == "QSGW_FP64"
    for l in range(L):
        e_chi = rel_fro(chi[l], case["chi"][l])
        dW = np.diagonal(Wg[l]) - np.diagonal(case["W"][l])
        e_dw = np.abs(dW / np.diagonal(case["W"][l])).max()
        e_w = rel_fro(Wg[l], case["W"][l])
        if fp64:
            assert e_chi <= 1e-12 and e_w <= 1e-10 and e_dw <= 1e-10, (l, e_chi, e_w, e_dw)
        else:
            assert e_chi <= 1e-6 and e_dw <= 1e-6, (l, e_chi, e_w, e_dw)
        assert np.array_equal(Wg[l], Wg[l].conj().T)
    if not fp64:
        # the inverse itself (its updates on the tensor cores in exact integer digits) at FP64
        # accuracy: against the oracle's inverse of the GPU's own chi0
        _, Wown, _, info = oracle.eps_w(chi, case["v"], want_eps=False, want_wc=False)
        assert np.all(info == 0)
        for l in range(L):
            assert rel_fro(Wg[l], Wown[l]) <= 1e-10, (l, rel_fro(Wg[l], Wown[l]))
