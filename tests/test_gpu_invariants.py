"""Invariants the paper states or implies (Sec. 2), checked on the GPU's own output in both
precisions (mid-size case, K > n_pb so every chi0(i omega) has full rank):

* chi0(i omega) is exactly Hermitian and negative semidefinite (every weight -2 Delta/(Delta^2 +
  omega^2) < 0);
* Loewner monotonicity in omega: chi0(i omega_{l+1}) - chi0(i omega_l) is positive semidefinite
  (|w_l| decreases in omega for every Delta);
* W = v^{1/2} eps^{-1} v^{1/2} is positive definite and W <= v (eps >= I); W^c = W - v is negative
  semidefinite.

Tolerances are relative to the spectral norm: 1e-6 for the mixed path, 1e-12 for FP64."""
import numpy as np
import pytest

from synthetic import coulomb_v
from synthetic.workloads import Workload

from test_gpu_fp64 import _dev, run_workload

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def N():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_03477_gb300 import native
    native.load()
    return native


@pytest.mark.parametrize("prec_name,tol", [("QSGW_FP64", 1e-12), ("QSGW_MIXED_F16X3", 1e-6)])
def test_gpu_output_invariants(N, prec_name, tol):
    wl = Workload("inv", n_q=1, n_k=2, n_occ=8, n_omega=12, s_div=50.0, n_pb_fixed=160, n_unocc_fixed=125, seed=21)
    n, L = 160, 12
    prec = getattr(N, prec_name)
    chi, _, _ = run_workload(N, wl, prec)  # [l, I, J]
    for l in range(L):
        assert np.array_equal(chi[l], chi[l].conj().T)
        ev = np.linalg.eigvalsh(chi[l])
        assert ev.max() <= tol * np.abs(ev).max(), (l, ev.max())
    for l in range(L - 1):
        ev = np.linalg.eigvalsh(chi[l + 1] - chi[l])
        assert ev.min() >= -tol * np.abs(np.linalg.eigvalsh(chi[l])).max(), (l, ev.min())

    v = coulomb_v(wl.seed, 0, n)
    ctx = N.qsgw_chi0_init([n], wl.omega, wl.spin, prec)
    try:
        from synthetic import eps_occ, eps_unocc, z_block
        for k in range(wl.n_k):
            zt = z_block(wl.seed, 0, k, n, wl.n_occ, 125, wl.s_div)
            N.qsgw_chi0_accumulate(ctx, 0, _dev(zt), n, wl.n_occ, 125, _dev(eps_occ(wl.seed, 0, k, wl.n_occ)),
                                   _dev(eps_unocc(wl.seed, 0, k, 125)), wl.omega)
        W = torch.empty((L, n, n), dtype=torch.complex128, device="cuda")
        Wc = torch.empty_like(W)
        N.qsgw_eps_inv(ctx, 0, _dev(v), W, n_omega=L)
        N.qsgw_eps_inv(ctx, 0, _dev(v), Wc, None, correlation_only=True, n_omega=L)
        W = W.cpu().numpy().transpose(0, 2, 1)
        Wc = Wc.cpu().numpy().transpose(0, 2, 1)
    finally:
        N.qsgw_chi0_destroy(ctx)
    V = np.diag(v)
    for l in range(L):
        scale = np.abs(np.linalg.eigvalsh(V)).max()
        assert np.linalg.eigvalsh(W[l]).min() > 0.0
        assert np.linalg.eigvalsh(V - W[l]).min() >= -tol * scale
        assert np.linalg.eigvalsh(Wc[l]).max() <= tol * scale
