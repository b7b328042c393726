"""The large streamed workload at full size: n_pb = 4000, 64 k-points x 120 occupied x 1200
unoccupied (K = 9,216,000), 16 frequencies. Z is drawn on the device per k-point inside
qsgw_chi0_accumulate_synthetic and never stored whole. The oracle checks a sampled block of
rows (incl. the first/last row and the diagonal of the block) over all 9.2M columns."""
import numpy as np
import pytest

import oracle
from synthetic import LARGE, eps_occ, eps_unocc, z_rows

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


def test_large_streamed_mixed_sampled(N):
    wl = LARGE
    n, L, no, nu = wl.n_pb(0), wl.n_omega, wl.n_occ, wl.n_unocc_fixed
    ctx = N.qsgw_chi0_init([n], wl.omega, wl.spin, N.QSGW_MIXED_F16X3)
    try:
        eo = _dev(np.concatenate([eps_occ(wl.seed, 0, k, no) for k in range(wl.n_k)]))
        eu = _dev(np.concatenate([eps_unocc(wl.seed, 0, k, nu) for k in range(wl.n_k)]))
        N.qsgw_chi0_accumulate_synthetic(ctx, 0, wl.seed, 0, 0, wl.n_k, no, [nu] * wl.n_k, eo, eu, wl.s_div)
        chi = torch.empty((L, n, n), dtype=torch.complex128, device="cuda")
        N.qsgw_chi0_finalize(ctx, 0, chi)
        rng = np.random.default_rng(2)
        rows = np.unique(np.concatenate([[0, 3999, 2047, 2048], rng.integers(0, n, 4)]))
        sub = chi.cpu().numpy().transpose(0, 2, 1)[:, rows][:, :, rows]
        del chi
    finally:
        N.qsgw_chi0_destroy(ctx)
    ZS = z_rows(wl.seed, 0, rows, wl.n_k, no, lambda k: nu, wl.s_div)
    d = np.concatenate([oracle.delta(eps_occ(wl.seed, 0, k, no), eps_unocc(wl.seed, 0, k, nu))[0] for k in range(wl.n_k)])
    ref = oracle.chi0_rows(ZS, ZS, d, wl.omega, wl.spin)
    for l in range(L):
        dg = np.sqrt(np.abs(np.diag(ref[l])))
        assert np.all(np.abs(sub[l] - ref[l]) <= 1e-6 * np.outer(dg, dg)), l
        assert rel_fro(sub[l], ref[l]) <= 1e-6
