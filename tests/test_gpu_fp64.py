"""FP64 path on the GPU against the FP64 oracle, element by element, through the C ABI."""
import numpy as np
import pytest

import oracle
from synthetic import TINY, MEDIUM, coulomb_v, eps_occ, eps_unocc, z_block, z_rows
from synthetic.workloads import Workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def N():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_03477_gb300 import native
    native.load()
    return native


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run_workload(N, wl, prec, q=0, ks=None, host=False, split=1):
    """Accumulate k-points of a workload through the C ABI; returns (chi0 [l,I,J] numpy, Zrows, delta)."""
    n, L = wl.n_pb(q), wl.n_omega
    ctx = N.qsgw_chi0_init([n], wl.omega, wl.spin, prec)
    Zr, ds = [], []
    try:
        for k in (range(wl.n_k) if ks is None else ks):
            nu = wl.n_unocc(q, k)
            zt = z_block(wl.seed, q, k, n, wl.n_occ, nu, wl.s_div)
            eo, eu = eps_occ(wl.seed, q, k, wl.n_occ), eps_unocc(wl.seed, q, k, nu)
            Zr.append(zt.T)
            ds.append(oracle.delta(eo, eu)[0])
            if split == 1:
                Z, EO, EU = (zt, eo, eu) if host else (_dev(zt), _dev(eo), _dev(eu))
                N.qsgw_chi0_accumulate(ctx, 0, Z, n, wl.n_occ, nu, EO, EU, wl.omega)
            else:  # split the occupied index across calls: same columns, different call boundaries
                bounds = np.linspace(0, wl.n_occ, split + 1).astype(int)
                for a, b in zip(bounds[:-1], bounds[1:]):
                    if b > a:
                        N.qsgw_chi0_accumulate(ctx, 0, _dev(zt[a * nu:b * nu]), n, b - a, nu, _dev(eo[a:b]), _dev(eu),
                                               wl.omega)
        chi = torch.empty((L, n, n), dtype=torch.complex128, device="cuda")
        N.qsgw_chi0_finalize(ctx, 0, chi)
        out = chi.cpu().numpy().transpose(0, 2, 1)
    finally:
        N.qsgw_chi0_destroy(ctx)
    return out, np.concatenate(Zr, axis=1), np.concatenate(ds)


def rel_fro(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_tiny_fp64_chi0_and_w(N):
    chi, Z, d = run_workload(N, TINY, N.QSGW_FP64)
    ref = oracle.chi0_full(Z, d, TINY.omega, TINY.spin)
    for l in range(TINY.n_omega):
        assert rel_fro(chi[l], ref[l]) < 1e-12
        assert np.abs(chi[l] - ref[l]).max() < 1e-12 * np.abs(ref[l]).max()
        assert np.array_equal(chi[l], chi[l].conj().T)
        assert np.all(np.diag(chi[l]).imag == 0)
    # eps and W through the ABI against the oracle on the oracle's chi0
    n, L = TINY.n_pb(0), TINY.n_omega
    v = coulomb_v(TINY.seed, 0, n)
    ctx = N.qsgw_chi0_init([n], TINY.omega, TINY.spin, N.QSGW_FP64)
    try:
        for k in range(TINY.n_k):
            nu = TINY.n_unocc(0, k)
            zt = z_block(TINY.seed, 0, k, n, TINY.n_occ, nu, TINY.s_div)
            N.qsgw_chi0_accumulate(ctx, 0, _dev(zt), n, TINY.n_occ, nu, _dev(eps_occ(TINY.seed, 0, k, TINY.n_occ)),
                                   _dev(eps_unocc(TINY.seed, 0, k, nu)), TINY.omega)
        W = torch.empty((L, n, n), dtype=torch.complex128, device="cuda")
        E = torch.empty_like(W)
        Wc = torch.empty_like(W)
        info = N.qsgw_eps_inv(ctx, 0, _dev(v), W, E, n_omega=L)
        assert np.all(info == 0)
        N.qsgw_eps_inv(ctx, 0, _dev(v), Wc, None, correlation_only=True, n_omega=L)
    finally:
        N.qsgw_chi0_destroy(ctx)
    eps_ref, W_ref, Wc_ref, info_ref = oracle.eps_w(ref, v)
    Wg, Eg, Wcg = (x.cpu().numpy().transpose(0, 2, 1) for x in (W, E, Wc))
    for l in range(L):
        assert rel_fro(Eg[l], eps_ref[l]) < 1e-12
        assert rel_fro(Wg[l], W_ref[l]) < 1e-10
        assert np.abs(np.diag(Wg[l]) - np.diag(W_ref[l])).max() < 1e-10 * np.abs(np.diag(W_ref[l])).max()
        assert np.abs(Wcg[l] - Wc_ref[l]).max() < 1e-10 * v.max()
        assert np.array_equal(Wg[l], Wg[l].conj().T)


@pytest.mark.parametrize("n_pb,n_occ,n_unocc,L", [(1, 1, 1, 1), (100, 3, 7, 5), (130, 5, 13, 16), (64, 1, 1, 2)])
def test_ragged_shapes_fp64(N, n_pb, n_occ, n_unocc, L):
    wl = Workload(f"ragged {n_pb}", n_q=1, n_k=2, n_occ=n_occ, n_omega=L, s_div=50.0, n_pb_fixed=n_pb,
                  n_unocc_fixed=n_unocc, seed=7)
    chi, Z, d = run_workload(N, wl, N.QSGW_FP64)
    ref = oracle.chi0_full(Z, d, wl.omega, wl.spin)
    assert rel_fro(chi, ref) < 1e-12
    assert np.abs(chi - ref).max() <= 1e-12 * np.abs(ref).max()


def test_split_invariance_and_host_staging(N):
    wl = Workload("split", n_q=1, n_k=3, n_occ=6, n_omega=4, s_div=30.0, n_pb_fixed=96, n_unocc_fixed=20, seed=3)
    a, Z, d = run_workload(N, wl, N.QSGW_FP64)
    b, _, _ = run_workload(N, wl, N.QSGW_FP64, split=3)
    c, _, _ = run_workload(N, wl, N.QSGW_FP64, host=True)
    ref = oracle.chi0_full(Z, d, wl.omega, wl.spin)
    assert rel_fro(a, ref) < 1e-12 and rel_fro(b, ref) < 1e-12
    assert rel_fro(a, b) < 1e-13
    assert np.array_equal(a, c)


def test_domain_error_is_sticky_and_reported(N):
    n = 32
    ctx = N.qsgw_chi0_init([n], [0.01, 0.1], 2.0, N.QSGW_FP64)
    try:
        zt = z_block(1, 0, 0, n, 2, 3, 16.0)
        eo = np.array([-0.5, 0.2])
        eu = np.array([0.1, 0.3, 0.9])  # 0.1 - 0.2 < 0
        N.qsgw_chi0_accumulate(ctx, 0, _dev(zt), n, 2, 3, _dev(eo), _dev(eu), [0.01, 0.1])
        chi = torch.empty((2, n, n), dtype=torch.complex128, device="cuda")
        with pytest.raises(N.QsgwError) as e:
            N.qsgw_chi0_finalize(ctx, 0, chi)
        assert e.value.status == N.QSGW_ERR_DOMAIN
        N.qsgw_chi0_sync(ctx)  # cleared once reported
        with pytest.raises(N.QsgwError) as e:  # omega grid mismatch: synchronous argument error
            N.qsgw_chi0_accumulate(ctx, 0, _dev(zt), n, 2, 3, _dev(eo), _dev(eu), [0.01, 0.2])
        assert e.value.status == N.QSGW_ERR_ARG
    finally:
        N.qsgw_chi0_destroy(ctx)


def test_not_positive_definite_reports_info(N):
    """A negative spin factor makes chi0 positive semidefinite, so eps = 1 - D chi0 D loses definiteness."""
    n = 40
    om = [0.01, 30.0]
    ctx = N.qsgw_chi0_init([n], om, -2.0, N.QSGW_FP64)
    try:
        zt = z_block(1, 0, 0, n, 8, 32, 16.0) * 10.0
        N.qsgw_chi0_accumulate(ctx, 0, _dev(zt), n, 8, 32, _dev(eps_occ(1, 0, 0, 8)), _dev(eps_unocc(1, 0, 0, 32)), om)
        W = torch.empty((2, n, n), dtype=torch.complex128, device="cuda")
        info = N.qsgw_eps_inv(ctx, 0, _dev(np.full(n, 50.0)), W, n_omega=2, raise_not_pd=False)
        assert info[0] > 0
    finally:
        N.qsgw_chi0_destroy(ctx)
    # the index is that of the first non-positive pivot of a Cholesky factorisation of eps
    d = oracle.delta(eps_occ(1, 0, 0, 8), eps_unocc(1, 0, 0, 32))[0]
    chi = oracle.chi0_full(np.ascontiguousarray(zt.T), d, np.array(om), -2.0)
    _, _, _, info_ref = oracle.eps_w(chi, np.full(n, 50.0), want_eps=False, want_wc=False)
    assert info_ref[0] > 0 and list(info) == list(info_ref)


def test_device_generator_matches_host_generator(N):
    n, no, nu = 70, 3, 11
    Z = torch.empty((no * nu, n + 2), dtype=torch.complex128, device="cuda")
    N.qsgw_synth_z(1, 5, 9, n, no, nu, 200.0, Z, n + 2)
    torch.cuda.synchronize()
    got = Z.cpu().numpy()[:, :n]
    ref = z_block(1, 5, 9, n, no, nu, 200.0)
    assert np.abs(got - ref).max() <= 4e-16 * np.abs(ref).max() * 8


def test_accumulate_synthetic_equals_explicit(N):
    wl = Workload("synthetic", n_q=1, n_k=3, n_occ=4, n_omega=3, s_div=40.0, n_pb_fixed=80, n_unocc_fixed=9, seed=1)
    a, Z, d = run_workload(N, wl, N.QSGW_FP64)
    n = wl.n_pb(0)
    ctx = N.qsgw_chi0_init([n], wl.omega, wl.spin, N.QSGW_FP64)
    try:
        eo = np.concatenate([eps_occ(wl.seed, 0, k, wl.n_occ) for k in range(wl.n_k)])
        eu = np.concatenate([eps_unocc(wl.seed, 0, k, 9) for k in range(wl.n_k)])
        N.qsgw_chi0_accumulate_synthetic(ctx, 0, wl.seed, 0, 0, wl.n_k, wl.n_occ, [9] * wl.n_k, _dev(eo), _dev(eu),
                                         wl.s_div)
        chi = torch.empty((wl.n_omega, n, n), dtype=torch.complex128, device="cuda")
        N.qsgw_chi0_finalize(ctx, 0, chi)
        b = chi.cpu().numpy().transpose(0, 2, 1)
    finally:
        N.qsgw_chi0_destroy(ctx)
    assert rel_fro(a, b) < 1e-14


def test_medium_fp64_sampled_entries(N):
    """n_pb=1500, L=12 at full size over two k-points (FP64 runs at ~1 TFLOP/s on this part), sampled entries."""
    wl, ks = MEDIUM, [0, 37]
    n = wl.n_pb(0)
    ctx = N.qsgw_chi0_init([n], wl.omega, wl.spin, N.QSGW_FP64)
    try:
        Zd = torch.empty((wl.n_occ * 400, n), dtype=torch.complex128, device="cuda")
        for k in ks:
            N.qsgw_synth_z(wl.seed, 0, k, n, wl.n_occ, 400, wl.s_div, Zd, n)
            N.qsgw_chi0_accumulate(ctx, 0, Zd, n, wl.n_occ, 400, _dev(eps_occ(wl.seed, 0, k, wl.n_occ)),
                                   _dev(eps_unocc(wl.seed, 0, k, 400)), wl.omega)
        chi = torch.empty((wl.n_omega, n, n), dtype=torch.complex128, device="cuda")
        N.qsgw_chi0_finalize(ctx, 0, chi)
        got = chi.cpu().numpy().transpose(0, 2, 1)
    finally:
        N.qsgw_chi0_destroy(ctx)
    rng = np.random.default_rng(2)
    I = np.unique(np.concatenate([[0, 63, 64, 1499], rng.integers(0, n, 8)]))
    J = np.unique(np.concatenate([[0, 127, 1436, 1499], rng.integers(0, n, 8)]))
    ZI = np.concatenate([z_rows(wl.seed, 0, I, k + 1, wl.n_occ, lambda kk: 400, wl.s_div, k_begin=k) for k in ks], 1)
    ZJ = np.concatenate([z_rows(wl.seed, 0, J, k + 1, wl.n_occ, lambda kk: 400, wl.s_div, k_begin=k) for k in ks], 1)
    d = np.concatenate([oracle.delta(eps_occ(wl.seed, 0, k, wl.n_occ), eps_unocc(wl.seed, 0, k, 400))[0] for k in ks])
    ref = oracle.chi0_rows(ZI, ZJ, d, wl.omega, wl.spin)  # [l, i, j]
    sub = got[:, I][:, :, J]
    assert np.abs(sub - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.linalg.norm(sub - ref) <= 1e-12 * np.linalg.norm(ref)
