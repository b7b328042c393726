"""Mixed-precision (tcgen05, exact-leading-digit BF16 slices) chi0 path against the FP64 oracle.

Tolerance: relative Frobenius error <= 1e-6 per frequency on chi0 and <= 1e-6 on diag W (the
accuracy bar of the mixed form). Per element, |err_IJ| <= 1e-6 * sqrt(|chi_II chi_JJ|), the
Cauchy-Schwarz scale of a semidefinite matrix.
"""
import numpy as np
import pytest

import oracle
from synthetic import MEDIUM, TINY, coulomb_v, eps_occ, eps_unocc, z_block, z_rows
from synthetic.workloads import Workload

from test_gpu_fp64 import _dev, rel_fro, run_workload

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


def _check_chi(chi, ref):
    for l in range(ref.shape[0]):
        assert rel_fro(chi[l], ref[l]) <= TOL, (l, rel_fro(chi[l], ref[l]))
        d = np.sqrt(np.abs(np.diag(ref[l])))
        assert np.all(np.abs(chi[l] - ref[l]) <= TOL * np.outer(d, d) + 1e-300)
        assert np.array_equal(chi[l], chi[l].conj().T)


def test_tiny_mixed(N):
    chi, Z, d = run_workload(N, TINY, N.QSGW_MIXED_F16X3)
    ref = oracle.chi0_full(Z, d, TINY.omega, TINY.spin)
    _check_chi(chi, ref)


@pytest.mark.parametrize("n_pb,n_occ,n_unocc,L", [(1, 1, 1, 1), (100, 3, 7, 5), (130, 5, 13, 16), (65, 7, 80, 12),
                                                  (200, 9, 61, 9), (70, 2, 300, 3),
                                                  # K = 2048 (one whole chunk), K = 2064 (a chunk + one K-block)
                                                  (96, 16, 128, 12), (96, 8, 258, 12),
                                                  # one frequency: the sqrt(w) row image serves both operands
                                                  (300, 9, 130, 1), (257, 16, 128, 1), (33, 3, 700, 1)])
def test_ragged_shapes_mixed(N, n_pb, n_occ, n_unocc, L):
    wl = Workload(f"ragged {n_pb}", n_q=1, n_k=2, n_occ=n_occ, n_omega=L, s_div=50.0, n_pb_fixed=n_pb,
                  n_unocc_fixed=n_unocc, seed=11)
    chi, Z, d = run_workload(N, wl, N.QSGW_MIXED_F16X3)
    ref = oracle.chi0_full(Z, d, wl.omega, wl.spin)
    _check_chi(chi, ref)


def test_split_invariance_mixed(N):
    wl = Workload("split", n_q=1, n_k=2, n_occ=12, n_omega=12, s_div=30.0, n_pb_fixed=150, n_unocc_fixed=90, seed=3)
    a, Z, d = run_workload(N, wl, N.QSGW_MIXED_F16X3)
    b, _, _ = run_workload(N, wl, N.QSGW_MIXED_F16X3, split=5)
    ref = oracle.chi0_full(Z, d, wl.omega, wl.spin)
    _check_chi(a, ref)
    _check_chi(b, ref)


def test_domain_error_mixed(N):
    n = 48
    ctx = N.qsgw_chi0_init([n], [0.01, 0.1], 2.0, N.QSGW_MIXED_F16X3)
    try:
        zt = z_block(1, 0, 0, n, 2, 3, 16.0)
        N.qsgw_chi0_accumulate(ctx, 0, _dev(zt), n, 2, 3, _dev(np.array([-0.5, 0.2])), _dev(np.array([0.1, 0.3, 0.9])),
                               [0.01, 0.1])
        chi = torch.empty((2, n, n), dtype=torch.complex128, device="cuda")
        with pytest.raises(N.QsgwError) as e:
            N.qsgw_chi0_finalize(ctx, 0, chi)
        assert e.value.status == N.QSGW_ERR_DOMAIN
    finally:
        N.qsgw_chi0_destroy(ctx)


def test_midsize_mixed_chi0_and_w(N):
    """n_pb=256 with four k-points of the medium generator (K=64000, 12 frequencies): full chi0 and W."""
    wl = Workload("mid", n_q=1, n_k=4, n_occ=40, n_omega=12, s_div=200.0, n_pb_fixed=256, n_unocc_fixed=400, seed=1)
    n, L = 256, 12
    chi, Z, d = run_workload(N, wl, N.QSGW_MIXED_F16X3)
    ref = oracle.chi0_full(Z, d, wl.omega, wl.spin)
    _check_chi(chi, ref)
    v = coulomb_v(wl.seed, 0, n)
    ctx = N.qsgw_chi0_init([n], wl.omega, wl.spin, N.QSGW_MIXED_F16X3)
    try:
        for k in range(wl.n_k):
            zt = z_block(wl.seed, 0, k, n, wl.n_occ, 400, wl.s_div)
            N.qsgw_chi0_accumulate(ctx, 0, _dev(zt), n, wl.n_occ, 400, _dev(eps_occ(wl.seed, 0, k, wl.n_occ)),
                                   _dev(eps_unocc(wl.seed, 0, k, 400)), wl.omega)
        W = torch.empty((L, n, n), dtype=torch.complex128, device="cuda")
        info = N.qsgw_eps_inv(ctx, 0, _dev(v), W, n_omega=L)
        assert np.all(info == 0)
        Wg = W.cpu().numpy().transpose(0, 2, 1)
    finally:
        N.qsgw_chi0_destroy(ctx)
    _, Wref, _, _ = oracle.eps_w(ref, v, want_eps=False, want_wc=False)
    for l in range(L):
        dW = np.abs(np.diag(Wg[l]) - np.diag(Wref[l])) / np.abs(np.diag(Wref[l]))
        assert dW.max() <= TOL, (l, dW.max())
        assert rel_fro(Wg[l], Wref[l]) <= TOL


def test_medium_mixed_full_size_sampled(N):
    """The medium workload at full size (n_pb=1500, 64 k-points, K=1.024M, 12 frequencies) in the
    launch configuration the benchmark times; oracle on a sampled block of entries incl. the diagonal."""
    wl = MEDIUM
    n = wl.n_pb(0)
    ctx = N.qsgw_chi0_init([n], wl.omega, wl.spin, N.QSGW_MIXED_F16X3)
    try:
        Zd = torch.empty((wl.n_occ * 400, n), dtype=torch.complex128, device="cuda")
        for k in range(wl.n_k):
            N.qsgw_synth_z(wl.seed, 0, k, n, wl.n_occ, 400, wl.s_div, Zd, n)
            N.qsgw_chi0_accumulate(ctx, 0, Zd, n, wl.n_occ, 400, _dev(eps_occ(wl.seed, 0, k, wl.n_occ)),
                                   _dev(eps_unocc(wl.seed, 0, k, 400)), wl.omega)
        chi = torch.empty((wl.n_omega, n, n), dtype=torch.complex128, device="cuda")
        N.qsgw_chi0_finalize(ctx, 0, chi)
        got = chi.cpu().numpy().transpose(0, 2, 1)
    finally:
        N.qsgw_chi0_destroy(ctx)
    rng = np.random.default_rng(4)
    S = np.unique(np.concatenate([[0, 63, 64, 1279, 1280, 1499], rng.integers(0, n, 6)]))
    ZS = z_rows(wl.seed, 0, S, wl.n_k, wl.n_occ, lambda k: 400, wl.s_div)
    d = np.concatenate([oracle.delta(eps_occ(wl.seed, 0, k, wl.n_occ), eps_unocc(wl.seed, 0, k, 400))[0]
                        for k in range(wl.n_k)])
    ref = oracle.chi0_rows(ZS, ZS, d, wl.omega, wl.spin)
    sub = got[:, S][:, :, S]
    for l in range(wl.n_omega):
        dg = np.sqrt(np.abs(np.diag(ref[l])))
        assert np.all(np.abs(sub[l] - ref[l]) <= TOL * np.outer(dg, dg))
        assert rel_fro(sub[l], ref[l]) <= TOL


def test_pinned_host_blocks_double_buffered(N):
    """Host Z from pinned memory, five blocks whose sizes grow and shrink (so both staging slots
    are reused and regrown while the copy stream runs ahead of the kernels): the result equals
    the device-pointer path bit for bit (same kernels on the same values), and the oracle."""
    n, L = 140, 12
    wl = Workload("pinned", n_q=1, n_k=5, n_occ=4, n_omega=L, s_div=40.0, n_pb_fixed=n, seed=5)
    shapes = [(4, 90), (6, 400), (3, 30), (8, 700), (5, 200)]  # (n_occ, n_unocc) per block
    blocks = []
    for k, (no, nu) in enumerate(shapes):
        zt = z_block(wl.seed, 0, k, n, no, nu, wl.s_div)
        blocks.append((zt, eps_occ(wl.seed, 0, k, no), eps_unocc(wl.seed, 0, k, nu), no, nu))

    def run(mode):
        ctx = N.qsgw_chi0_init([n], wl.omega, wl.spin, N.QSGW_MIXED_F16X3)
        keep = []
        try:
            for zt, eo, eu, no, nu in blocks:
                if mode == "pinned":  # pinned Z, pageable eps
                    Zh = torch.from_numpy(np.ascontiguousarray(zt)).pin_memory()
                    keep.append(Zh)  # pinned host data must stay unchanged until the sync
                    N.qsgw_chi0_accumulate(ctx, 0, Zh, n, no, nu, eo, eu, wl.omega)
                elif mode == "eps_host":  # device Z, pageable eps
                    Zd = _dev(zt)
                    keep.append(Zd)
                    N.qsgw_chi0_accumulate(ctx, 0, Zd, n, no, nu, eo.copy(), eu.copy(), wl.omega)
                else:
                    N.qsgw_chi0_accumulate(ctx, 0, _dev(zt), n, no, nu, _dev(eo), _dev(eu), wl.omega)
            chi = torch.empty((L, n, n), dtype=torch.complex128, device="cuda")
            N.qsgw_chi0_finalize(ctx, 0, chi)
            return chi.cpu().numpy().transpose(0, 2, 1)
        finally:
            N.qsgw_chi0_destroy(ctx)

    a, b, c = run("pinned"), run("device"), run("eps_host")
    assert np.array_equal(a, b) and np.array_equal(c, b)
    Z = np.concatenate([zt.T for zt, *_ in blocks], axis=1)
    d = np.concatenate([oracle.delta(eo, eu)[0] for _, eo, eu, _, _ in blocks])
    _check_chi(a, oracle.chi0_full(Z, d, wl.omega, wl.spin))


def test_complex64_input_is_bit_identical(N):
    """qsgw_chi0_accumulate_c64: the mixed path rounds Z to FP32 before forming digits, so
    complex64 input (device or pinned host) gives exactly the complex128 result; FP64 contexts
    reject it."""
    n, L = 150, 12
    wl = Workload("c64", n_q=1, n_k=2, n_occ=5, n_omega=L, s_div=40.0, n_pb_fixed=n, seed=9)
    shapes = [(5, 700), (3, 250)]
    blocks = []
    for k, (no, nu) in enumerate(shapes):
        zt = z_block(wl.seed, 0, k, n, no, nu, wl.s_div)
        blocks.append((zt, eps_occ(wl.seed, 0, k, no), eps_unocc(wl.seed, 0, k, nu), no, nu))

    def run(mode):
        ctx = N.qsgw_chi0_init([n], wl.omega, wl.spin, N.QSGW_MIXED_F16X3)
        keep = []
        try:
            for zt, eo, eu, no, nu in blocks:
                EO, EU = _dev(eo), _dev(eu)
                if mode == "c128":
                    N.qsgw_chi0_accumulate(ctx, 0, _dev(zt), n, no, nu, EO, EU, wl.omega)
                else:
                    z64 = torch.from_numpy(np.ascontiguousarray(zt.astype(np.complex64)))
                    z64 = z64.cuda() if mode == "c64_dev" else z64.pin_memory()
                    keep.append(z64)
                    N.qsgw_chi0_accumulate_c64(ctx, 0, z64, n, no, nu, EO, EU, wl.omega)
            chi = torch.empty((L, n, n), dtype=torch.complex128, device="cuda")
            N.qsgw_chi0_finalize(ctx, 0, chi)
            return chi.cpu().numpy().transpose(0, 2, 1)
        finally:
            N.qsgw_chi0_destroy(ctx)

    ref = run("c128")
    assert np.array_equal(run("c64_dev"), ref)
    assert np.array_equal(run("c64_host"), ref)
    Z = np.concatenate([zt.T for zt, *_ in blocks], axis=1)
    d = np.concatenate([oracle.delta(eo, eu)[0] for _, eo, eu, _, _ in blocks])
    _check_chi(ref, oracle.chi0_full(Z, d, wl.omega, wl.spin))
    ctx = N.qsgw_chi0_init([n], wl.omega, wl.spin, N.QSGW_FP64)
    try:
        zt, eo, eu, no, nu = blocks[0]
        with pytest.raises(N.QsgwError) as e:
            N.qsgw_chi0_accumulate_c64(ctx, 0, _dev(zt.astype(np.complex64)), n, no, nu, _dev(eo), _dev(eu), wl.omega)
        assert e.value.status == N.QSGW_ERR_ARG
    finally:
        N.qsgw_chi0_destroy(ctx)
