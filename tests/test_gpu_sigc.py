"""The imaginary-axis correlation self-energy I^c, Eq. (sigci), on the GPU against the FP64 oracle.

I^c is a general complex contraction (not a Hermitian update), so the bound is per element and
relative to the sum of the magnitudes of its terms,
  A_nm = sum_{k,n',i} |w_i| (|Z_{n'n}|^T |W^c_i| |Z_{n'm}|),
the standard error bound of a matrix product: FP64 <= 1e-12 A, mixed <= 2e-6 A (both contractions
round their inputs to FP32 once: 2^-23 each, plus the exact-digit truncation).

W^c is a realistic one: the oracle's W^c of a synthetic chi0 (negative semidefinite, decaying
along the imaginary axis), made exactly Hermitian. Cases: two k-points with ragged sizes and one
target degenerate with a band (dE = 0); band batches of 5, 5, 2 with n_qp = 700 (three row tiles
of the final product, a second operand block at row 768); determinism; reset; the error paths."""
import numpy as np
import pytest

import oracle
from synthetic import z_block
from synthetic.workloads import Workload

from test_gpu_fp64 import _dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

L = 6
OMEGA = Workload("s", n_q=1, n_k=1, n_occ=1, n_omega=L, s_div=1.0).omega


@pytest.fixture(scope="module")
def N():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_03477_gb300 import native
    native.load()
    return native


def _wc(n_pb, seed):
    """W^c[l, mu, nu] from the oracle's chi0 -> eps -> W^c chain on synthetic columns."""
    rng = np.random.default_rng(seed)
    zt = z_block(seed, 0, 0, n_pb, 6, 50, 30.0)
    d = rng.uniform(0.05, 3.0, zt.shape[0])
    chi = oracle.chi0_full(zt.T, d, OMEGA, 2.0)
    v = 4 * np.pi / rng.uniform(0.3, 6.0, n_pb) ** 2
    _, _, wc, info = oracle.eps_w(chi, v, want_eps=False, want_wc=True)
    assert np.all(np.asarray(info) == 0)
    return 0.5 * (wc + wc.conj().transpose(0, 2, 1))


def _case(seed, n_qp, n_pb, bands):
    rng = np.random.default_rng(seed)
    Zc = [z_block(seed, 1, k, n_pb, nb, n_qp, 20.0) for k, nb in enumerate(bands)]  # (nb * n_qp, n_pb)
    e_qp = np.sort(rng.uniform(-0.4, 0.4, n_qp))
    e_band = [np.sort(rng.uniform(-0.8, 3.0, nb)) for nb in bands]
    e_band[0][min(2, bands[0] - 1)] = e_qp[0]  # one degenerate pair: dE = 0
    Wc = [_wc(n_pb, seed + 100 + k) for k in range(len(bands))]
    return Zc, e_qp, e_band, Wc


def _gpu(N, prec, n_qp, n_pb, Zc, e_qp, e_band, Wc):
    ctx = N.qsgw_sigc_init(n_qp, n_pb, OMEGA, prec)
    try:
        keep = []
        for k in range(len(Zc)):
            keep.append((_dev(Zc[k]), _dev(e_band[k]), _dev(np.ascontiguousarray(Wc[k].transpose(0, 2, 1)))))
            eq = _dev(e_qp)
            keep.append(eq)
            N.qsgw_sigc_accumulate(ctx, keep[-2][0], n_pb, len(e_band[k]), eq, keep[-2][1], keep[-2][2])
        out = torch.empty((n_qp, n_qp), dtype=torch.complex128, device="cuda")
        N.qsgw_sigc_finalize(ctx, out)
        return out.cpu().numpy().T  # [n, m]
    finally:
        N.qsgw_chi0_destroy(ctx)


def _bound(Zc, e_qp, e_band, Wc):
    n_qp = e_qp.size
    A = np.zeros((n_qp, n_qp))
    for Z, eb, W in zip(Zc, e_band, Wc):
        for b in range(eb.size):
            Zb = np.abs(Z[b * n_qp:(b + 1) * n_qp])
            w = np.abs(np.array([oracle.sigc_weights(e - eb[b], OMEGA) for e in e_qp]))  # [n, i]
            for i in range(L):
                A += w[:, i:i + 1] * (Zb @ np.abs(W[i]) @ Zb.T)
    return A


@pytest.mark.parametrize("prec_name,tol", [("QSGW_FP64", 1e-12), ("QSGW_MIXED_F16X3", 2e-6)])
@pytest.mark.parametrize("n_qp,n_pb,bands", [(5, 37, [7, 3]), (700, 70, [12])])
def test_sigc_against_oracle(N, prec_name, tol, n_qp, n_pb, bands):
    Zc, e_qp, e_band, Wc = _case(31, n_qp, n_pb, bands)
    ref = oracle.sigc(Zc, e_qp, e_band, OMEGA, Wc)
    A = _bound(Zc, e_qp, e_band, Wc)
    got = _gpu(N, getattr(N, prec_name), n_qp, n_pb, Zc, e_qp, e_band, Wc)
    err = np.abs(got - ref)
    assert np.all(err <= tol * A + 1e-300), (err / A).max()
    assert np.linalg.norm(ref) > 0 and np.all(np.isfinite(got))


def test_sigc_deterministic_and_reset(N):
    n_qp, n_pb = 9, 40
    Zc, e_qp, e_band, Wc = _case(37, n_qp, n_pb, [6])
    a = _gpu(N, N.QSGW_MIXED_F16X3, n_qp, n_pb, Zc, e_qp, e_band, Wc)
    b = _gpu(N, N.QSGW_MIXED_F16X3, n_qp, n_pb, Zc, e_qp, e_band, Wc)
    assert np.array_equal(a, b)
    ctx = N.qsgw_sigc_init(n_qp, n_pb, OMEGA, N.QSGW_MIXED_F16X3)
    try:
        Z, eb, W, eq = _dev(Zc[0]), _dev(e_band[0]), _dev(np.ascontiguousarray(Wc[0].transpose(0, 2, 1))), _dev(e_qp)
        N.qsgw_sigc_accumulate(ctx, Z, n_pb, 6, eq, eb, W)
        N.qsgw_chi0_reset(ctx, 0)
        out = torch.empty((n_qp, n_qp), dtype=torch.complex128, device="cuda")
        N.qsgw_sigc_finalize(ctx, out)
        assert torch.count_nonzero(out).item() == 0
        N.qsgw_sigc_accumulate(ctx, Z, n_pb, 6, eq, eb, W)
        N.qsgw_sigc_finalize(ctx, out)
        assert np.array_equal(out.cpu().numpy().T, a)
    finally:
        N.qsgw_chi0_destroy(ctx)


def test_sigc_errors(N):
    n_qp, n_pb = 4, 16
    with pytest.raises(N.QsgwError):
        N.qsgw_sigc_init(n_qp, n_pb, [0.1, 0.1, 0.5])  # not increasing
    with pytest.raises(N.QsgwError):
        N.qsgw_sigc_init(n_qp, n_pb, [0.0, 0.5])  # omega_0 must be > 0
    Zc, e_qp, e_band, Wc = _case(41, n_qp, n_pb, [3])
    ctx = N.qsgw_sigc_init(n_qp, n_pb, OMEGA, N.QSGW_FP64)
    try:
        Z, eb, W = _dev(Zc[0]), _dev(e_band[0]), _dev(np.ascontiguousarray(Wc[0].transpose(0, 2, 1)))
        bad = e_qp.copy()
        bad[1] = np.nan
        eq = _dev(bad)
        N.qsgw_sigc_accumulate(ctx, Z, n_pb, 3, eq, eb, W)
        out = torch.empty((n_qp, n_qp), dtype=torch.complex128, device="cuda")
        with pytest.raises(N.QsgwError) as ei:
            N.qsgw_sigc_finalize(ctx, out)
        assert ei.value.status == -2  # QSGW_ERR_DOMAIN
        with pytest.raises(N.QsgwError) as ei:  # chi0-only call on this context
            N.qsgw_chi0_finalize(ctx, 0, out)
        assert ei.value.status == -7  # QSGW_ERR_STATE
    finally:
        N.qsgw_chi0_destroy(ctx)
    ctx = N.qsgw_chi0_init([n_pb], OMEGA, 2.0, N.QSGW_FP64)
    try:
        with pytest.raises(N.QsgwError) as ei:
            N.qsgw_sigc_accumulate(ctx, Z, n_pb, 3, _dev(e_qp), eb, W)
        assert ei.value.status == -7
    finally:
        N.qsgw_chi0_destroy(ctx)


def test_sigc_medium_shapes_sampled(N):
    """I^c at the benchmark's shapes: n_pb = 1500, 12 frequencies, n_qp = 64 targets, 64 bands (one
    band batch of 4096 rows), mixed precision, W^c of plasmon-pole form -A/(1 + w^2/Wp^2) P with P
    Hermitian positive definite. Checked on 4 sampled targets (rows and columns) against the
    oracle, which needs only those targets' columns of Z."""
    from synthetic import MEDIUM as W
    n_qp, n_pb, n_band = 64, 1500, 64
    om = W.omega
    rng = np.random.default_rng(43)
    B = rng.standard_normal((n_pb, n_pb)) + 1j * rng.standard_normal((n_pb, n_pb))
    P = B @ B.conj().T / n_pb
    P = 0.5 * (P + P.conj().T)
    f = 0.8 / (1.0 + (om / 0.6) ** 2)
    Wc = -f[:, None, None] * P[None]
    Zc = z_block(47, 2, 0, n_pb, n_band, n_qp, 200.0)
    e_qp = np.sort(rng.uniform(-0.3, 0.4, n_qp))
    e_band = np.sort(rng.uniform(-0.8, 3.0, n_band))
    ctx = N.qsgw_sigc_init(n_qp, n_pb, om, N.QSGW_MIXED_F16X3)
    try:
        Zd, eq, eb = _dev(Zc), _dev(e_qp), _dev(e_band)
        Wd = _dev(np.ascontiguousarray(Wc.transpose(0, 2, 1)))
        N.qsgw_sigc_accumulate(ctx, Zd, n_pb, n_band, eq, eb, Wd)
        out = torch.empty((n_qp, n_qp), dtype=torch.complex128, device="cuda")
        N.qsgw_sigc_finalize(ctx, out)
        got = out.cpu().numpy().T
    finally:
        N.qsgw_chi0_destroy(ctx)
    t = np.array([0, 21, 40, 63])
    cols = (np.arange(n_band)[:, None] * n_qp + t[None, :]).ravel()  # rows (n', t) of the sample
    Zs = Zc[cols]
    ref = oracle.sigc([Zs], e_qp[t], [e_band], om, [Wc])
    A = np.zeros((t.size, t.size))
    for b in range(n_band):
        Zb = np.abs(Zs[b * t.size:(b + 1) * t.size])
        w = np.abs(np.array([oracle.sigc_weights(e - e_band[b], om) for e in e_qp[t]]))
        A += sum(w[:, i:i + 1] * (Zb @ np.abs(Wc[i]) @ Zb.T) for i in range(om.size))
    err = np.abs(got[np.ix_(t, t)] - ref)
    assert np.all(err <= 2e-6 * A), (err / A).max()
