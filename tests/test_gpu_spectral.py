"""Real-axis route, Eqs. (impolf) and (hilbert), on the GPU against the FP64 oracle:

* the spectral weights S_j of every histogram bin (FP64 <= 1e-12, mixed <= 1e-6 relative per bin,
  plus the per-element Cauchy-Schwarz bound of a semidefinite matrix), on ragged shapes with
  columns outside the bins;
* chi0 on the real axis at sampled bin centres (Hermitian part from the Hilbert transformation,
  anti-Hermitian part -pi S_i / width), per element within the bound the S_j bound implies;
* deterministic: two runs give the same bits; Delta <= 0 reported; chi0-only calls rejected."""
import numpy as np
import pytest

import oracle
from synthetic import eps_occ, eps_unocc, z_block

from test_gpu_fp64 import _dev, rel_fro

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

EDGES = 0.06 * 1.05 ** np.arange(0, 80)  # 79 bins over [0.06, 2.8) Ry; Delta reaches 3.8, so some fall outside


@pytest.fixture(scope="module")
def N():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_03477_gb300 import native
    native.load()
    return native


def _blocks(n, shapes, seed=17):
    return [(z_block(seed, 0, k, n, no, nu, 60.0), eps_occ(seed, 0, k, no), eps_unocc(seed, 0, k, nu), no, nu)
            for k, (no, nu) in enumerate(shapes)]


def _gpu_S(N, prec, n, blocks, bins_out=None, edges=EDGES):
    ctx = N.qsgw_spectral_init(n, edges, prec)
    try:
        for zt, eo, eu, no, nu in blocks:
            N.qsgw_spectral_accumulate(ctx, _dev(zt), n, no, nu, _dev(eo), _dev(eu))
        nb = edges.size - 1
        S = torch.empty((nb, n, n), dtype=torch.complex128, device="cuda")
        N.qsgw_spectral_finalize(ctx, S)
        P = None
        if bins_out is not None:
            P = torch.empty((len(bins_out), n, n), dtype=torch.complex128, device="cuda")
            N.qsgw_spectral_real_axis(ctx, S, bins_out, P)
            P = P.cpu().numpy().transpose(0, 2, 1)
        return S.cpu().numpy().transpose(0, 2, 1), P
    finally:
        N.qsgw_chi0_destroy(ctx)


def _p_bound(ref, edges, bins_out, tol):
    """Per-element bound on the real-axis chi0 at the centres of bins_out, propagated from the per-
    element bound tol * sqrt(S_j,II S_j,JJ) on every S_j through out = sum_j K_j S_j - i pi S_i / width,
    plus FP64 rounding of the Hilbert sum (1e-13 of the sum of term magnitudes)."""
    e = np.asarray(edges)
    dg = np.sqrt(np.abs(np.diagonal(ref, axis1=1, axis2=2)))  # [bin, I]
    cs = dg[:, :, None] * dg[:, None, :]                      # Cauchy-Schwarz scale of every S_j
    out = []
    for i in bins_out:
        w = 0.5 * (e[i] + e[i + 1])
        k = np.abs([oracle.hilbert_weight(w, e[j], e[j + 1]) for j in range(ref.shape[0])])
        b = tol * (np.tensordot(k, cs, axes=1) + np.pi / (e[i + 1] - e[i]) * cs[i])
        out.append(b + 1e-13 * np.tensordot(k, np.abs(ref), axes=1) + 1e-300)
    return np.array(out)


def _oracle_S(blocks, edges=EDGES):
    Z = np.concatenate([zt.T for zt, *_ in blocks], axis=1)
    d = np.concatenate([oracle.delta(eo, eu)[0] for _, eo, eu, _, _ in blocks])
    return oracle.hist_spectral(Z, Z, d, edges)


@pytest.mark.parametrize("prec_name,tol", [("QSGW_FP64", 1e-12), ("QSGW_MIXED_F16X3", 1e-6)])
@pytest.mark.parametrize("n,shapes", [(70, [(5, 130), (3, 61)]), (130, [(9, 300)])])
def test_spectral_weights_and_real_axis(N, prec_name, tol, n, shapes):
    blocks = _blocks(n, shapes)
    ref, outside = _oracle_S(blocks)
    assert outside > 0
    bins_out = [5, 33, 60, 78]
    S, P = _gpu_S(N, getattr(N, prec_name), n, blocks, bins_out)
    for j in range(ref.shape[0]):
        nrm = np.linalg.norm(ref[j])
        if nrm == 0.0:
            assert np.all(S[j] == 0), j
            continue
        assert rel_fro(S[j], ref[j]) <= tol, (j, rel_fro(S[j], ref[j]))
        dg = np.sqrt(np.abs(np.diag(ref[j])))
        assert np.all(np.abs(S[j] - ref[j]) <= tol * np.outer(dg, dg) + 1e-300), j
        assert np.array_equal(S[j], S[j].conj().T)
    Pref = oracle.real_axis_chi0(ref, EDGES, bins_out)
    bound = _p_bound(ref, EDGES, bins_out, tol)
    for o in range(len(bins_out)):
        assert np.all(np.abs(P[o] - Pref[o]) <= bound[o]), (o, (np.abs(P[o] - Pref[o]) / bound[o]).max())


def test_spectral_deterministic_and_errors(N):
    n = 64
    blocks = _blocks(n, [(4, 90), (2, 45)])
    a, _ = _gpu_S(N, N.QSGW_MIXED_F16X3, n, blocks)
    b, _ = _gpu_S(N, N.QSGW_MIXED_F16X3, n, blocks)
    assert np.array_equal(a, b)
    ctx = N.qsgw_spectral_init(n, EDGES, N.QSGW_FP64)
    try:
        zt, eo, eu, no, nu = blocks[0]
        with pytest.raises(N.QsgwError) as e:
            N.qsgw_chi0_accumulate(ctx, 0, _dev(zt), n, no, nu, _dev(eo), _dev(eu), [0.0])
        assert e.value.status == N.QSGW_ERR_STATE
        bad = eu.copy()
        bad[3] = eo.max() - 0.01  # Delta <= 0 for that column
        N.qsgw_spectral_accumulate(ctx, _dev(zt), n, no, nu, _dev(eo), _dev(bad))
        S = torch.empty((EDGES.size - 1, n, n), dtype=torch.complex128, device="cuda")
        with pytest.raises(N.QsgwError) as e:
            N.qsgw_spectral_finalize(ctx, S)
        assert e.value.status == N.QSGW_ERR_DOMAIN
    finally:
        N.qsgw_chi0_destroy(ctx)
    with pytest.raises(N.QsgwError) as e:
        N.qsgw_spectral_init(n, EDGES[::-1], N.QSGW_FP64)  # edges must increase
    assert e.value.status == N.QSGW_ERR_ARG


def test_spectral_many_sparse_bins(N):
    """n_pb = 600 over 156 log bins (0.04 * 1.03^j Ry), 3,000 columns: most bins hold one K-block
    (<= 16 columns) or none, so one launch of 32 bins gives every CTA many one-K-block tiles."""
    edges = 0.04 * 1.03 ** np.arange(0, 157)
    blocks = _blocks(600, [(20, 90), (12, 100)], seed=23)
    ref, _ = _oracle_S(blocks, edges)
    assert sum(np.linalg.norm(r) > 0 for r in ref) > 64
    S, _ = _gpu_S(N, N.QSGW_MIXED_F16X3, 600, blocks, edges=edges)
    for j in range(ref.shape[0]):
        nrm = np.linalg.norm(ref[j])
        if nrm == 0.0:
            assert np.all(S[j] == 0), j
            continue
        assert rel_fro(S[j], ref[j]) <= 1e-6, (j, rel_fro(S[j], ref[j]))


STAGE_EDGES = np.array([0.05, 0.6, 1.0, 1.5, 4.0])  # 4 wide bins: thousands of columns per bin and call


@pytest.mark.parametrize("prec_name,tol", [("QSGW_FP64", 1e-12), ("QSGW_MIXED_F16X3", 1e-6)])
def test_spectral_staging_paths(N, prec_name, tol):
    """The per-bin staging (4096 columns) on all its paths, against the oracle. Bin 3 takes 5277
    columns in call 0 (more than its staging: updated at once), 1973 in call 1 (staged), 2787 in
    call 2 (staging full: flushed first), 5170 in call 3 (flushed, then updated at once). A readout
    after call 1 flushes every bin, and accumulation goes on after it."""
    n = 48
    blocks = _blocks(n, [(20, 400), (10, 300), (16, 250), (20, 400)], seed=29)
    nb = STAGE_EDGES.size - 1
    ctx = N.qsgw_spectral_init(n, STAGE_EDGES, getattr(N, prec_name))
    try:
        keep = []
        for i, (zt, eo, eu, no, nu) in enumerate(blocks):
            keep.append((_dev(zt), _dev(eo), _dev(eu)))
            N.qsgw_spectral_accumulate(ctx, keep[-1][0], n, no, nu, keep[-1][1], keep[-1][2])
            if i == 1:
                S = torch.empty((nb, n, n), dtype=torch.complex128, device="cuda")
                N.qsgw_spectral_finalize(ctx, S)
                mid = S.cpu().numpy().transpose(0, 2, 1)
        N.qsgw_spectral_finalize(ctx, S)
        end = S.cpu().numpy().transpose(0, 2, 1)
    finally:
        N.qsgw_chi0_destroy(ctx)
    for got, ref in ((mid, _oracle_S(blocks[:2], STAGE_EDGES)[0]), (end, _oracle_S(blocks, STAGE_EDGES)[0])):
        for j in range(nb):
            assert np.linalg.norm(ref[j]) > 0
            assert rel_fro(got[j], ref[j]) <= tol, (j, rel_fro(got[j], ref[j]))


def test_spectral_reset_drops_staged_columns(N):
    """qsgw_chi0_reset(ctx, j) clears bin j with the columns staged for it: after block 0, a reset
    of bin 2 and block 1, bin 2 holds block 1 alone and the other bins both blocks."""
    n = 48
    blocks = _blocks(n, [(10, 300), (16, 250)], seed=29)
    ctx = N.qsgw_spectral_init(n, STAGE_EDGES, N.QSGW_MIXED_F16X3)
    try:
        keep = []
        for i, (zt, eo, eu, no, nu) in enumerate(blocks):
            keep.append((_dev(zt), _dev(eo), _dev(eu)))
            N.qsgw_spectral_accumulate(ctx, keep[-1][0], n, no, nu, keep[-1][1], keep[-1][2])
            if i == 0:
                N.qsgw_chi0_reset(ctx, 2)
        S = torch.empty((4, n, n), dtype=torch.complex128, device="cuda")
        N.qsgw_spectral_finalize(ctx, S)
        got = S.cpu().numpy().transpose(0, 2, 1)
    finally:
        N.qsgw_chi0_destroy(ctx)
    both, _ = _oracle_S(blocks, STAGE_EDGES)
    second, _ = _oracle_S(blocks[1:], STAGE_EDGES)
    for j in range(4):
        ref = second[j] if j == 2 else both[j]
        assert rel_fro(got[j], ref) <= 1e-6, j


@pytest.mark.parametrize("bins_out", [[40], list(range(3, 75, 6)), list(range(2, 79, 6))])
def test_real_axis_output_groups(N, bins_out):
    """The real-axis kernel takes outputs in groups of 4, 8 or 12 (one output; 12 in one group;
    13 as two groups of 8, the last padded), FP64 against the oracle, ragged n_pb = 70."""
    blocks = _blocks(70, [(5, 130), (3, 61)])
    ref, _ = _oracle_S(blocks)
    S, P = _gpu_S(N, N.QSGW_FP64, 70, blocks, bins_out)
    Pref = oracle.real_axis_chi0(ref, EDGES, bins_out)
    bound = _p_bound(ref, EDGES, bins_out, 1e-12)
    for o in range(len(bins_out)):
        assert np.all(np.abs(P[o] - Pref[o]) <= bound[o]), (o, (np.abs(P[o] - Pref[o]) / bound[o]).max())


def test_realaxis_medium_full_size_sampled(N):
    """The real-axis route at the benchmark's size and launch configuration: n_pb = 1500, 64 k-points
    x 40 x 400 columns (Z drawn on the device, one k-point at a time), 156 log bins 0.04 * 1.03^j
    Ry, mixed precision. S_j of every bin and the real-axis chi0 at four bin centres are checked on
    a 5 x 5 block of sampled rows against the oracle over all 1,024,000 columns."""
    from synthetic import MEDIUM as W
    n, nk, no, nu = 1500, W.n_k, W.n_occ, 400
    edges = 0.04 * 1.03 ** np.arange(0, 157)
    nb = edges.size - 1
    rows = np.array([0, 17, 700, 1250, 1499])
    bins_out = [30, 80, 120, 150]
    ctx = N.qsgw_spectral_init(n, edges, N.QSGW_MIXED_F16X3)
    try:
        Z = torch.empty((no * nu, n), dtype=torch.complex128, device="cuda")
        for k in range(nk):
            N.qsgw_synth_z(W.seed, 0, k, n, no, nu, W.s_div, Z, n)
            N.qsgw_spectral_accumulate(ctx, Z, n, no, nu, _dev(eps_occ(W.seed, 0, k, no)), _dev(eps_unocc(W.seed, 0, k, nu)))
            N.qsgw_chi0_sync(ctx)
        del Z
        S = torch.empty((nb, n, n), dtype=torch.complex128, device="cuda")
        N.qsgw_spectral_finalize(ctx, S)
        P = torch.empty((len(bins_out), n, n), dtype=torch.complex128, device="cuda")
        N.qsgw_spectral_real_axis(ctx, S, bins_out, P)
        r = torch.from_numpy(rows).cuda()
        Sb = S[:, r][:, :, r].cpu().numpy().transpose(0, 2, 1)
        Pb = P[:, r][:, :, r].cpu().numpy().transpose(0, 2, 1)
        del S, P
    finally:
        N.qsgw_chi0_destroy(ctx)
    from synthetic import z_rows
    ZR = z_rows(W.seed, 0, rows, nk, no, lambda k: nu, W.s_div)
    d = np.concatenate([oracle.delta(eps_occ(W.seed, 0, k, no), eps_unocc(W.seed, 0, k, nu))[0] for k in range(nk)])
    ref, outside = oracle.hist_spectral(ZR, ZR, d, edges)
    assert outside == 0
    for j in range(nb):
        if np.linalg.norm(ref[j]) == 0.0:
            assert np.all(Sb[j] == 0), j
            continue
        assert rel_fro(Sb[j], ref[j]) <= 1e-6, (j, rel_fro(Sb[j], ref[j]))
        dg = np.sqrt(np.abs(np.diag(ref[j])))
        assert np.all(np.abs(Sb[j] - ref[j]) <= 1e-6 * np.outer(dg, dg) + 1e-300), j
    Pref = oracle.real_axis_chi0(ref, edges, bins_out)
    bound = _p_bound(ref, edges, bins_out, 1e-6)
    for o in range(len(bins_out)):
        assert np.all(np.abs(Pb[o] - Pref[o]) <= bound[o]), (o, (np.abs(Pb[o] - Pref[o]) / bound[o]).max())
