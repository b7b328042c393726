"""Batched accumulation over uneven q-points (one persistent launch per batch call) vs the oracle."""
import numpy as np
import pytest

import oracle
from synthetic import BATCHED, eps_occ, eps_unocc, z_block, z_rows
from synthetic.workloads import Workload

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


SHAPES = [(70, 5, 13), (130, 7, 40), (200, 9, 61), (97, 3, 300)]  # (n_pb, n_occ, n_unocc) per q
OMEGA = Workload("b", n_q=1, n_k=1, n_occ=1, n_omega=12, s_div=1.0).omega


def _inputs(q, k, n_pb, n_occ, n_unocc):
    zt = z_block(1, q, k, n_pb, n_occ, n_unocc, 60.0)
    return zt, eps_occ(1, q, k, n_occ), eps_unocc(1, q, k, n_unocc)


def _run(N, prec, batched, n_k=2):
    ctx = N.qsgw_chi0_init([s[0] for s in SHAPES], OMEGA, 2.0, prec)
    dev = {}
    for q, (n, no, nu) in enumerate(SHAPES):
        for k in range(n_k):
            zt, eo, eu = _inputs(q, k, n, no, nu)
            dev[q, k] = (_dev(zt), _dev(eo), _dev(eu))
    try:
        for k in range(n_k):
            if batched:
                N.qsgw_chi0_accumulate_batch(ctx, [(q, dev[q, k][0], n, no, nu, dev[q, k][1], dev[q, k][2])
                                                   for q, (n, no, nu) in enumerate(SHAPES)])
            else:
                for q, (n, no, nu) in enumerate(SHAPES):
                    N.qsgw_chi0_accumulate(ctx, q, dev[q, k][0], n, no, nu, dev[q, k][1], dev[q, k][2], OMEGA)
        out = []
        for q, (n, _, _) in enumerate(SHAPES):
            chi = torch.empty((12, n, n), dtype=torch.complex128, device="cuda")
            N.qsgw_chi0_finalize(ctx, q, chi)
            out.append(chi.cpu().numpy().transpose(0, 2, 1))
    finally:
        N.qsgw_chi0_destroy(ctx)
    return out


def _oracle(n_k=2):
    refs = []
    for q, (n, no, nu) in enumerate(SHAPES):
        Zs, ds = [], []
        for k in range(n_k):
            zt, eo, eu = _inputs(q, k, n, no, nu)
            Zs.append(zt.T)
            ds.append(oracle.delta(eo, eu)[0])
        refs.append(oracle.chi0_full(np.concatenate(Zs, 1), np.concatenate(ds), OMEGA, 2.0))
    return refs


def test_batch_mixed_uneven_q(N):
    got = _run(N, N.QSGW_MIXED_F16X3, batched=True)
    seq = _run(N, N.QSGW_MIXED_F16X3, batched=False)
    for g, s_, r in zip(got, seq, _oracle()):
        for l in range(12):
            assert rel_fro(g[l], r[l]) <= 1e-6
            d = np.sqrt(np.abs(np.diag(r[l])))
            assert np.all(np.abs(g[l] - r[l]) <= 1e-6 * np.outer(d, d))
        # same digits and products; only the split of chunks between CTAs (and so the order of
        # double-float additions) differs from the one-q-at-a-time path
        assert rel_fro(g, s_) <= 1e-12


def test_batch_fp64_equals_sequential(N):
    got = _run(N, N.QSGW_FP64, batched=True)
    seq = _run(N, N.QSGW_FP64, batched=False)
    for g, s_, r in zip(got, seq, _oracle()):
        assert np.array_equal(g, s_)
        assert rel_fro(g, r) <= 1e-12


def test_batch_argument_errors(N):
    ctx = N.qsgw_chi0_init([64, 64], OMEGA, 2.0, N.QSGW_MIXED_F16X3)
    try:
        zt, eo, eu = _inputs(0, 0, 64, 2, 3)
        Z, EO, EU = _dev(zt), _dev(eo), _dev(eu)
        with pytest.raises(N.QsgwError) as e:  # the same q twice
            N.qsgw_chi0_accumulate_batch(ctx, [(0, Z, 64, 2, 3, EO, EU), (0, Z, 64, 2, 3, EO, EU)])
        assert e.value.status == N.QSGW_ERR_ARG
        with pytest.raises(N.QsgwError) as e:  # host arrays are not accepted in a batch
            N.qsgw_chi0_accumulate_batch(ctx, [(1, zt, 64, 2, 3, eo, eu)])
        assert e.value.status == N.QSGW_ERR_ARG
        with pytest.raises(N.QsgwError) as e:  # q out of range
            N.qsgw_chi0_accumulate_batch(ctx, [(2, Z, 64, 2, 3, EO, EU)])
        assert e.value.status == N.QSGW_ERR_ARG
    finally:
        N.qsgw_chi0_destroy(ctx)


def test_batch_graph_capture_replay(N):
    """After a warm-up call, the batched sequence is only kernel launches: capture it in a CUDA graph
    on the context's stream and replay it; the result equals the directly launched sequence."""
    ref = _run(N, N.QSGW_MIXED_F16X3, batched=True)
    stream = torch.cuda.Stream()
    ctx = N.qsgw_chi0_init([s[0] for s in SHAPES], OMEGA, 2.0, N.QSGW_MIXED_F16X3, stream=stream)
    try:
        dev = {}
        for q, (n, no, nu) in enumerate(SHAPES):
            for k in range(2):
                zt, eo, eu = _inputs(q, k, n, no, nu)
                dev[q, k] = (_dev(zt), _dev(eo), _dev(eu))
        torch.cuda.synchronize()

        def work():
            for k in range(2):
                N.qsgw_chi0_accumulate_batch(ctx, [(q, dev[q, k][0], n, no, nu, dev[q, k][1], dev[q, k][2])
                                                   for q, (n, no, nu) in enumerate(SHAPES)])
        work()  # warm-up: allocations happen here
        N.qsgw_chi0_sync(ctx)
        for q in range(len(SHAPES)):
            N.qsgw_chi0_reset(ctx, q)
        N.qsgw_chi0_sync(ctx)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream, capture_error_mode="relaxed"):
            work()
        g.replay()
        torch.cuda.synchronize()
        for q, (n, _, _) in enumerate(SHAPES):
            chi = torch.empty((12, n, n), dtype=torch.complex128, device="cuda")
            N.qsgw_chi0_finalize(ctx, q, chi)
            got = chi.cpu().numpy().transpose(0, 2, 1)
            assert np.array_equal(got, ref[q])
    finally:
        N.qsgw_chi0_destroy(ctx)


def test_batched_workload_full_size_sampled(N):
    """The batched workload at full size: 24 q-points, n_pb ~ U{900..2200}, 32 k-points with
    n_unocc ~ U{250..600} per (q, k), 12 frequencies; one batch call (24 blocks) per k-point.
    Oracle on the diagonal and a 4x4 block of sampled rows of every q-point."""
    wl = BATCHED
    npb = [wl.n_pb(q) for q in range(wl.n_q)]
    ctx = N.qsgw_chi0_init(npb, wl.omega, wl.spin, N.QSGW_MIXED_F16X3)
    got = []
    try:
        eo_d = {}
        for k in range(wl.n_k):
            blocks, keep = [], []
            for q in range(wl.n_q):
                nu = wl.n_unocc(q, k)
                Z = torch.empty((wl.n_occ * nu, npb[q]), dtype=torch.complex128, device="cuda")
                N.qsgw_synth_z(wl.seed, q, k, npb[q], wl.n_occ, nu, wl.s_div, Z, npb[q])
                EO = _dev(eps_occ(wl.seed, q, k, wl.n_occ))
                EU = _dev(eps_unocc(wl.seed, q, k, nu))
                keep.append((Z, EO, EU))
                blocks.append((q, Z, npb[q], wl.n_occ, nu, EO, EU))
            N.qsgw_chi0_accumulate_batch(ctx, blocks)
            N.qsgw_chi0_sync(ctx)
            del keep
        rng = np.random.default_rng(9)
        for q in range(wl.n_q):
            rows = np.unique(np.concatenate([[0, npb[q] - 1], rng.integers(0, npb[q], 2)]))
            chi = torch.empty((wl.n_omega, npb[q], npb[q]), dtype=torch.complex128, device="cuda")
            N.qsgw_chi0_finalize(ctx, q, chi)
            got.append((rows, chi.cpu().numpy().transpose(0, 2, 1)[:, rows][:, :, rows]))
            del chi
    finally:
        N.qsgw_chi0_destroy(ctx)
    for q in range(wl.n_q):
        rows, sub = got[q]
        ZS = z_rows(wl.seed, q, rows, wl.n_k, wl.n_occ, lambda k: wl.n_unocc(q, k), wl.s_div)
        d = np.concatenate([oracle.delta(eps_occ(wl.seed, q, k, wl.n_occ), eps_unocc(wl.seed, q, k, wl.n_unocc(q, k)))[0]
                            for k in range(wl.n_k)])
        ref = oracle.chi0_rows(ZS, ZS, d, wl.omega, wl.spin)
        for l in range(wl.n_omega):
            dg = np.sqrt(np.abs(np.diag(ref[l])))
            assert np.all(np.abs(sub[l] - ref[l]) <= 1e-6 * np.outer(dg, dg)), (q, l)
            assert rel_fro(sub[l], ref[l]) <= 1e-6


def test_batch_many_short_items(N):
    """Many work items of one or two K-blocks (K <= 32 columns) per CTA: 16 q-points of
    n_pb = 600 at 12 frequencies, about 2,500 tiles per launch, 16 per CTA. The producer
    publishes items ahead of the consumers by up to NS + 1; this holds only while the item ring is
    longer than that, which tiles of many K-blocks never tested."""
    shapes = [(600, 1, nu) for nu in (13, 16, 5, 9, 1, 16, 32, 11, 3, 16, 7, 29, 2, 16, 16, 8)]
    ctx = N.qsgw_chi0_init([s[0] for s in shapes], OMEGA, 2.0, N.QSGW_MIXED_F16X3)
    got = []
    try:
        for k in range(2):
            keep = [(_dev(z_block(3, q, k, n, no, nu, 60.0)), _dev(eps_occ(3, q, k, no)), _dev(eps_unocc(3, q, k, nu)))
                    for q, (n, no, nu) in enumerate(shapes)]
            N.qsgw_chi0_accumulate_batch(ctx, [(q, keep[q][0], n, no, nu, keep[q][1], keep[q][2])
                                               for q, (n, no, nu) in enumerate(shapes)])
            N.qsgw_chi0_sync(ctx)
        for q, (n, _, _) in enumerate(shapes):
            chi = torch.empty((12, n, n), dtype=torch.complex128, device="cuda")
            N.qsgw_chi0_finalize(ctx, q, chi)
            got.append(chi.cpu().numpy().transpose(0, 2, 1))
    finally:
        N.qsgw_chi0_destroy(ctx)
    for q, (n, no, nu) in enumerate(shapes):
        Z = np.concatenate([z_block(3, q, k, n, no, nu, 60.0).T for k in range(2)], 1)
        d = np.concatenate([oracle.delta(eps_occ(3, q, k, no), eps_unocc(3, q, k, nu))[0] for k in range(2)])
        ref = oracle.chi0_full(Z, d, OMEGA, 2.0)
        for l in range(12):
            assert rel_fro(got[q][l], ref[l]) <= 1e-6, (q, l)
            dg = np.sqrt(np.abs(np.diag(ref[l])))
            assert np.all(np.abs(got[q][l] - ref[l]) <= 1e-6 * np.outer(dg, dg)), (q, l)
