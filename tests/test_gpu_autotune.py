"""The tile-plan autotuner of the batched mixed path (uneven q-points in one persistent launch):

* every plan the tuner may pick (the three widest tile widths, with and without the tail cut) gives
  chi0 within the mixed-precision bars against the FP64 oracle, for 12 and 16 frequencies;
* qsgw_chi0_autotune times the candidates on scratch accumulators: the context's chi0 is the same
  whether or not the tuner ran between two accumulate calls, and the chosen plan is a candidate;
* the choice is written to the plan file and read back by a new context; bad plans are refused."""
import numpy as np
import pytest

import oracle
from synthetic import eps_occ, eps_unocc, omega_grid, z_block

from test_gpu_fp64 import _dev, rel_fro

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SHAPES = [(70, 5, 13), (130, 7, 40), (200, 9, 61), (97, 3, 300)]  # (n_pb, n_occ, n_unocc) per q


@pytest.fixture(scope="module")
def N():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_03477_gb300 import native
    native.load()
    return native


def _inputs(q, k, n_pb, n_occ, n_unocc):
    return z_block(5, q, k, n_pb, n_occ, n_unocc, 60.0), eps_occ(5, q, k, n_occ), eps_unocc(5, q, k, n_unocc)


def _blocks(k):
    out = []
    for q, (n, no, nu) in enumerate(SHAPES):
        zt, eo, eu = _inputs(q, k, n, no, nu)
        out.append((q, _dev(zt), n, no, nu, _dev(eo), _dev(eu)))
    return out


def _oracle(L, n_k=2):
    refs = []
    for q, (n, no, nu) in enumerate(SHAPES):
        Zs, ds = [], []
        for k in range(n_k):
            zt, eo, eu = _inputs(q, k, n, no, nu)
            Zs.append(zt.T)
            ds.append(oracle.delta(eo, eu)[0])
        refs.append(oracle.chi0_full(np.concatenate(Zs, 1), np.concatenate(ds), omega_grid(L), 2.0))
    return refs


def _readout(N, ctx, L):
    out = []
    for q, (n, _, _) in enumerate(SHAPES):
        chi = torch.empty((L, n, n), dtype=torch.complex128, device="cuda")
        N.qsgw_chi0_finalize(ctx, q, chi)
        out.append(chi.cpu().numpy().transpose(0, 2, 1))
    return out


def _check(got, refs, L):
    for g, r in zip(got, refs):
        for l in range(L):
            assert rel_fro(g[l], r[l]) <= 1e-6
            d = np.sqrt(np.abs(np.diag(r[l])))
            assert np.all(np.abs(g[l] - r[l]) <= 1e-6 * np.outer(d, d))


@pytest.mark.parametrize("L", [12, 16])
def test_every_candidate_plan_passes_parity(N, L):
    refs = _oracle(L)
    blocks = [_blocks(0), _blocks(1)]
    cands = N.qsgw_tile_plan_candidates(L)
    assert len(cands) == 6
    for plan in cands:
        ctx = N.qsgw_chi0_init([s[0] for s in SHAPES], omega_grid(L), 2.0, N.QSGW_MIXED_F16X3)
        try:
            N.qsgw_chi0_set_tile_plan(ctx, plan)
            for k in range(2):
                N.qsgw_chi0_accumulate_batch(ctx, blocks[k])
            got = _readout(N, ctx, L)
        finally:
            N.qsgw_chi0_destroy(ctx)
        _check(got, refs, L)


def test_autotune_leaves_chi0_untouched_and_persists(N, tmp_path, monkeypatch):
    L = 12
    cache = tmp_path / "plans.txt"
    monkeypatch.setenv("QSGW_TUNE_CACHE", str(cache))
    refs = _oracle(L)
    blocks = [_blocks(0), _blocks(1)]
    ctx = N.qsgw_chi0_init([s[0] for s in SHAPES], omega_grid(L), 2.0, N.QSGW_MIXED_F16X3)
    try:
        N.qsgw_chi0_accumulate_batch(ctx, blocks[0])
        plan, ms = N.qsgw_chi0_autotune(ctx, blocks[1], reps=2)  # between the two accumulate calls
        assert plan in N.qsgw_tile_plan_candidates(L) and ms > 0
        N.qsgw_chi0_accumulate_batch(ctx, blocks[1])
        got = _readout(N, ctx, L)
    finally:
        N.qsgw_chi0_destroy(ctx)
    _check(got, refs, L)
    lines = [x.split() for x in cache.read_text().splitlines()]
    assert lines and lines[-1][0] == "qsgw-plan" and int(lines[-1][1]) == L
    assert (int(lines[-1][4]), int(lines[-1][5])) == plan
    # a new context reads the plan back (a malformed line is skipped) and uses it
    with open(cache, "a") as f:
        f.write("not a plan line\n")
    ctx = N.qsgw_chi0_init([s[0] for s in SHAPES], omega_grid(L), 2.0, N.QSGW_MIXED_F16X3)
    try:
        for k in range(2):
            N.qsgw_chi0_accumulate_batch(ctx, blocks[k])
        _check(_readout(N, ctx, L), refs, L)
        with pytest.raises(N.QsgwError) as e:  # 7 * 12 = 84 is not a multiple of 16
            N.qsgw_chi0_set_tile_plan(ctx, (7, 0))
        assert e.value.status == N.QSGW_ERR_ARG
        N.qsgw_chi0_set_tile_plan(ctx, None)
    finally:
        N.qsgw_chi0_destroy(ctx)
    ctx64 = N.qsgw_chi0_init([64], omega_grid(L), 2.0, N.QSGW_FP64)
    try:
        with pytest.raises(N.QsgwError) as e:
            N.qsgw_chi0_set_tile_plan(ctx64, (20, 0))
        assert e.value.status == N.QSGW_ERR_STATE
    finally:
        N.qsgw_chi0_destroy(ctx64)
