"""The decomposition the GPU path uses for I^c, Eq. (sigci), checked on the CPU against the oracle.

Both contractions of I^c run on the Hermitian-update kernels as the off-diagonal block of a
stacked operand. This test builds the two stacked operands in numpy with the layout the kernels
use (rows [0, M) scaled band rows, zero rows up to the next multiple of 128, then the second row
set; columns (i, mu) and (band, nu)), takes the off-diagonal blocks of conj(S) S^T, and compares
the result with the oracle. Band batches, the zero padding and the conjugations are what it pins.
"""
import numpy as np

import oracle

ALIGN = 128
MESH = 0.04 * (1.8 ** np.arange(5) - 1.0) + 0.01


def _rand(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _stacked_sigc(Zcols, e_qp, e_band, Wc, batch_bands):
    """I^c by the two stacked products, band batch by band batch (one k-point)."""
    n_qp, n_pb, L = e_qp.size, Zcols.shape[1], MESH.size
    w = np.array([[oracle.sigc_weights(eq - eb, MESH) for eq in e_qp] for eb in e_band])  # [band, n, i]
    Y3 = -(-n_qp // ALIGN) * ALIGN
    acc3 = np.zeros((n_qp, n_qp), dtype=complex)
    for b0 in range(0, e_band.size, batch_bands):
        nb = min(batch_bands, e_band.size - b0)
        M = nb * n_qp
        Y0 = -(-M // ALIGN) * ALIGN
        Zt = Zcols[b0 * n_qp:(b0 + nb) * n_qp]  # rows (band, target), columns mu
        S2 = np.zeros((Y0 + n_pb, L * n_pb), dtype=complex)
        for i in range(L):
            S2[:M, i * n_pb:(i + 1) * n_pb] = w[b0:b0 + nb, :, i].reshape(M, 1) * Zt
            S2[Y0:, i * n_pb:(i + 1) * n_pb] = Wc[i].conj()  # row nu, column mu: conj(W_i[nu, mu])
        D = S2[:M].conj() @ S2[Y0:].T  # block (I < M, J >= Y0) of conj(S2) S2^T
        S3 = np.zeros((Y3 + n_qp, nb * n_pb), dtype=complex)
        for b in range(nb):
            S3[:n_qp, b * n_pb:(b + 1) * n_pb] = D[b * n_qp:(b + 1) * n_qp].conj()
            S3[Y3:, b * n_pb:(b + 1) * n_pb] = Zt[b * n_qp:(b + 1) * n_qp]
        acc3 += S3[:n_qp].conj() @ S3[Y3:].T
    return -acc3


def test_stacked_products_equal_the_oracle():
    rng = np.random.default_rng(3)
    n_qp, n_pb, nbands = 7, 11, 5
    Zcols = _rand(rng, (nbands * n_qp, n_pb))
    e_qp = rng.uniform(-0.3, 0.3, n_qp)
    e_band = rng.uniform(-0.8, 2.5, nbands)
    e_band[1] = e_qp[4]  # dE = 0
    B = _rand(rng, (MESH.size, n_pb, n_pb))
    Wc = -np.einsum("lij,lkj->lik", B, B.conj()) / n_pb
    Wc = 0.5 * (Wc + Wc.conj().transpose(0, 2, 1))
    ref = oracle.sigc([Zcols], e_qp, [e_band], MESH, [Wc])
    for batch in (1, 2, 5):  # several band batches, ragged last batch, one batch
        got = _stacked_sigc(Zcols, e_qp, e_band, Wc, batch)
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max()), batch


def test_stacked_products_over_two_k_points_add():
    rng = np.random.default_rng(4)
    n_qp, n_pb = 3, 6
    parts, Zs, eb, Ws = [], [], [], []
    e_qp = rng.uniform(-0.3, 0.3, n_qp)
    for nb in (2, 4):
        Z = _rand(rng, (nb * n_qp, n_pb))
        e = rng.uniform(-0.8, 2.5, nb)
        B = _rand(rng, (MESH.size, n_pb, n_pb))
        W = -np.einsum("lij,lkj->lik", B, B.conj()) / n_pb
        W = 0.5 * (W + W.conj().transpose(0, 2, 1))
        parts.append(_stacked_sigc(Z, e_qp, e, W, 3))
        Zs.append(Z)
        eb.append(e)
        Ws.append(W)
    ref = oracle.sigc(Zs, e_qp, eb, MESH, Ws)
    assert np.allclose(parts[0] + parts[1], ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
