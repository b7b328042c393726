"""Pins for the exchange self-energy oracle, Eq. (sigx) (Sec. 2):

    Sigma^x_nm(q) = - sum_k sum_{n' occ} sum_mu conj(Z^{(q-k)n', qn}_{k mu}) v_mu(k) Z^{(q-k)n', qm}_{k mu}.

* one transition column: the closed form -v conj(z_n) z_m;
* a single nonzero column (k, n', mu): the weight is v_mu(k) of that k and mu, not of n' or of the
  flat column index (pins the index order);
* constant weights: the library GEMM -c Z^* Z^T (numpy);
* rank-one Z (Z[n, r] = a_n b_r): -(sum_r w_r |b_r|^2) conj(a_n) a_m;
* Hermitian exactly, negative semidefinite for v > 0, additive over k-points.
"""
import numpy as np

import oracle


def _rand(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_sigx_single_column_closed_form():
    rng = np.random.default_rng(1)
    z = _rand(rng, (4, 1))
    S = oracle.sigx(z, [1], 1, np.array([[0.7]]))
    assert np.allclose(S, -0.7 * np.outer(z[:, 0].conj(), z[:, 0]), rtol=1e-15, atol=1e-15)


def test_sigx_weight_attaches_to_k_and_mu():
    n_k, occ, n_pb = 2, [2, 3], 3
    v = np.array([[1.0, 2.0, 3.0], [5.0, 7.0, 11.0]])
    K = n_pb * sum(occ)
    rng = np.random.default_rng(2)
    z = _rand(rng, 3)
    for k, nprime, mu in [(0, 1, 2), (1, 0, 1), (1, 2, 0)]:
        Z = np.zeros((3, K), dtype=np.complex128)
        col = n_pb * sum(occ[:k]) + nprime * n_pb + mu
        Z[:, col] = z
        S = oracle.sigx(Z, occ, n_pb, v)
        assert np.allclose(S, -v[k, mu] * np.outer(z.conj(), z), rtol=1e-14, atol=1e-14), (k, nprime, mu)


def test_sigx_constant_weight_is_a_gemm():
    rng = np.random.default_rng(3)
    occ, n_pb = [3, 2, 4], 5
    Z = _rand(rng, (6, n_pb * sum(occ)))
    S = oracle.sigx(Z, occ, n_pb, np.full((3, n_pb), 1.5))
    assert np.allclose(S, -1.5 * (Z.conj() @ Z.T), rtol=1e-13, atol=1e-13)


def test_sigx_rank_one_closed_form():
    rng = np.random.default_rng(4)
    occ, n_pb = [2, 3], 4
    v = rng.uniform(0.2, 3.0, (2, n_pb))
    a = _rand(rng, 5)
    b = _rand(rng, n_pb * sum(occ))
    w = np.concatenate([np.tile(v[k], occ[k]) for k in range(2)])  # the weight of column (k, n', mu)
    S = oracle.sigx(np.outer(a, b), occ, n_pb, v)
    assert np.allclose(S, -np.sum(w * np.abs(b) ** 2) * np.outer(a.conj(), a), rtol=1e-13, atol=1e-13)


def test_sigx_hermitian_nsd_and_additive_over_k():
    rng = np.random.default_rng(5)
    occ, n_pb, n_qp = [3, 2, 4, 1], 6, 7
    v = rng.uniform(0.1, 4.0, (4, n_pb))
    Z = _rand(rng, (n_qp, n_pb * sum(occ)))
    S = oracle.sigx(Z, occ, n_pb, v)
    assert np.array_equal(S, S.conj().T)
    assert np.linalg.eigvalsh(S).max() <= 1e-13 * np.abs(S).max()
    cut = n_pb * sum(occ[:2])
    S1 = oracle.sigx(Z[:, :cut], occ[:2], n_pb, v[:2])
    S2 = oracle.sigx(Z[:, cut:], occ[2:], n_pb, v[2:])
    assert np.allclose(S1 + S2, S, rtol=1e-13, atol=1e-13)
