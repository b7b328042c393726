"""Pins for the imaginary-axis correlation self-energy of the oracle, Eq. (sigci) (Sec. 2).

Integration weights w_i(dE) (the reading: dE/(dE^2+w^2) integrated exactly, W^c constant below
the first mesh point, linear between mesh points, decaying as 1/w^2 beyond the last):
* they integrate that piecewise model of X exactly: scipy quadrature of the continuous integral;
* odd in dE, zero at dE = 0;
* a plasmon-pole X(w) = 1/(1 + w^2/Wp^2), whose integral has the closed form
  sign(dE) Wp / (2 (Wp + |dE|)), is reproduced on a fine mesh, with second-order convergence;
* for |dE| far above the mesh they reduce to (1/(pi dE)) times the integral of each hat function.

I^c itself:
* W^c = c_i * identity with one band reduces to a row-scaled Gram matrix (numpy matmul);
* degenerate targets above every band and W^c negative semidefinite give a Hermitian positive
  semidefinite I^c;
* the plasmon-pole W^c = -A f(w) P reproduces sum_n' A g(dE) conj(Z) P Z^T;
* linear in W^c and additive over k-points.
"""
import numpy as np
import pytest

import oracle

integrate = pytest.importorskip("scipy.integrate")

MESH = 0.04 * (1.8 ** np.arange(12) - 1.0) + 0.01  # the chi0 frequency mesh (Ry)


def _model_integral(dE, omega, X):
    """(1/pi) int_0^inf dE/(dE^2+w^2) X(w) dw for X piecewise linear on the mesh, X_0 below it and
    X_{L-1} (omega_{L-1}/w)^2 above it, by adaptive quadrature."""
    k = lambda w: dE / (dE * dE + w * w)
    q = lambda f, a, b: integrate.quad(f, a, b, limit=400, epsabs=0.0, epsrel=1e-13)[0]
    tot = q(lambda w: k(w) * X[0], 0.0, omega[0])
    for i in range(len(omega) - 1):
        a, b = omega[i], omega[i + 1]
        tot += q(lambda w: k(w) * (X[i] * (b - w) + X[i + 1] * (w - a)) / (b - a), a, b)
    W = omega[-1]
    tot += integrate.quad(lambda w: k(w) * X[-1] * (W / w) ** 2, W, np.inf, limit=400, epsabs=0.0, epsrel=1e-13)[0]
    return tot / np.pi


@pytest.mark.parametrize("dE", [0.003, 0.05, 0.3, 2.5, -0.3, -0.003, 40.0])
def test_weights_integrate_the_piecewise_model(dE):
    rng = np.random.default_rng(5)
    for mesh in (MESH, np.array([0.2, 0.5, 0.55, 3.0])):
        X = rng.uniform(-1.0, 1.0, mesh.size)
        got = oracle.sigc_weights(dE, mesh) @ X
        ref = _model_integral(dE, mesh, X)
        assert abs(got - ref) <= 1e-11 * max(1.0, abs(ref)), (dE, got, ref)


def test_weights_odd_and_zero_at_zero():
    for dE in (1e-6, 0.01, 0.7, 9.0):
        assert np.allclose(oracle.sigc_weights(-dE, MESH), -oracle.sigc_weights(dE, MESH), rtol=1e-15, atol=0)
        assert np.all(oracle.sigc_weights(dE, MESH) > 0)
    assert np.all(oracle.sigc_weights(0.0, MESH) == 0.0)


@pytest.mark.parametrize("dE", [0.02, 0.4, -1.5])
def test_plasmon_pole_closed_form_and_convergence(dE):
    Wp = 1.0
    exact = np.sign(dE) * Wp / (2.0 * (Wp + abs(dE)))
    errs = []
    for n in (200, 400, 800):
        mesh = np.geomspace(1e-4, 1e4, n)
        X = 1.0 / (1.0 + (mesh / Wp) ** 2)
        errs.append(abs(oracle.sigc_weights(dE, mesh) @ X - exact))
    assert errs[-1] <= 1e-4 * abs(exact)
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5  # second order in the mesh spacing


def test_large_dE_limit_is_hat_function_integrals():
    dE = 1e7
    h = np.diff(MESH)
    hat = np.empty(MESH.size)
    hat[0] = MESH[0] + h[0] / 2
    hat[1:-1] = (h[:-1] + h[1:]) / 2
    hat[-1] = h[-1] / 2 + MESH[-1]  # the 1/w^2 tail integrates to omega_{L-1}
    assert np.allclose(oracle.sigc_weights(dE, MESH) * np.pi * dE, hat, rtol=1e-5, atol=0)


def _rand(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_scalar_wc_one_band_is_a_row_scaled_gram_matrix():
    rng = np.random.default_rng(7)
    n_qp, n_pb = 5, 9
    Z = _rand(rng, (n_qp, n_pb))  # one band: row n is Z[n' n, :]
    c = rng.uniform(-2.0, -0.1, MESH.size)
    Wc = c[:, None, None] * np.eye(n_pb)[None]
    e_qp = np.array([-0.3, 0.0, 0.1, 0.45, 0.2])
    e_band = np.array([0.1])  # one target degenerate with the band: dE = 0 there
    got = oracle.sigc([Z], e_qp, [e_band], MESH, [Wc])
    s = np.array([oracle.sigc_weights(e - e_band[0], MESH) @ c for e in e_qp])
    ref = -s[:, None] * (Z.conj() @ Z.T)
    assert np.allclose(got, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())
    assert np.all(got[2] == 0)


def _nsd_wc(rng, n_pb, L, scale=1.0):
    B = _rand(rng, (L, n_pb, n_pb)) * scale
    W = -np.einsum("lij,lkj->lik", B, B.conj()) / n_pb
    return 0.5 * (W + W.conj().transpose(0, 2, 1))


def test_degenerate_targets_give_hermitian_psd():
    rng = np.random.default_rng(11)
    n_qp, n_pb, bands = 4, 7, [3, 2]
    Zc = [_rand(rng, (nb * n_qp, n_pb)) for nb in bands]
    e_band = [rng.uniform(-0.8, 0.0, nb) for nb in bands]
    Wc = [_nsd_wc(rng, n_pb, MESH.size) for _ in bands]
    got = oracle.sigc(Zc, np.full(n_qp, 0.2), e_band, MESH, Wc)
    assert np.abs(got - got.conj().T).max() <= 1e-13 * np.abs(got).max()
    ev = np.linalg.eigvalsh(0.5 * (got + got.conj().T))
    assert ev.min() >= -1e-12 * ev.max() and ev.max() > 0


def test_plasmon_pole_end_to_end():
    rng = np.random.default_rng(13)
    n_qp, n_pb, nb = 4, 6, 3
    Wp, A = 0.8, 1.7
    mesh = np.geomspace(1e-4, 1e4, 800)
    B = _rand(rng, (n_pb, n_pb))
    P = B @ B.conj().T / n_pb
    Wc = -A * (1.0 / (1.0 + (mesh / Wp) ** 2))[:, None, None] * P[None]
    Z = _rand(rng, (nb * n_qp, n_pb))
    e_qp = np.array([-0.2, 0.05, 0.3, 0.9])
    e_band = np.array([-0.5, 0.1, 1.4])
    got = oracle.sigc([Z], e_qp, [e_band], mesh, [Wc])
    ref = np.zeros((n_qp, n_qp), dtype=complex)
    for b in range(nb):
        Zb = Z[b * n_qp:(b + 1) * n_qp]
        dE = e_qp - e_band[b]
        g = np.sign(dE) * Wp / (2.0 * (Wp + np.abs(dE)))
        ref += A * g[:, None] * (Zb.conj() @ P @ Zb.T)
    assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max()


def test_linear_in_wc_and_additive_over_k():
    rng = np.random.default_rng(17)
    n_qp, n_pb = 3, 5
    bands = [2, 3]
    Zc = [_rand(rng, (nb * n_qp, n_pb)) for nb in bands]
    e_qp = rng.uniform(-0.3, 0.3, n_qp)
    e_band = [rng.uniform(-0.8, 2.0, nb) for nb in bands]
    W1 = [_nsd_wc(rng, n_pb, MESH.size) for _ in bands]
    W2 = [_nsd_wc(rng, n_pb, MESH.size) for _ in bands]
    I1 = oracle.sigc(Zc, e_qp, e_band, MESH, W1)
    I2 = oracle.sigc(Zc, e_qp, e_band, MESH, W2)
    I12 = oracle.sigc(Zc, e_qp, e_band, MESH, [a + 2.0 * b for a, b in zip(W1, W2)])
    assert np.allclose(I12, I1 + 2.0 * I2, rtol=1e-12, atol=1e-13 * np.abs(I12).max())
    per_k = sum(oracle.sigc([Zc[k]], e_qp, [e_band[k]], MESH, [W1[k]]) for k in range(2))
    assert np.allclose(I1, per_k, rtol=1e-13, atol=1e-14 * np.abs(I1).max())
