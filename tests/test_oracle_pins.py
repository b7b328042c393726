"""Pins for the FP64 oracle: each check ties it to something other than itself.

* Two-level closed form (tests/golden/two_level.txt), derived from Eq. (polfx), Eq.
  (dielectricfunction) and Eq. (screenedcoulomb).
* The paper's own resolvent form of Eq. (polfx), 1/(w - Delta + i delta) - 1/(w + Delta - i delta),
  evaluated in complex arithmetic at w = i omega with the paper's index convention
  Pi_{mu nu} = sum Z_mu Z_nu^* (brute-force loops over k, n, n').
* Library special cases: a numpy GEMM for Z^H diag(w) Z, numpy.linalg.inv for eps^{-1}.
* Invariants the paper states or implies (Sec. 2): Hermiticity, negative definiteness of
  Pi on the imaginary axis, Pi(w) = Pi(-w), eps >= I, W <= v, W^c negative semidefinite,
  plus the omega -> 0 and omega -> infinity limits and monotone decay in omega.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _two_level_rows():
    rows = []
    with open(os.path.join(GOLDEN, "two_level.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            lhs, rhs = line.split("|")
            zr, zi, d, om, v, s = map(float, lhs.split())
            chi, eps, w = rhs.split()
            rows.append((zr, zi, d, om, v, s, float(chi), float(eps), float(Fraction(w))))
    return rows


@pytest.mark.parametrize("row", _two_level_rows())
def test_two_level_closed_form(row):
    zr, zi, d, om, v, s, chi_x, eps_x, w_x = row
    Z = np.array([[zr + 1j * zi]])
    chi = oracle.chi0_full(Z, np.array([d]), np.array([om]), s)
    assert chi.shape == (1, 1, 1)
    assert abs(chi[0, 0, 0] - chi_x) <= 4e-16 * abs(chi_x)
    eps, W, Wc, info = oracle.eps_w(chi, np.array([v]))
    assert info[0] == 0
    assert abs(eps[0, 0, 0] - eps_x) <= 4e-16 * abs(eps_x)
    assert abs(W[0, 0, 0] - w_x) <= 4e-16 * abs(w_x)
    assert abs(Wc[0, 0, 0] - (w_x - v)) <= 4e-15 * abs(v)


def test_weight_is_the_resolvent_of_eq_polfx():
    """w_l(Delta) equals [1/(w - Delta + i0) - 1/(w + Delta - i0)] at w = i omega (complex arithmetic)."""
    rng = np.random.default_rng(3)
    for _ in range(200):
        d = rng.uniform(0.01, 5.0)
        om = rng.uniform(0.0, 30.0)
        w = 1j * om
        bracket = 1.0 / (w - d) - 1.0 / (w + d)
        assert abs(bracket.imag) < 1e-15 * abs(bracket.real)
        assert abs(oracle.weight(d, om) - bracket.real) <= 1e-14 * abs(bracket.real)


def test_brute_force_paper_convention():
    """Sextuple loop over (l, mu, nu, k, n, n') with the resolvent and Pi_{mu nu} = sum Z_mu Z_nu^*.

    The oracle's chi0_IJ carries the conjugate on the row index, so chi0[l, I, J] = Pi[l, J, I]."""
    rng = np.random.default_rng(11)
    N, nk, nocc, nunocc, s = 5, 2, 3, 4, 2.0
    omega = np.array([0.01, 0.3, 2.5])
    eo = np.sort(rng.uniform(-0.8, 0.0, (nk, nocc)), axis=1)
    eu = np.sort(rng.uniform(0.05, 3.0, (nk, nunocc)), axis=1)
    Zk = rng.normal(size=(nk, nocc, nunocc, N)) + 1j * rng.normal(size=(nk, nocc, nunocc, N))
    Pi = np.zeros((omega.size, N, N), dtype=complex)
    for li, om in enumerate(omega):
        w = 1j * om
        for mu in range(N):
            for nu in range(N):
                acc = 0j
                for k in range(nk):
                    for n in range(nocc):
                        for m in range(nunocc):
                            dlt = eu[k, m] - eo[k, n]
                            acc += Zk[k, n, m, mu] * np.conj(Zk[k, n, m, nu]) * (1.0 / (w - dlt) - 1.0 / (w + dlt))
                Pi[li, mu, nu] = s * acc
    # oracle input: rows I, columns r = (k, n, m) with m fastest
    Zrows = Zk.reshape(nk * nocc * nunocc, N).T
    d = np.concatenate([oracle.delta(eo[k], eu[k])[0] for k in range(nk)])
    chi = oracle.chi0_full(Zrows, d, omega, s)
    np.testing.assert_allclose(chi, Pi.transpose(0, 2, 1), rtol=1e-13, atol=1e-13 * np.abs(Pi).max())


def test_library_gemm_special_case(tiny_oracle):
    """chi0(l) = s * Z^H diag(w_l) Z with Z[r, I] = z_{I,r}, by numpy matmul."""
    t = tiny_oracle
    Zr = t["Z"].T  # (K, N)
    for l, om in enumerate(t["omega"]):
        w = -2.0 * t["delta"] / (t["delta"] ** 2 + om ** 2)
        ref = t["spin"] * (Zr.conj().T @ (w[:, None] * Zr))
        err = np.abs(t["chi"][l] - ref).max() / np.abs(ref).max()
        assert err < 1e-13, (l, err)


def test_hermitian_exact_and_negative_definite(tiny_oracle):
    chi = tiny_oracle["chi"]
    for l in range(chi.shape[0]):
        assert np.array_equal(chi[l], chi[l].conj().T)  # full matrix computed, no mirroring
        ev = np.linalg.eigvalsh(chi[l])
        assert ev.max() < -1e-8 * np.abs(ev).max()  # negative definite (K >> N)


def test_even_in_omega():
    """Pi(w) = Pi(-w) (Sec. 2): the imaginary-axis weights depend on omega^2 only."""
    rng = np.random.default_rng(5)
    Z = rng.normal(size=(6, 40)) + 1j * rng.normal(size=(6, 40))
    d = rng.uniform(0.05, 3.0, 40)
    om = np.array([0.01, 0.7, 4.0])
    assert np.array_equal(oracle.chi0_full(Z, d, om, 2.0), oracle.chi0_full(Z, d, -om, 2.0))


def test_monotone_decay_in_omega(tiny_oracle):
    """-chi0(i omega_l) - (-chi0(i omega_{l+1})) is PSD, hence |chi_II| strictly decreases with l."""
    chi = tiny_oracle["chi"]
    for l in range(chi.shape[0] - 1):
        diff = chi[l + 1] - chi[l]
        ev = np.linalg.eigvalsh(diff)
        assert ev.min() > -1e-12 * np.abs(chi[l]).max()
        assert np.all(np.abs(np.diag(chi[l + 1])) < np.abs(np.diag(chi[l])))


def test_small_and_large_omega_limits(tiny_oracle):
    t = tiny_oracle
    Z, d, s = t["Z"], t["delta"], t["spin"]
    Zr = Z.T
    chi0 = oracle.chi0_full(Z, d, np.array([1e-9]), s)[0]
    ref0 = -2.0 * s * (Zr.conj().T @ ((1.0 / d)[:, None] * Zr))
    assert np.abs(chi0 - ref0).max() < 1e-12 * np.abs(ref0).max()
    big = 1e4
    chib = oracle.chi0_full(Z, d, np.array([big]), s)[0]
    refb = -(2.0 * s / big ** 2) * (Zr.conj().T @ (d[:, None] * Zr))
    assert np.abs(chib - refb).max() < 1e-6 * np.abs(refb).max()  # next term is O(Delta^2 / omega^2)


def test_eps_w_invariants(tiny_oracle):
    t = tiny_oracle
    v = t["v"]
    D = np.sqrt(v)
    assert np.all(t["info"] == 0)
    for l in range(t["chi"].shape[0]):
        eps, W, Wc = t["eps"][l], t["W"][l], t["Wc"][l]
        # eps = I - D chi D, eps >= I
        np.testing.assert_allclose(eps, np.eye(v.size) - D[:, None] * t["chi"][l] * D[None, :], rtol=0, atol=0)
        assert np.linalg.eigvalsh(eps - np.eye(v.size)).min() > -1e-9 * np.abs(eps).max()
        # eps * (D^-1 W D^-1) = I
        einv = W / (D[:, None] * D[None, :])
        res = np.abs(eps @ einv - np.eye(v.size)).max()
        assert res < 1e-11, res
        # library special case for the inverse
        ref = np.linalg.inv(eps)
        assert np.abs(einv - ref).max() < 1e-12 * np.abs(ref).max()
        # W PD, W <= v, W^c = W - diag(v) NSD
        assert np.linalg.eigvalsh(W).min() > 0
        assert np.linalg.eigvalsh(np.diag(v) - W).min() > -1e-10 * v.max()
        np.testing.assert_allclose(Wc, W - np.diag(v), rtol=0, atol=1e-14 * v.max())
        assert np.linalg.eigvalsh(Wc).max() < 1e-10 * v.max()


def test_cholesky_factor_and_failure():
    rng = np.random.default_rng(7)
    X = rng.normal(size=(9, 9)) + 1j * rng.normal(size=(9, 9))
    A = X @ X.conj().T + 9 * np.eye(9)
    Lf, info = oracle.cholesky(A)
    assert info == 0
    np.testing.assert_allclose(Lf @ Lf.conj().T, A, rtol=0, atol=1e-12 * np.abs(A).max())
    assert np.allclose(np.triu(Lf, 1), 0)
    np.testing.assert_allclose(Lf, np.linalg.cholesky(A), rtol=1e-12, atol=1e-12)
    B = np.diag([1.0, 2.0, -1.0, 4.0]).astype(complex)
    assert oracle.cholesky(B)[1] == 3


def test_delta_rejects_nonpositive():
    d, bad = oracle.delta(np.array([-0.5, 0.1]), np.array([0.05, 0.2, 3.0]))
    np.testing.assert_allclose(d, [0.55, 0.7, 3.5, -0.05, 0.1, 2.9])
    assert bad == 1
