"""Pins for the real-axis route of the oracle, Eqs. (impolf) and (hilbert) (Sec. 2):

* one transition column lands, with weight conj(z_I) z_J, in the bin holding its Delta
  (half-open bins [L, R));
* the Hilbert-transformation weight of a bin with uniform density equals the principal-value
  integral (1/(R-L)) P.V. int_L^R [1/(w-D) - 1/(w+D)] dD computed by scipy's Cauchy quadrature,
  for w left of, inside and right of the bin;
* Kramers-Kronig consistency with the imaginary-axis route: the histogram integrated along the
  imaginary axis, sum_j S_j (1/(R_j-L_j)) int_{L_j}^{R_j} -2D/(D^2+w^2) dD, reproduces chi0(i w)
  of Eq. (polfx) within the rigorous bound sum_r |z_I,r| |z_J,r| max_{D in bin(r)} |w(D) - w(Delta_r)|;
* the real-axis chi0 is the sum of a Hermitian and i times a Hermitian matrix, its
  anti-Hermitian part being -pi S_i/(R_i-L_i).
"""
import numpy as np
import pytest

import oracle

scipy_integrate = pytest.importorskip("scipy.integrate")


def _rand(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_single_column_lands_in_its_bin():
    edges = np.array([0.1, 0.2, 0.3, 0.5])
    rng = np.random.default_rng(1)
    z = _rand(rng, (3, 1))
    for delta, j in [(0.15, 0), (0.2, 1), (0.49, 2), (0.05, None), (0.5, None)]:
        S, outside = oracle.hist_spectral(z, z, np.array([delta]), edges)
        want = np.zeros_like(S)
        if j is not None:
            want[j] = np.outer(z[:, 0].conj(), z[:, 0])
        assert np.allclose(S, want, rtol=1e-15, atol=1e-15) and outside == (j is None)
        others = [b for b in range(3) if b != j]
        assert np.all(S[others] == 0)


@pytest.mark.parametrize("w", [0.05, 0.41, 0.45, 0.49, 0.8, 2.0])
def test_hilbert_weight_is_the_principal_value_integral(w):
    lo, hi = 0.4, 0.5
    pv, _ = scipy_integrate.quad(lambda D: 1.0, lo, hi, weight="cauchy", wvar=w) if lo < w < hi else \
        scipy_integrate.quad(lambda D: 1.0 / (D - w), lo, hi)
    reg, _ = scipy_integrate.quad(lambda D: 1.0 / (w + D), lo, hi)
    want = (-pv - reg) / (hi - lo)  # 1/(w-D) = -1/(D-w)
    assert abs(oracle.hilbert_weight(w, lo, hi) - want) <= 1e-10 * max(1.0, abs(want))


def test_kramers_kronig_consistency_with_the_imaginary_axis():
    rng = np.random.default_rng(3)
    n, K = 6, 400
    Z = _rand(rng, (n, K))
    delta = rng.uniform(0.05, 3.0, K)
    edges = 0.04 * 1.01 ** np.arange(0, int(np.log(3.2 / 0.04) / np.log(1.01)) + 2)
    S, outside = oracle.hist_spectral(Z, Z, delta, edges)
    assert outside == 0
    lo, hi = edges[:-1], edges[1:]
    for om in [0.01, 0.3, 2.0]:
        direct = oracle.chi0_full(Z, delta, np.array([om]), 1.0)[0]
        binw = -np.log((hi ** 2 + om ** 2) / (lo ** 2 + om ** 2)) / (hi - lo)  # bin average of -2D/(D^2+w^2)
        from_hist = np.tensordot(binw, S, axes=1)
        # rigorous bound: |w(Delta_r) - bin average| <= max over the bin of |w(D) - w(Delta_r)|
        j = np.searchsorted(edges, delta, side="right") - 1
        grid = np.linspace(0.0, 1.0, 65)
        D = lo[j][:, None] + (hi[j] - lo[j])[:, None] * grid[None, :]
        wfun = lambda x: -2.0 * x / (x * x + om * om)
        dev = np.abs(wfun(D) - wfun(delta)[:, None]).max(axis=1) * 1.001  # sampled max, small margin
        bound = (np.abs(Z) * dev) @ np.abs(Z).T
        assert np.all(np.abs(from_hist - direct) <= bound + 1e-14), om
        assert np.abs(from_hist - direct).max() < 1e-2 * np.abs(direct).max()


def test_real_axis_chi0_parts():
    rng = np.random.default_rng(4)
    n, K = 5, 200
    Z = _rand(rng, (n, K))
    delta = rng.uniform(0.1, 1.0, K)
    edges = np.linspace(0.05, 1.05, 41)
    S, _ = oracle.hist_spectral(Z, Z, delta, edges)
    P = oracle.real_axis_chi0(S, edges, [3, 20, 39])
    for k, i in enumerate([3, 20, 39]):
        herm = 0.5 * (P[k] + P[k].conj().T)
        anti = (P[k] - P[k].conj().T) / 2j
        assert np.allclose(anti, -np.pi / (edges[i + 1] - edges[i]) * S[i], rtol=1e-13, atol=1e-13)
        assert np.allclose(herm, sum(oracle.hilbert_weight(0.5 * (edges[i] + edges[i + 1]), edges[j], edges[j + 1]) * S[j]
                                     for j in range(40)), rtol=1e-12, atol=1e-12)
