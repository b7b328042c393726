"""Pins for the real-axis route of the oracle, Eqs. (impolf) and (hilbert) (Sec. 2):

* one transition column lands, with weight conj(z_I) z_J, in the bin holding its Delta
  (half-open bins [L, R));
* the Hilbert-transformation weight of a bin with uniform density equals the principal-value
  integral (1/(R-L)) P.V. int_L^R [1/(w-D) - 1/(w+D)] dD computed by scipy's Cauchy quadrature,
  for w left of, inside and right of the bin;
* Kramers-Kronig consistency with the imaginary-axis route: the histogram integrated along the
  imaginary axis, sum_j S_j (1/(R_j-L_j)) int_{L_j}^{R_j} -2D/(D^2+w^2) dD, reproduces chi0(i w)
  of Eq. (polfx) within the rigorous bound sum_r |z_I,r| |z_J,r| max_{D in bin(r)} |w(D) - w(Delta_r)|;
* the real-axis chi0 at a bin centre equals the bin-averaged retarded resolvent of Eq. (polf01),
  (1/(R_j-L_j)) int_{L_j}^{R_j} [1/(w-D+i eta) - 1/(w+D-i eta)] dD, integrated in closed form with
  complex logarithms at a small eta > 0 and applied to spectral weights binned by numpy.histogram,
  on uneven log bins (this fixes the sign of the i pi term, the bin it comes from, the bin width
  and the centre frequency, independently of the oracle's real-log form);
* at the centres of empty bins below and above the whole spectrum it equals the direct resolvent
  sum sum_r conj(z_I) z_J [1/(w-Delta_r) - 1/(w+Delta_r)] within the exact bound
  sum_r |z_I||z_J| max(|f(L_r)-f(Delta_r)|, |f(R_r)-f(Delta_r)|) (f is monotone in each bin there),
  with no anti-Hermitian part.
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


def _numpy_histogram_S(Z, delta, edges):
    """S[j, I, J] = sum over columns in bin j of conj(Z[I]) Z[J], binned by numpy.histogram (real and
    imaginary parts of the weights separately; numpy closes its last bin, no Delta sits on an edge)."""
    n = Z.shape[0]
    S = np.zeros((edges.size - 1, n, n), dtype=np.complex128)
    for i in range(n):
        for j in range(n):
            w = Z[i].conj() * Z[j]
            S[:, i, j] = (np.histogram(delta, bins=edges, weights=w.real)[0]
                          + 1j * np.histogram(delta, bins=edges, weights=w.imag)[0])
    return S


def _retarded_bin_kernel(w, lo, hi, eta):
    """(1/(hi-lo)) int_lo^hi [1/(w - D + i eta) - 1/(w + D - i eta)] dD by the complex logarithm
    (principal branch): the antiderivatives are -log(w - D + i eta) and -log(w + D - i eta)."""
    res = np.log(w - lo + 1j * eta) - np.log(w - hi + 1j * eta)
    anti = np.log(w + hi - 1j * eta) - np.log(w + lo - 1j * eta)
    return (res - anti) / (hi - lo)


def test_real_axis_chi0_is_the_bin_averaged_retarded_resolvent():
    rng = np.random.default_rng(4)
    n, K = 5, 300
    Z = _rand(rng, (n, K))
    delta = rng.uniform(0.3, 1.0, K)
    edges = 0.05 * 1.08 ** np.arange(0, 55)  # uneven log bins over [0.05, 3.2)
    S, outside = oracle.hist_spectral(Z, Z, delta, edges)
    assert outside == 0
    S_np = _numpy_histogram_S(Z, delta, edges)
    assert np.allclose(S, S_np, rtol=1e-13, atol=1e-13)
    occupied = [j for j in range(S.shape[0]) if np.abs(S_np[j]).max() > 0]
    bins_out = [occupied[0], occupied[len(occupied) // 2], occupied[-1], 2, 50]  # inside and outside the spectrum
    P = oracle.real_axis_chi0(S, edges, bins_out)
    lo, hi = edges[:-1], edges[1:]
    for o, i in enumerate(bins_out):
        w = 0.5 * (edges[i] + edges[i + 1])
        kern = _retarded_bin_kernel(w, lo, hi, 1e-13)
        want = np.tensordot(kern, S_np, axes=1)
        scale = np.tensordot(np.abs(kern), np.abs(S_np), axes=1)
        assert np.all(np.abs(P[o] - want) <= 1e-9 * scale + 1e-13), (i, np.abs(P[o] - want).max())
        # the anti-Hermitian part comes from the bin that holds w alone
        anti = (P[o] - P[o].conj().T) / 2j
        assert np.allclose(anti, -np.pi / (hi[i] - lo[i]) * S_np[i], rtol=1e-12, atol=1e-12)


def test_real_axis_chi0_matches_the_direct_resolvent_sum_off_the_spectrum():
    rng = np.random.default_rng(6)
    n, K = 6, 400
    Z = _rand(rng, (n, K))
    delta = rng.uniform(0.3, 1.0, K)
    edges = 0.05 * 1.02 ** np.arange(0, 208)  # uneven log bins over [0.05, 3.0)
    S, _ = oracle.hist_spectral(Z, Z, delta, edges)
    j_of = np.searchsorted(edges, delta, side="right") - 1
    L_r, R_r = edges[j_of], edges[j_of + 1]
    below = int(np.searchsorted(edges, 0.12)) - 1
    above = int(np.searchsorted(edges, 2.0)) - 1
    assert np.abs(S[below]).max() == 0 and np.abs(S[above]).max() == 0
    P = oracle.real_axis_chi0(S, edges, [below, above])
    absZ = np.abs(Z)
    for o, i in enumerate([below, above]):
        w = 0.5 * (edges[i] + edges[i + 1])
        f = lambda D: 1.0 / (w - D) - 1.0 / (w + D)  # Eq. (polf01) at real w away from every Delta
        direct = (Z.conj() * f(delta)) @ Z.T
        dev = np.maximum(np.abs(f(L_r) - f(delta)), np.abs(f(R_r) - f(delta)))
        bound = (absZ * dev) @ absZ.T
        assert np.all(np.abs(P[o] - direct) <= bound * (1 + 1e-12) + 1e-13), w
        assert bound.max() < 0.1 * np.abs(direct).max()  # tight enough to catch a dropped or flipped term
        assert np.array_equal(P[o], P[o].conj().T)  # empty bin: no anti-Hermitian part
