"""Pins for the seeded input generators (host side)."""
import numpy as np
import pytest

from synthetic import BATCHED, MEDIUM, TINY, coulomb_v, eps_occ, eps_unocc, omega_grid, philox4x32_10, z_block, z_rows
from synthetic.philox import u53

# Known-answer vectors for Philox4x32-10 published with the Random123 library (Salmon et al., SC'11):
# (counter c0..c3, key k0 k1) -> output words.
KAT = [
    ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
    ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
    ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
     (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
]


@pytest.mark.parametrize("ctr,key,out", KAT)
def test_philox_known_answers(ctr, key, out):
    got = philox4x32_10(*ctr, *key)
    assert tuple(int(x) for x in got) == out


def test_u53_range():
    assert u53(0, 0) == 0.0
    assert u53(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53


def test_omega_grid():
    om = omega_grid(12)
    assert om[0] == pytest.approx(0.01)
    assert om[1] == pytest.approx(0.04 * 0.8 + 0.01)
    assert np.all(np.diff(om) > 0)


def test_z_moments_and_row_scale():
    zt = z_block(1, 0, 3, 64, 8, 32, 16.0)  # (K, N)
    assert zt.shape == (256, 64) and zt.dtype == np.complex128
    s = 1.0 / (1.0 + np.arange(64) / 16.0)
    u = zt / s[None, :]
    assert abs(u.real.mean()) < 0.02 and abs(u.imag.mean()) < 0.02
    assert u.real.var() == pytest.approx(0.5, rel=0.05)
    assert u.imag.var() == pytest.approx(0.5, rel=0.05)
    # rows helper gives the same numbers
    rows = z_rows(1, 0, [0, 5, 63], 4, 8, lambda k: 32, 16.0, k_begin=3)
    np.testing.assert_array_equal(rows[:, :256], zt[:, [0, 5, 63]].T)


def test_eps_ranges_sorted():
    eo = eps_occ(1, 0, 2, 40)
    eu = eps_unocc(1, 0, 2, 400)
    assert np.all(np.diff(eo) >= 0) and np.all(np.diff(eu) >= 0)
    assert eo.min() >= -0.8 and eo.max() <= 0.0
    assert eu.min() >= 0.05 and eu.max() <= 3.0
    assert eu.min() - eo.max() >= 0.05


def test_coulomb_v():
    v = coulomb_v(1, 0, 1500)
    g = np.sqrt(4 * np.pi / v)
    assert g.min() >= 0.3 and g.max() <= 6.0


def test_workload_shapes():
    assert TINY.n_cols(0) == 2048 and MEDIUM.n_cols(0) == 1_024_000
    assert MEDIUM.flops() == pytest.approx(1.107e14, rel=1e-3)
    npb = [BATCHED.n_pb(q) for q in range(24)]
    assert min(npb) >= 900 and max(npb) <= 2200 and len(set(npb)) > 10
    nu = [BATCHED.n_unocc(q, k) for q in range(3) for k in range(32)]
    assert min(nu) >= 250 and max(nu) <= 600
