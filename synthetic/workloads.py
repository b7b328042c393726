"""Seeded synthetic inputs shaped like the paper's workloads (Table 2: n_pb 982-5231,
n_occ 92-460, n_unocc ~270-1350, n_BZ 16-48, ~11 imaginary frequencies).

The paper's inputs (PMT eigenfunctions of (InAs)n(GaSb)n and Ni2MnGa) are not available,
so every input here is drawn from Philox4x32-10 with a fixed counter layout:

  key  = (seed, (q << 8) | tag)      tags: Z=0, eps_occ=1, eps_unocc=2, |G|=3, shapes=4
  Z    : counter (k, n, m, I) -> Box-Muller on u1 = u53(w0,w1) mapped to (0,1], u2 = u53(w2,w3):
         a = sqrt(-ln u1) cos(2 pi u2), b = sqrt(-ln u1) sin(2 pi u2)  (each N(0, 1/2)),
         z_{I,knm} = (a + i b) * s_I,  s_I = 1 / (1 + I / s_div)
  eps  : counter (k, n, 0, 0) -> U[lo, hi] from u53(w0, w1); sorted ascending per k
  |G_I|: counter (I, 0, 0, 0) -> U[0.3, 6] bohr^-1, v_I = 4 pi / |G_I|^2 (plane-wave form
         of the Coulomb eigenvalues, Sec. 2)
  shapes (batched workload): n_pb(q) from counter (q, 0, 0, 0), n_unocc(q, k) from
         counter (q, k + 1, 0, 0), integer U{a..b} = a + floor(u53 * (b - a + 1))

Column order inside one k-point: r = n * n_unocc + m (unoccupied index fastest), matching
the paper's Z(1:n_pb, n', n) storage. A Z block is returned as a C-ordered (K, N) array
`Zt` with Zt[r, I] = z_{I,r}; its memory is the column-major N x K matrix (I fastest).

This module holds none of the method's arithmetic: it only draws inputs.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

from .philox import philox4x32_10, u53

TAG_Z, TAG_EPS_OCC, TAG_EPS_UNOCC, TAG_G, TAG_SHAPE = 0, 1, 2, 3, 4


def omega_grid(n_omega: int) -> np.ndarray:
    """Imaginary frequencies omega_l = 0.04 * (1.8^l - 1) + 0.01 Ry, l = 0..n_omega-1."""
    l = np.arange(n_omega, dtype=np.float64)
    return 0.04 * (1.8 ** l - 1.0) + 0.01


def _key1(q: int, tag: int) -> int:
    return ((int(q) << 8) | int(tag)) & 0xFFFFFFFF


def uniform(seed: int, q: int, tag: int, c0, c1, lo: float, hi: float) -> np.ndarray:
    w0, w1, _, _ = philox4x32_10(c0, c1, 0, 0, seed, _key1(q, tag))
    return lo + (hi - lo) * u53(w0, w1)


def eps_occ(seed: int, q: int, k: int, n_occ: int) -> np.ndarray:
    """Occupied levels of k-point k: U[-0.8, 0] Ry, sorted ascending."""
    return np.sort(uniform(seed, q, TAG_EPS_OCC, k, np.arange(n_occ), -0.8, 0.0))


def eps_unocc(seed: int, q: int, k: int, n_unocc: int) -> np.ndarray:
    """Unoccupied levels of k-point k: U[0.05, 3.0] Ry, sorted ascending."""
    return np.sort(uniform(seed, q, TAG_EPS_UNOCC, k, np.arange(n_unocc), 0.05, 3.0))


def coulomb_v(seed: int, q: int, n_pb: int) -> np.ndarray:
    """Diagonal Coulomb eigenvalues v_I = 4 pi / |G_I|^2 with |G_I| ~ U[0.3, 6]."""
    g = uniform(seed, q, TAG_G, np.arange(n_pb), 0, 0.3, 6.0)
    return 4.0 * math.pi / (g * g)


def row_scale(n_pb: int, s_div: float) -> np.ndarray:
    return 1.0 / (1.0 + np.arange(n_pb, dtype=np.float64) / s_div)


def _z_values(seed, q, k, n, m, I, s):
    w0, w1, w2, w3 = philox4x32_10(k, n, m, I, seed, _key1(q, TAG_Z))
    u1 = (u53(w0, w1) + 2.0 ** -53)  # (0, 1]
    u2 = u53(w2, w3)
    rad = np.sqrt(-np.log(u1))
    ang = 2.0 * math.pi * u2
    return (rad * np.cos(ang) + 1j * (rad * np.sin(ang))) * s


def z_block(seed: int, q: int, k: int, n_pb: int, n_occ: int, n_unocc: int, s_div: float) -> np.ndarray:
    """All columns of k-point k as a C-ordered (n_occ*n_unocc, n_pb) complex128 array Zt."""
    r = np.arange(n_occ * n_unocc, dtype=np.int64)
    n = (r // n_unocc)[:, None]
    m = (r % n_unocc)[:, None]
    I = np.arange(n_pb, dtype=np.int64)[None, :]
    s = row_scale(n_pb, s_div)[None, :]
    return np.ascontiguousarray(_z_values(seed, q, k, n, m, I, s))


def z_rows(seed: int, q: int, rows, n_k: int, n_occ: int, unocc_of_k, s_div: float, k_begin: int = 0) -> np.ndarray:
    """Rows I in `rows` of Z over all columns of k-points k_begin..n_k-1, shape (len(rows), K).

    `unocc_of_k(k)` gives n_unocc for k-point k. Columns follow (k, n, m) order."""
    rows = np.asarray(rows, dtype=np.int64)
    s = (1.0 / (1.0 + rows.astype(np.float64) / s_div))[:, None]
    parts = []
    for k in range(k_begin, n_k):
        nu = int(unocc_of_k(k))
        r = np.arange(n_occ * nu, dtype=np.int64)
        n = (r // nu)[None, :]
        m = (r % nu)[None, :]
        parts.append(_z_values(seed, q, k, n, m, rows[:, None], s))
    return np.concatenate(parts, axis=1)


def shape_uniform_int(seed: int, q: int, c1: int, a: int, b: int) -> int:
    w0, w1, _, _ = philox4x32_10(q, c1, 0, 0, seed, _key1(0, TAG_SHAPE))
    return a + int(math.floor(float(u53(w0, w1)) * (b - a + 1)))


@dataclass
class Workload:
    """One synthetic chi0 workload. For the batched workload n_pb/n_unocc vary per q / (q, k)."""

    name: str
    n_q: int
    n_k: int
    n_occ: int
    n_omega: int
    s_div: float
    spin: float = 2.0
    seed: int = 1
    n_pb_fixed: int | None = None
    n_unocc_fixed: int | None = None
    n_pb_range: tuple[int, int] | None = None
    n_unocc_range: tuple[int, int] | None = None
    omega: np.ndarray = field(default=None)

    def __post_init__(self):
        if self.omega is None:
            self.omega = omega_grid(self.n_omega)

    def n_pb(self, q: int) -> int:
        if self.n_pb_fixed is not None:
            return self.n_pb_fixed
        a, b = self.n_pb_range
        return shape_uniform_int(self.seed, q, 0, a, b)

    def n_unocc(self, q: int, k: int) -> int:
        if self.n_unocc_fixed is not None:
            return self.n_unocc_fixed
        a, b = self.n_unocc_range
        return shape_uniform_int(self.seed, q, k + 1, a, b)

    def n_cols(self, q: int) -> int:
        return sum(self.n_occ * self.n_unocc(q, k) for k in range(self.n_k))

    def flops(self, q: int | None = None) -> float:
        """Algorithmic chi0 flops F = 4 K N (N+1) L (complex HERK, upper triangle)."""
        qs = range(self.n_q) if q is None else [q]
        return float(sum(4.0 * self.n_cols(qq) * self.n_pb(qq) * (self.n_pb(qq) + 1) * self.n_omega for qq in qs))


# The five synthetic workloads (tiny, medium FP64, medium mixed, batched uneven, large streamed).
TINY = Workload("tiny n_pb=64 K=2048 L=6", n_q=1, n_k=8, n_occ=8, n_omega=6, s_div=16.0, n_pb_fixed=64, n_unocc_fixed=32)
MEDIUM = Workload("medium n_pb=1500 K=1.024M L=12", n_q=1, n_k=64, n_occ=40, n_omega=12, s_div=200.0,
                  n_pb_fixed=1500, n_unocc_fixed=400)
BATCHED = Workload("batched 24 q n_pb~U{900..2200} n_k=32 L=12", n_q=24, n_k=32, n_occ=40, n_omega=12, s_div=200.0,
                   n_pb_range=(900, 2200), n_unocc_range=(250, 600))
LARGE = Workload("large n_pb=4000 K=9.216M L=16", n_q=1, n_k=64, n_occ=120, n_omega=16, s_div=200.0,
                 n_pb_fixed=4000, n_unocc_fixed=1200)
