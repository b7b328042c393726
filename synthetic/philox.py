"""Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, "Parallel random
numbers: as easy as 1, 2, 3", SC'11), vectorised over numpy uint64 arrays.

This is the host-side generator that feeds the oracle and the tests. The CUDA library has
its own device implementation of the same published definition; the two are pinned to the
published known-answer vectors independently and share no code.

Definition used (Philox-4x32 with R=10 rounds):
  round:   (c0,c1,c2,c3) -> (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0))
  key bump between rounds: k0 += W0, k1 += W1 (mod 2^32); the first round uses the key as given.
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Return the four 32-bit output words (as uint64 arrays) for counters c0..c3 and key k0,k1.

    All arguments broadcast; values must lie in [0, 2^32)."""
    c0 = np.asarray(c0, dtype=np.uint64) & MASK32
    c1 = np.asarray(c1, dtype=np.uint64) & MASK32
    c2 = np.asarray(c2, dtype=np.uint64) & MASK32
    c3 = np.asarray(c3, dtype=np.uint64) & MASK32
    k0 = np.asarray(k0, dtype=np.uint64) & MASK32
    k1 = np.asarray(k1, dtype=np.uint64) & MASK32
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    for rnd in range(10):
        if rnd:
            k0 = (k0 + W0) & MASK32
            k1 = (k1 + W1) & MASK32
        p0 = M0 * c0  # < 2^64: exact in uint64
        p1 = M1 * c2
        c0, c1, c2, c3 = ((p1 >> _S32) ^ c1 ^ k0, p1 & MASK32, (p0 >> _S32) ^ c3 ^ k1, p0 & MASK32)
    return c0, c1, c2, c3


_TWO_M53 = 2.0 ** -53


def u53(w_hi, w_lo):
    """53-bit uniform in [0, 1) from two 32-bit words: ((w_hi << 21) | (w_lo >> 11)) * 2^-53."""
    w_hi = np.asarray(w_hi, dtype=np.uint64)
    w_lo = np.asarray(w_lo, dtype=np.uint64)
    bits = (w_hi << np.uint64(21)) | (w_lo >> np.uint64(11))
    return bits.astype(np.float64) * _TWO_M53
