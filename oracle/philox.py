"""Philox4x64-10 counter-based generator (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11).

The paper fixes no random-number generator. The circuit sampler draws one
Philox4x64-10 block per gate (j, k) with key (seed, sample) and counter
(j, k, 0, 0). This file implements the generator from its published
definition: ten rounds of two 64x64->128-bit multiplies and Weyl key bumps.
A scalar version uses Python integers. A vectorised version uses numpy
uint64 arrays.
"""
from __future__ import annotations

import numpy as np

MASK64 = (1 << 64) - 1
PHILOX_M0 = 0xD2E7470EE14C6C93
PHILOX_M1 = 0xCA5A826395121157
PHILOX_W0 = 0x9E3779B97F4A7C15   # golden ratio
PHILOX_W1 = 0xBB67AE8584CAA73B   # sqrt(3) - 1


def philox4x64_scalar(ctr, key, rounds: int = 10):
    """One Philox4x64 block: ctr = (x0, x1, x2, x3), key = (k0, k1)."""
    x0, x1, x2, x3 = (int(c) & MASK64 for c in ctr)
    k0, k1 = (int(k) & MASK64 for k in key)
    for rnd in range(rounds):
        if rnd > 0:
            k0 = (k0 + PHILOX_W0) & MASK64
            k1 = (k1 + PHILOX_W1) & MASK64
        p0 = PHILOX_M0 * x0
        p1 = PHILOX_M1 * x2
        hi0, lo0 = p0 >> 64, p0 & MASK64
        hi1, lo1 = p1 >> 64, p1 & MASK64
        x0, x1, x2, x3 = hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0
    return x0, x1, x2, x3


_M32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def _mulhilo(a: np.ndarray, b: np.uint64):
    """Full 128-bit product of uint64 arrays, split as (hi, lo)."""
    a_lo, a_hi = a & _M32, a >> _S32
    b_lo, b_hi = np.uint64(int(b) & 0xFFFFFFFF), np.uint64(int(b) >> 32)
    p0 = a_lo * b_lo
    p1 = a_lo * b_hi
    p2 = a_hi * b_lo
    p3 = a_hi * b_hi
    mid = (p0 >> _S32) + (p1 & _M32) + (p2 & _M32)
    hi = p3 + (p1 >> _S32) + (p2 >> _S32) + (mid >> _S32)
    lo = a * np.uint64(int(b))
    return hi, lo


def philox4x64_vec(x0, x1, x2, x3, k0: int, k1: int, rounds: int = 10):
    """Vectorised Philox4x64 over uint64 counter arrays with a scalar key."""
    x0 = np.asarray(x0, dtype=np.uint64).copy()
    x1 = np.asarray(x1, dtype=np.uint64).copy()
    x2 = np.asarray(x2, dtype=np.uint64).copy()
    x3 = np.asarray(x3, dtype=np.uint64).copy()
    kk0, kk1 = int(k0) & MASK64, int(k1) & MASK64
    with np.errstate(over='ignore'):
        for rnd in range(rounds):
            if rnd > 0:
                kk0 = (kk0 + PHILOX_W0) & MASK64
                kk1 = (kk1 + PHILOX_W1) & MASK64
            hi0, lo0 = _mulhilo(x0, np.uint64(PHILOX_M0))
            hi1, lo1 = _mulhilo(x2, np.uint64(PHILOX_M1))
            x0, x1, x2, x3 = (hi1 ^ x1 ^ np.uint64(kk0), lo1,
                              hi0 ^ x3 ^ np.uint64(kk1), lo0)
    return x0, x1, x2, x3
