"""Philox4x32-10 counter-based generator and the Gaussian auxiliary fields.

TEST INFRASTRUCTURE: part of the CPU oracle.  Only tests, the smoke check and
the CPU-baseline leg of the benchmark may import it.

The generator is Philox4x32 with 10 rounds as published by Salmon, Moraes,
Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11).  The
GPU library implements the same published definition independently.

The auxiliary fields x ~ p(x) = (2 pi)^(-N_gamma/2) exp(-|x|^2/2) of Sec. 2.2
(Eq. hs2) are drawn by the Box-Muller transform from the generator's words:

* key     = (seed & 0xffffffff, seed >> 32)
* counter = (gamma >> 1, walker, step, 0) for the field pair (2k, 2k+1)
* u1 from words (x0, x1), u2 from (x2, x3), each
  u = fl(fl(a + 0.5) * 2^-53) with a = (x_hi >> 5) * 2^26 + (x_lo >> 6)
* xi[2k] = sqrt(-2 ln u1) cos(2 pi u2), xi[2k+1] = sqrt(-2 ln u1) sin(2 pi u2)

The comb of the population control takes its uniform from the counter
(0, 0xffffffff, step, 0), words (x0, x1).
"""
from __future__ import annotations

import numpy as np

_MASK = np.uint64(0xFFFFFFFF)
_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)
_SH32 = np.uint64(32)

TWO_PI = 6.283185307179586
COMB_WALKER = 0xFFFFFFFF


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox rounds on broadcastable uint32-valued arrays.

    Each round: (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2 (32x32 -> 64 bit),
    new counter = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); the key is bumped
    by the Weyl constants (W0, W1) before every round but the first.
    """
    c0, c1, c2, c3, k0, k1 = (np.asarray(v, dtype=np.uint64) & _MASK
                              for v in (c0, c1, c2, c3, k0, k1))
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    for r in range(10):
        if r:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> _SH32, p0 & _MASK
        hi1, lo1 = p1 >> _SH32, p1 & _MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def _key(seed: int):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return np.uint64(seed & 0xFFFFFFFF), np.uint64(seed >> 32)


def uniform53(x_hi, x_lo):
    """u in (0, 1]: fl(fl(a + 0.5) * 2^-53), a = (x_hi>>5)*2^26 + (x_lo>>6)."""
    a = (np.asarray(x_hi, np.uint64) >> np.uint64(5)) * np.uint64(1 << 26) \
        + (np.asarray(x_lo, np.uint64) >> np.uint64(6))
    return (a.astype(np.float64) + 0.5) * (2.0 ** -53)


def gaussian_fields(seed: int, step: int, walkers, nchol: int) -> np.ndarray:
    """xi[w, g] ~ N(0, 1) for the given walker indices at one step."""
    walkers = np.asarray(walkers, dtype=np.uint64).reshape(-1, 1)
    npair = (nchol + 1) // 2
    pair = np.arange(npair, dtype=np.uint64).reshape(1, -1)
    k0, k1 = _key(seed)
    x0, x1, x2, x3 = philox4x32_10(pair, walkers, np.uint64(step), 0, k0, k1)
    u1 = uniform53(x0, x1)
    u2 = uniform53(x2, x3)
    r = np.sqrt(-2.0 * np.log(u1))
    ang = TWO_PI * u2
    xi = np.empty((walkers.shape[0], 2 * npair))
    xi[:, 0::2] = r * np.cos(ang)
    xi[:, 1::2] = r * np.sin(ang)
    return xi[:, :nchol]


def comb_uniform(seed: int, step: int) -> float:
    """The single uniform that places the comb's teeth at one step."""
    k0, k1 = _key(seed)
    x0, x1, _, _ = philox4x32_10(0, COMB_WALKER, np.uint64(step), 0, k0, k1)
    return float(uniform53(x0, x1))
