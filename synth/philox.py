"""Counter-based random numbers: Philox4x32-10.

Written from its published definition (Salmon, Moraes, Dror, Shaw, "Parallel random
numbers: as easy as 1, 2, 3", SC'11): a 4x32-bit counter is mixed with a 2x32-bit key by
ten rounds of two 32x32->64-bit multiplies, the key being bumped by two Weyl constants
between rounds.  Every random draw of the synthetic events is addressed by
(key = (run seed, event), counter = (object, stream, block, kind)), so any subset of the
inputs can be regenerated without generating the rest, on any machine.

This module holds no Kalman-filter arithmetic; it only produces bits and the usual
uniform / Gaussian transforms of them.
"""
from __future__ import annotations

import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def _u32(a) -> np.ndarray:
    return np.asarray(a, dtype=np.uint64) & _MASK


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox rounds on broadcastable arrays of 32-bit words (held in uint64).

    Returns the four output words as uint64 arrays with values < 2**32.
    """
    c0, c1, c2, c3 = _u32(c0), _u32(c1), _u32(c2), _u32(c3)
    k0, k1 = _u32(k0), _u32(k1)
    c0, c1, c2, c3, k0, k1 = np.broadcast_arrays(c0, c1, c2, c3, k0, k1)
    for r in range(10):
        if r:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> _S32, p0 & _MASK
        hi1, lo1 = p1 >> _S32, p1 & _MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def uniform53(a, b) -> np.ndarray:
    """Two 32-bit words -> a double in the open interval (0, 1) with 53 random bits."""
    hi = (np.asarray(a, dtype=np.uint64) >> np.uint64(5)).astype(np.float64)
    lo = (np.asarray(b, dtype=np.uint64) >> np.uint64(6)).astype(np.float64)
    return (hi * 67108864.0 + lo + 0.5) / 9007199254740992.0


def uniforms(key, counter):
    """Two independent U(0,1) doubles per counter: returns (u0, u1)."""
    c0, c1, c2, c3 = counter
    k0, k1 = key
    r0, r1, r2, r3 = philox4x32_10(c0, c1, c2, c3, k0, k1)
    return uniform53(r0, r1), uniform53(r2, r3)


def normals(key, counter):
    """Two independent N(0,1) doubles per counter (Box-Muller on `uniforms`)."""
    u0, u1 = uniforms(key, counter)
    rad = np.sqrt(-2.0 * np.log(u0))
    ang = 2.0 * np.pi * u1
    return rad * np.cos(ang), rad * np.sin(ang)
