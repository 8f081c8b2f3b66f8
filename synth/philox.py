"""Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11), vectorised in numpy.

Every draw is a pure function of (key, counter), so any subset of a bunch can
be regenerated without generating the rest, and the host and the oracle see
identical numbers.
"""
import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint32(0x9E3779B9)
_W1 = np.uint32(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox4x32 rounds on uint32 arrays (broadcastable); returns 4 arrays."""
    c0 = np.asarray(c0, dtype=np.uint32)
    c1 = np.asarray(c1, dtype=np.uint32)
    c2 = np.asarray(c2, dtype=np.uint32)
    c3 = np.asarray(c3, dtype=np.uint32)
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    k0 = np.uint32(k0)
    k1 = np.uint32(k1)
    with np.errstate(over="ignore"):
        for r in range(10):
            p0 = _M0 * c0.astype(np.uint64)
            p1 = _M1 * c2.astype(np.uint64)
            hi0 = (p0 >> _S32).astype(np.uint32)
            lo0 = (p0 & _MASK).astype(np.uint32)
            hi1 = (p1 >> _S32).astype(np.uint32)
            lo1 = (p1 & _MASK).astype(np.uint32)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
            if r < 9:
                k0 = np.uint32((int(k0) + int(_W0)) & 0xFFFFFFFF)
                k1 = np.uint32((int(k1) + int(_W1)) & 0xFFFFFFFF)
    return c0, c1, c2, c3


def uniform53(a, b):
    """Two uint32 words -> double uniform on [0, 1) with 53 random bits."""
    hi = (a >> np.uint32(5)).astype(np.float64)   # 27 bits
    lo = (b >> np.uint32(6)).astype(np.float64)   # 26 bits
    return (hi * 67108864.0 + lo) * (1.0 / 9007199254740992.0)


def normal_pairs(seed, index, stream, attempt=0):
    """Two independent standard normals per (seed, index, stream, attempt).

    Counter = (index low word, index high word, stream, attempt),
    key = (seed low word, seed high word). Box-Muller on two 53-bit uniforms.
    """
    index = np.asarray(index, dtype=np.uint64)
    c0 = (index & _MASK).astype(np.uint32)
    c1 = (index >> _S32).astype(np.uint32)
    seed = int(seed)
    r0, r1, r2, r3 = philox4x32_10(c0, c1, np.uint32(stream), np.uint32(attempt),
                                   seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    u1 = 1.0 - uniform53(r0, r1)          # (0, 1]
    u2 = uniform53(r2, r3)
    rad = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * np.pi * u2
    return rad * np.cos(ang), rad * np.sin(ang)


def uniforms(seed, index, stream):
    """Two uniforms on [0, 1) per (seed, index, stream)."""
    index = np.asarray(index, dtype=np.uint64)
    c0 = (index & _MASK).astype(np.uint32)
    c1 = (index >> _S32).astype(np.uint32)
    seed = int(seed)
    r0, r1, r2, r3 = philox4x32_10(c0, c1, np.uint32(stream), np.uint32(0),
                                   seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    return uniform53(r0, r1), uniform53(r2, r3)
