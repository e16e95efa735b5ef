"""Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, "Parallel
random numbers: as easy as 1, 2, 3", SC'11), vectorised over numpy arrays.

This module draws the synthetic inputs only; it holds none of the GW arithmetic.
The CUDA library carries its own implementation of the same published
definition, so that a device-side generator and this host-side one produce the
same integers for the same (counter, key).
"""
import numpy as np

_MASK = 0xFFFFFFFF
# round multipliers and Weyl key increments of Philox4x32 (SC'11, Table 2)
_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = 0x9E3779B9
_W1 = 0xBB67AE85


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox rounds on counters (c0..c3) with key (k0, k1).

    All arguments are broadcastable integer arrays/scalars holding 32-bit
    values. Returns four uint32 arrays.
    """
    x0 = np.asarray(c0, dtype=np.uint64) & np.uint64(_MASK)
    x1 = np.asarray(c1, dtype=np.uint64) & np.uint64(_MASK)
    x2 = np.asarray(c2, dtype=np.uint64) & np.uint64(_MASK)
    x3 = np.asarray(c3, dtype=np.uint64) & np.uint64(_MASK)
    x0, x1, x2, x3 = np.broadcast_arrays(x0, x1, x2, x3)
    key0 = np.asarray(k0, dtype=np.uint64) & np.uint64(_MASK)
    key1 = np.asarray(k1, dtype=np.uint64) & np.uint64(_MASK)
    m32 = np.uint64(_MASK)
    s32 = np.uint64(32)
    for r in range(10):
        if r:
            key0 = (key0 + np.uint64(_W0)) & m32
            key1 = (key1 + np.uint64(_W1)) & m32
        p0 = _M0 * x0
        p1 = _M1 * x2
        hi0, lo0 = p0 >> s32, p0 & m32
        hi1, lo1 = p1 >> s32, p1 & m32
        x0, x1, x2, x3 = hi1 ^ x1 ^ key0, lo1, hi0 ^ x3 ^ key1, lo0
    return (x0.astype(np.uint32), x1.astype(np.uint32),
            x2.astype(np.uint32), x3.astype(np.uint32))


def uniform53(a, b):
    """Uniform double in [0, 1) from two 32-bit words (27 + 26 high bits)."""
    a = np.asarray(a, dtype=np.uint64)
    b = np.asarray(b, dtype=np.uint64)
    hi = (a >> np.uint64(5)).astype(np.float64)
    lo = (b >> np.uint64(6)).astype(np.float64)
    return (hi * 67108864.0 + lo) * (1.0 / 9007199254740992.0)


def normal_pair(x0, x1, x2, x3):
    """Box-Muller (1958) pair of standard normals from one Philox output block.

    u1 in (0, 1] from (x0, x1), u2 in [0, 1) from (x2, x3);
    returns (r cos 2 pi u2, r sin 2 pi u2) with r = sqrt(-2 ln u1).
    """
    u1 = 1.0 - uniform53(x0, x1)
    u2 = uniform53(x2, x3)
    r = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * np.pi * u2
    return r * np.cos(ang), r * np.sin(ang)


def split_index(idx):
    """64-bit element index -> (low 32 bits, high 32 bits)."""
    idx = np.asarray(idx, dtype=np.uint64)
    return idx & np.uint64(_MASK), idx >> np.uint64(32)
