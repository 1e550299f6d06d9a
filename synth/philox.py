"""Philox4x32-10 counter-based generator, vectorised over numpy arrays.

Written from the published definition (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11, section 3.3 and
table 2): a 4-word counter and a 2-word key go through ten rounds; each
round multiplies counter words 0 and 2 by the constants M0, M1, keeps the
high and low halves of the 64-bit products, xors the high halves with the
other two counter words and the key, and permutes; the key is bumped by
the Weyl constants W0, W1 between rounds.

Also here: the mapping of two 32-bit words to a double in [0, 1) with 53
random bits, and the Box-Muller transform to standard normals.
"""
import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Return the four 32-bit output words for counters (c0..c3), key (k0, k1).

    All arguments broadcast against each other; the results are uint32
    arrays of the broadcast shape.
    """
    c0, c1, c2, c3, k0, k1 = np.broadcast_arrays(
        *(np.asarray(v, dtype=np.uint64) & _MASK for v in (c0, c1, c2, c3, k0, k1)))
    c0, c1, c2, c3 = c0.copy(), c1.copy(), c2.copy(), c3.copy()
    k0, k1 = k0.copy(), k1.copy()
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> _S32, p0 & _MASK
        hi1, lo1 = p1 >> _S32, p1 & _MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0
    return tuple(v.astype(np.uint32) for v in (c0, c1, c2, c3))


def uniform53(a, b):
    """Double in [0, 1) from two 32-bit words: 27 bits of a, 26 bits of b."""
    a = np.asarray(a, dtype=np.uint64) >> np.uint64(5)
    b = np.asarray(b, dtype=np.uint64) >> np.uint64(6)
    return (a.astype(np.float64) * 67108864.0 + b.astype(np.float64)) * (1.0 / 9007199254740992.0)


def box_muller(u1, u2):
    """Two independent N(0,1) variates from two uniforms in [0, 1)."""
    r = np.sqrt(-2.0 * np.log1p(-u1))      # 1 - u1 lies in (0, 1]
    th = 2.0 * np.pi * u2
    return r * np.cos(th), r * np.sin(th)


def gaussians(n_pairs_per_item, c_first, c_second, key, stream, counter_slot=2):
    """Standard normals, 2 per generator call, n_pairs_per_item calls per item.

    ``c_first`` and ``c_second`` are the per-item counter words 0 and 1 (any
    broadcastable integer arrays); the call index runs in counter word
    ``counter_slot``; the key is (seed, stream).  Returns shape
    item_shape + (2 * n_pairs_per_item,).
    """
    c_first = np.asarray(c_first, dtype=np.uint64)
    c_second = np.asarray(c_second, dtype=np.uint64)
    shape = np.broadcast(c_first, c_second).shape
    out = np.empty(shape + (2 * n_pairs_per_item,), dtype=np.float64)
    for k in range(n_pairs_per_item):
        ctr = [c_first, c_second, np.uint64(0), np.uint64(0)]
        ctr[counter_slot] = np.uint64(k)
        w = philox4x32_10(ctr[0], ctr[1], ctr[2], ctr[3], key, stream)
        z0, z1 = box_muller(uniform53(w[0], w[1]), uniform53(w[2], w[3]))
        out[..., 2 * k] = z0
        out[..., 2 * k + 1] = z1
    return out
