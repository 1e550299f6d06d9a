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

Box-Muller needs a logarithm and a sine / cosine.  They are written out here
from their series (log through atanh, sin and cos through Taylor series after
an exact reduction to [0, pi/4]) with only additions, multiplications, one
division and one square root, every operation rounded once (numpy evaluates
each array operation separately, with no fused multiply-add).  A device-side
generator that performs the same operations in the same order, each rounded
to nearest, therefore produces the same bits; the library's CUDA heat bath
does that.  Accuracy: a few units in the last place (tests pin it against
numpy's own log, sin and cos).
"""
import math
from fractions import Fraction

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


# Constants of the functions below: each is the double nearest to an exact value.
_LN2 = Fraction("0.69314718055994530941723212145817656807550013436026")
LN2_HI = float(Fraction(math.floor(_LN2 * 2 ** 32), 2 ** 32))   # 32 significant bits: e * LN2_HI is exact
LN2_LO = float(_LN2 - Fraction(LN2_HI))
PI_HALF = float(Fraction("1.57079632679489661923132169163975144209858469968755"))
SQRT_HALF = float(Fraction("0.70710678118654752440084436210484903928483593768847"))
ATANH_C = [float(Fraction(1, 2 * k + 1)) for k in range(11)]                         # w^k / (2k+1)
SIN_C = [float(Fraction((-1) ** k, math.factorial(2 * k + 1))) for k in range(10)]    # x^(2k+1) terms
COS_C = [float(Fraction((-1) ** k, math.factorial(2 * k))) for k in range(10)]        # x^(2k) terms


def log_unit(v):
    """Natural logarithm of v in (0, 1] (any positive normal v works).

    v = f 2^e with f in [sqrt(1/2), sqrt(2)) (frexp, exact); log f = 2 atanh(z) with
    z = (f - 1) / (f + 1), |z| <= 0.1716, and atanh(z) = z sum_k z^2k / (2k + 1) summed
    to k = 10 (the first omitted term is below 2^-60 relative); log v = e ln 2 + log f
    with ln 2 split in two so that e ln 2_hi is exact."""
    f, e = np.frexp(np.asarray(v, dtype=np.float64))
    small = f < SQRT_HALF
    f = np.where(small, f * 2.0, f)
    e = np.where(small, e - 1, e).astype(np.float64)
    z = (f - 1.0) / (f + 1.0)
    w = z * z
    s = ATANH_C[10] * w + ATANH_C[9]
    for c in ATANH_C[8::-1]:
        s = s * w + c
    q = z * s
    return e * LN2_HI + (e * LN2_LO + (q + q))


def sincos_2pi(u):
    """(sin 2 pi u, cos 2 pi u) for u in [0, 1).

    4u = n + f with the quadrant n = floor(4u) and f in [0, 1), both exact; for
    f > 1/2 the complementary angle 1 - f (exact) is used, so the series run on
    x = (pi / 2) h with h in [0, 1/2], x in [0, pi/4]: sin x = x + x^3 (...) and
    cos x = 1 + x^2 (...) to the x^19 and x^18 terms, then the quadrant rotates them."""
    u = np.asarray(u, dtype=np.float64)
    q4 = u * 4.0
    n = np.floor(q4)
    f = q4 - n
    hi = f > 0.5
    h = np.where(hi, 1.0 - f, f)
    x = h * PI_HALF
    w = x * x
    ps = SIN_C[9] * w + SIN_C[8]
    for c in SIN_C[7:0:-1]:
        ps = ps * w + c
    sx = x + (x * w) * ps
    pc = COS_C[9] * w + COS_C[8]
    for c in COS_C[7:0:-1]:
        pc = pc * w + c
    cx = 1.0 + w * pc
    sf = np.where(hi, cx, sx)        # sin of (pi / 2) f
    cf = np.where(hi, sx, cx)        # cos of (pi / 2) f
    n = n.astype(np.int64)
    sin = np.choose(n, [sf, cf, -sf, -cf])
    cos = np.choose(n, [cf, -sf, -cf, sf])
    return sin, cos


def box_muller(u1, u2):
    """Two independent N(0,1) variates from two uniforms in [0, 1):
    r = sqrt(-2 log(1 - u1)) (1 - u1 lies in (0, 1], exactly), angle 2 pi u2."""
    r = np.sqrt(-2.0 * log_unit(1.0 - np.asarray(u1, dtype=np.float64)))
    s, c = sincos_2pi(u2)
    return r * c, r * s


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
