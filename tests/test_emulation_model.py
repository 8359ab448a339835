"""CPU model of the integer arithmetic inside the emulated-FP64 products (the
digit split and the final rounding of the tensor-core levels), checked against
exact rational arithmetic.  The GPU kernels themselves are held to FP64 bounds
by the GPU tests; this pins the scheme's two exact steps:

  * balanced base-2^7 digits: V = round(x 2^(7 ndig - e)) split into ndig-1 low
    digits in [-64, 63] and a top digit; extracting 7-bit fields of
    V + 64 (1 + 2^7 + ... + 2^(7(ndig-2))) gives the same digits as peeling V
    from its low end with nearest remainders;
  * the level sums of one 512-deep chunk stay below 2^24 for levels 0-3 (so
    their FP32 accumulation is exact), and (ah 2^28 + al) 2^k is rounded to the
    nearest double (ties to even) by a leading-bit / round-bit / sticky-bit
    construction on a 128-bit two's-complement value."""
import random
import struct
from fractions import Fraction

import pytest

M64 = (1 << 64) - 1
MAXD = 8


def peel(V, ndig):
    d = [0] * ndig
    for p in range(ndig - 1, 0, -1):
        r = V & 127
        if r >= 64:
            r -= 128
        d[p] = r
        V = (V - r) >> 7
    d[0] = V
    return d


def fields(V, ndig):
    U = V + (0x0001020408102040 >> (7 * (MAXD - ndig)))
    d = [0] * ndig
    for dd in range(1, ndig):
        d[dd] = ((U >> (7 * (ndig - 1 - dd))) & 127) - 64
    d[0] = U >> (7 * (ndig - 1))
    return d


def to_double(ah, al, k):
    h = ah >> 36
    l0 = (ah << 28) & M64
    l = (l0 + (al & M64)) & M64
    h = h + (-1 if al < 0 else 0) + (1 if l < l0 else 0)
    neg = h < 0
    H, L = h & M64, l
    if neg:
        L = (~L + 1) & M64
        H = (~H + (1 if L == 0 else 0)) & M64
    if H == 0 and L == 0:
        return 0.0
    msb = (127 - (64 - H.bit_length())) if H else (63 - (64 - L.bit_length()))
    sh = msb - 52
    if sh <= 0:
        mant, up = (L << (-sh)) & M64, False
    else:
        mant = ((L >> sh) | (H << (64 - sh))) & M64
        rbit = (L >> (sh - 1)) & 1
        sticky = (L & ((1 << (sh - 1)) - 1)) != 0
        up = bool(rbit) and (sticky or bool(mant & 1))
    if up:
        mant += 1
        if mant >> 53:
            mant >>= 1
            msb += 1
    e = msb + k + 1023
    assert 0 < e < 2047
    return struct.unpack("<d", struct.pack("<Q", (int(neg) << 63) | (e << 52) | (mant & ((1 << 52) - 1))))[0]


@pytest.mark.parametrize("ndig", range(1, MAXD + 1))
def test_field_extract_digits_equal_peeled_digits(ndig):
    rng = random.Random(ndig)
    for _ in range(3000):
        V = rng.randint(-(1 << (7 * ndig)), 1 << (7 * ndig))
        d = fields(V, ndig)
        assert d == peel(V, ndig)
        assert all(-64 <= x <= 63 for x in d[1:]) and abs(d[0]) <= 128
        assert sum(x << (7 * (ndig - 1 - p)) for p, x in enumerate(d)) == V


def test_leading_level_sums_fit_fp32_exactly():
    # worst case over a 512-deep chunk: top digits up to 128, lower digits up to 64
    top, low = 128, 64
    for lev in range(4):
        pairs = [(p, lev - p) for p in range(lev + 1)]
        worst = 512 * sum((top if p == 0 else low) * (top if q == 0 else low) for p, q in pairs)
        assert worst < 1 << 24, (lev, worst)


def test_integer_rounding_to_double_is_correctly_rounded():
    rng = random.Random(7)
    for _ in range(50000):
        ah = rng.randint(-(1 << 53), 1 << 53) >> rng.randint(0, 53)
        al = rng.randint(-(1 << 54), 1 << 54) >> rng.randint(0, 54)
        k = rng.randint(-300, 300)
        exact = Fraction(ah * (1 << 28) + al) * Fraction(2) ** k
        assert to_double(ah, al, k) == float(exact)
    # ties go to even
    assert to_double(0, (1 << 53) + 1, 0) == float(1 << 53)
    assert to_double(0, (1 << 53) + 3, 0) == float((1 << 53) + 4)
