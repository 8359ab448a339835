"""Philox4x32-10 counter-based generator and the random draws of the method.

Philox4x32-10 follows its published definition (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds of two
32x32->64 multiplications (multipliers 0xD2511F53 and 0xCD9E8D57) with a Weyl
key schedule (0x9E3779B9, 0xBB67AE85).

Stream layout (counter words c0..c3, key = (seed low word, seed high word)):
  tag 0  feature parameters   c = (0, g, r, 0),  g = global feature index,
                                  r = pair index (two uniforms per call)
  tag 1  count-sketch hashes  c = (1, i, kJ, 0), i = Jacobian row,
                                  kJ = index of the Jacobian evaluation
  tag 2  Gaussian sketch      c = (2, i, q, kJ), q = sketch-row pair index

The features are k, b ~ U[-R, R] (Sec. 2.2, Eq. 2.6); the sketch S_k is drawn
afresh for every Jacobian evaluation (Sec. 4.1).  Gaussian sketch entries are
Box-Muller normals rounded to the grid 2^-4 (nearest, ties to even): each is an
integer of magnitude at most 137 times 2^-4, i.e. one exact 8-bit digit of a
fixed-point tensor-core product (the paper uses a count sketch and fixes no
Gaussian variant; a rounded normal is still a sub-Gaussian embedding).

Parity pinned by the published known-answer vectors of Philox4x32-10
(tests/golden/philox4x32_10_kat.txt).
"""
import numpy as np

MASK32 = np.uint64(0xFFFFFFFF)
_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)


def _u64(x):
    return np.asarray(x, dtype=np.uint64)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10.  All arguments are uint32 values (held in
    uint64 arrays); returns four uint64 arrays of 32-bit words."""
    c0, c1, c2, c3 = (_u64(c) & MASK32 for c in (c0, c1, c2, c3))
    k0 = _u64(k0) & MASK32
    k1 = _u64(k1) & MASK32
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    c0, c1, c2, c3 = (c.copy() for c in (c0, c1, c2, c3))
    for rnd in range(10):
        if rnd:
            k0 = (k0 + _W0) & MASK32
            k1 = (k1 + _W1) & MASK32
        p0 = _M0 * c0
        p1 = _M1 * c2
        n0 = (p1 >> np.uint64(32)) ^ c1 ^ k0
        n1 = p1 & MASK32
        n2 = (p0 >> np.uint64(32)) ^ c3 ^ k1
        n3 = p0 & MASK32
        c0, c1, c2, c3 = n0, n1, n2, n3
    return c0, c1, c2, c3


def seed_key(seed):
    seed = int(seed)
    return seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF


def uniform53(a, b):
    """[0,1) double with 53 random bits from two 32-bit words:
    ((a >> 5) * 2^26 + (b >> 6)) * 2^-53."""
    hi = _u64(a) >> np.uint64(5)
    lo = _u64(b) >> np.uint64(6)
    return (hi * np.uint64(67108864) + lo).astype(np.float64) * (2.0 ** -53)


def features(G, fields, M, dim, R, seed):
    """Feature parameters, array [G, fields, M, dim+1]: k_1..k_dim then b,
    each uniform on [-R, R] (Sec. 2.2: components of k_ij and b_ij drawn
    uniformly from [-R_ij, R_ij])."""
    k0, k1 = seed_key(seed)
    nval = dim + 1
    npair = (nval + 1) // 2
    g = np.arange(G * fields * M, dtype=np.uint64)
    vals = []
    for r in range(npair):
        x0, x1, x2, x3 = philox4x32_10(0, g, r, 0, k0, k1)
        vals.append(uniform53(x0, x1))
        vals.append(uniform53(x2, x3))
    v = np.stack(vals[:nval], axis=1)
    v = R * (2.0 * v - 1.0)
    return v.reshape(G, fields, M, nval)


def count_sketch_hash(m, s, kJ, seed):
    """Bucket h(i) in [0, s) and sign sigma(i) in {+1,-1} of each Jacobian
    row for the count sketch S_k (Sec. 4.1): h = (x0 * s) >> 32,
    sigma = +1 if the low bit of x1 is 0."""
    k0, k1 = seed_key(seed)
    i = np.arange(m, dtype=np.uint64)
    x0, x1, _, _ = philox4x32_10(1, i, kJ, 0, k0, k1)
    h = ((x0 * np.uint64(s)) >> np.uint64(32)).astype(np.int64)
    sig = 1.0 - 2.0 * (x1 & np.uint64(1)).astype(np.float64)
    return h, sig


def round_bf16(x):
    """Round doubles to the nearest bfloat16 value (8 significant bits,
    ties to even), returned as doubles.  Inputs are finite and in the normal
    range of bfloat16."""
    bits = np.asarray(x, dtype=np.float64).view(np.uint64)
    lsb = (bits >> np.uint64(45)) & np.uint64(1)
    bits = (bits + np.uint64(0x0FFFFFFFFFFF) + lsb) & ~np.uint64((1 << 45) - 1)
    return bits.view(np.float64)


def _box_muller_pairs(q, rows, kJ, seed):
    """Both normals of the Box-Muller pair drawn with counter (2, i, q, kJ)
    for every pair index q and Jacobian row i: ([len(q), len(rows)], same)."""
    k0, k1 = seed_key(seed)
    rows = np.asarray(rows, dtype=np.uint64)
    q = np.asarray(q, dtype=np.uint64)
    x0, x1, x2, x3 = philox4x32_10(2, rows[None, :], q[:, None], kJ, k0, k1)
    u1 = uniform53(x0, x1)
    u2 = uniform53(x2, x3)
    rad = np.sqrt(-2.0 * np.log(1.0 - u1))
    th = 6.283185307179586 * u2
    return rad * np.cos(th), rad * np.sin(th)


def gaussian_sketch(s, rows, kJ, seed):
    """Columns `rows` of the Gaussian sketch S_k (s x m): entry (r, i) is the
    (r mod 2)-th Box-Muller normal of the pair drawn with counter
    (2, i, r div 2, kJ), rounded to the nearest multiple of 2^-4.
    Returns [s, len(rows)]."""
    assert s % 2 == 0
    return gaussian_sketch_range(0, s, rows, kJ, seed)


def gaussian_sketch_range(r0, r1, rows, kJ, seed):
    """Rows r0 <= r < r1 (both even) of the Gaussian sketch S_k, columns
    `rows`, by the definition of gaussian_sketch.  Returns [r1 - r0, len(rows)]."""
    assert r0 % 2 == 0 and r1 % 2 == 0 and r1 >= r0
    c, sn = _box_muller_pairs(np.arange(r0 // 2, r1 // 2), rows, kJ, seed)
    out = np.empty((r1 - r0, len(rows)))
    out[0::2] = c
    out[1::2] = sn
    return np.rint(16.0 * out) / 16.0


def gaussian_sketch_rows(srows, rows, kJ, seed):
    """Entries S_k[r, i] for the sketch rows r in `srows` and the Jacobian
    rows i in `rows` (the same definition as gaussian_sketch, for a few rows
    of a sketch too large to draw whole).  Returns [len(srows), len(rows)]."""
    srows = np.asarray(srows, dtype=np.uint64)
    c, sn = _box_muller_pairs(srows // np.uint64(2), rows, kJ, seed)
    out = np.where((srows % np.uint64(2) == 0)[:, None], c, sn)
    return np.rint(16.0 * out) / 16.0