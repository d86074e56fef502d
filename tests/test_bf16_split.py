"""The operand split of the tensor-core projection products, emulated on the
host in numpy (CPU only).

Every FP32 operand x is split into three bf16 numbers with round-to-nearest:
b0 = RN(x), b1 = RN(x - b0), b2 = x - b0 - b1, and the MMAs accumulate the six
products a0 b0 + a0 b1 + a1 b0 + a0 b2 + a1 b1 + a2 b0.  Checked here: the
differences are exact in FP32, b2 is itself a bf16 number (so x = b0 + b1 + b2
exactly), every piece product is exact in FP32 (8 x 8 significant bits), and
the six-product sum matches the exact product a b to 2^-22 relative (about one
FP32 rounding), against about 2^-9 for the leading product alone and 2^-19 for a
two-piece TF32 split.
"""
import numpy as np


def bf16_rn(x):
    """float32 -> the nearest bf16 number (ties to even), as float32."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32)


def tf32_trunc(x):
    """float32 with its low 13 mantissa bits cleared (the TF32 part the hardware reads)."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32)
    return (u & np.uint32(0xFFFFE000)).view(np.float32)


def split3(x):
    x = np.asarray(x, dtype=np.float32)
    b0 = bf16_rn(x)
    r = (x - b0).astype(np.float32)
    b1 = bf16_rn(r)
    b2 = (r - b1).astype(np.float32)
    return b0, b1, b2


def samples(n, seed, emax=60):
    rng = np.random.default_rng(seed)
    m = rng.uniform(1.0, 2.0, n) * rng.choice([-1.0, 1.0], n)
    e = rng.integers(-emax, emax, n)
    return (m * np.exp2(e)).astype(np.float32)


def test_split_is_exact():
    x = samples(200_000, 1)
    b0, b1, b2 = split3(x)
    # the differences were formed exactly in FP32
    assert np.array_equal(x.astype(np.float64) - b0.astype(np.float64), (x - b0).astype(np.float64))
    # the third piece is a bf16 number, so nothing is lost
    assert np.array_equal(bf16_rn(b2), b2)
    assert np.array_equal(b0.astype(np.float64) + b1.astype(np.float64) + b2.astype(np.float64),
                          x.astype(np.float64))
    # each piece has at most 8 significant bits and the pieces shrink by 2^-8 or more
    nz = b1 != 0
    assert np.all(np.abs(b1[nz]) <= np.abs(b0[nz]) * 2.0 ** -8)
    nz = b2 != 0
    assert np.all(np.abs(b2[nz]) <= np.abs(b1[nz]) * 2.0 ** -8)


def test_piece_products_are_exact_in_fp32():
    # exponents within +-30: the smallest piece products stay clear of FP32 underflow (the
    # projections' operands are normalised vectors, far from either end of the range)
    a, b = split3(samples(50_000, 2, 30)), split3(samples(50_000, 3, 30))
    for i in range(3):
        for j in range(3):
            p32 = (a[i] * b[j]).astype(np.float32)
            assert np.array_equal(p32.astype(np.float64), a[i].astype(np.float64) * b[j].astype(np.float64))


def test_six_products_match_fp32_products():
    x, y = samples(200_000, 4), samples(200_000, 5)
    a, b = split3(x), split3(y)
    exact = x.astype(np.float64) * y.astype(np.float64)
    six = sum(a[i].astype(np.float64) * b[j].astype(np.float64) for i, j in ((0, 0), (0, 1), (1, 0), (0, 2), (1, 1), (2, 0)))
    rel6 = np.abs(six - exact) / np.abs(exact)
    assert rel6.max() <= 2.0 ** -22
    lead = a[0].astype(np.float64) * b[0].astype(np.float64)
    assert (np.abs(lead - exact) / np.abs(exact)).max() > 2.0 ** -12   # one piece is far from enough
    # the two-piece TF32 split (truncated high part, the tensor core truncating the rest) is
    # more than an order of magnitude less accurate
    xh, yh = tf32_trunc(x), tf32_trunc(y)
    xl, yl = tf32_trunc((x - xh).astype(np.float32)), tf32_trunc((y - yh).astype(np.float32))
    tf = xh.astype(np.float64) * yh + xh.astype(np.float64) * yl + xl.astype(np.float64) * yh
    rel_tf = np.abs(tf - exact) / np.abs(exact)
    assert rel_tf.max() > 2.0 ** -21 and rel_tf.max() > 20 * rel6.max()
