"""Pins for the oracle's SLRME steps (Sec. III-B, Eqs. 8-10) and the
residual / decoder (Sec. III-C).

References: scipy.ndimage (Gaussian restoration), numpy.bincount (binned
sums), Python's correctly rounded int -> float, exact Fraction least
squares and numpy.polyfit (Eqs. 6-7), planted exact-linear data, Decimal
half-away rounding, and the reversibility invariant.
"""
import random
from decimal import ROUND_HALF_UP, Decimal
from fractions import Fraction

import numpy as np
import pytest
from scipy import ndimage

from oracle import oracle as O
from paper_2309_11072_gb300 import synth

# ------------------------------------------------------------------ GF


def test_gf_against_scipy_nearest():
    rng = np.random.default_rng(1)
    s3 = rng.integers(0, 256, size=(3, 17, 23)).astype(np.uint8)
    x3 = O.gf(s3, True)
    k = np.outer([1, 2, 1], [1, 2, 1])
    for c in range(3):
        ref = ndimage.correlate(s3[c].astype(np.int64), k, mode="nearest")
        assert np.array_equal(x3[c], ref)


def test_gf_constant_and_off():
    s3 = np.full((3, 5, 7), 201, np.uint8)
    assert (O.gf(s3, True) == 16 * 201).all()
    rng = np.random.default_rng(2)
    s3 = rng.integers(0, 256, size=(3, 4, 9)).astype(np.uint8)
    assert np.array_equal(O.gf(s3, False), 16 * s3.astype(np.int32))


def test_gf_single_pixel_and_single_row():
    one = np.full((3, 1, 1), 9, np.uint8)
    assert (O.gf(one) == 144).all()
    row = np.arange(6, dtype=np.uint8)[None, None, :].repeat(3, 0)
    x = O.gf(row)[0, 0]
    # one row: vertical taps all see the same row (4x), horizontal [1 2 1] with replication
    ref = 4 * np.convolve(np.pad(np.arange(6), 1, mode="edge"), [1, 2, 1], mode="valid")
    assert np.array_equal(x, ref)


# ------------------------------------------------------------------ sums


def test_bin_sums_against_bincount():
    rng = np.random.default_rng(3)
    h, w = 31, 29
    x3 = rng.integers(0, 4081, size=(3, h, w)).astype(np.int32)
    m3 = rng.integers(0, 256, size=(3, h, w)).astype(np.uint8)
    e = rng.integers(0, 256, size=(h, w)).astype(np.uint8)
    s = O.bin_sums(x3, m3, e)
    ee = e.reshape(-1)
    assert np.array_equal(s[:, 0], np.bincount(ee, minlength=256))
    for c in range(3):
        x = x3[c].reshape(-1).astype(np.int64)
        y = m3[c].reshape(-1).astype(np.int64)
        for j, wts in enumerate((x, y, x * y, x * x)):
            ref = np.zeros(256, dtype=np.int64)
            np.add.at(ref, ee, wts)
            assert np.array_equal(s[:, 1 + 4 * c + j], ref)


# ------------------------------------------------------------------ int128 -> double


def test_i128_to_double_correctly_rounded():
    rnd = random.Random(5)
    cases = [0, 1, -1, 2 ** 53, 2 ** 53 + 1, 2 ** 53 + 2, 2 ** 53 + 3, -(2 ** 53 + 1),
             2 ** 54 + 2, 2 ** 54 + 6, 2 ** 64 - 1, 2 ** 64, 2 ** 100 + 2 ** 47, 2 ** 100 + 2 ** 47 + 1,
             2 ** 126 - 1, -(2 ** 127), 2 ** 127 - 1]
    for _ in range(2000):
        nb = rnd.randint(1, 126)
        v = rnd.getrandbits(nb) * rnd.choice((1, -1))
        cases.append(v)
        # exact ties at many positions
        if nb > 55:
            t = (rnd.getrandbits(53) | (1 << 52)) << (nb - 53)
            cases.append(t + (1 << (nb - 54)))
    for v in cases:
        assert O.i128_to_double(v) == float(v), v


# ------------------------------------------------------------------ solve


def _sums_from_xy(x, y, c=0, E=7):
    s = np.zeros((256, 13), dtype=np.int64)
    x = np.asarray(x, dtype=np.int64)
    y = np.asarray(y, dtype=np.int64)
    s[E, 0] = len(x)
    s[E, 1 + 4 * c:5 + 4 * c] = [x.sum(), y.sum(), (x * y).sum(), (x * x).sum()]
    return s


def test_solve_planted_exact_line():
    # y = x / 16 + 3 exactly (a representable slope): a = 1/16, b = 3
    S = np.arange(0, 250)
    s = _sums_from_xy(16 * S, S + 3, c=1, E=130)
    a, b, n, nu = O.solve(s)
    assert a[1, 130] == np.float32(1 / 16) and b[1, 130] == np.float32(3)
    assert n[130] == 250 and nu == 1


@pytest.mark.parametrize("seed", range(6))
def test_solve_matches_exact_least_squares(seed):
    rng = np.random.default_rng(seed)
    nn = int(rng.integers(2, 400))
    x = rng.integers(0, 4081, size=nn)
    y = np.clip(np.round(x * rng.uniform(0, 0.1) + rng.normal(0, 20, nn)), 0, 255).astype(np.int64)
    s = _sums_from_xy(x, y, c=2, E=99)
    a, b, _, _ = O.solve(s)
    N, sx, sy, sxy, sxx = (int(v) for v in (s[99, 0], *s[99, 9:13]))
    dxx = N * sxx - sx * sx
    dxy = N * sxy - sx * sy
    if dxx == 0:
        return
    exact_a = Fraction(dxy, dxx)                            # Eq. (6)
    ad = float(a[2, 99])
    assert abs(Fraction(ad) - exact_a) <= abs(exact_a) * Fraction(1, 2 ** 23) + Fraction(1, 10 ** 30)
    exact_b = (Fraction(sy) - Fraction(ad) * sx) / N        # Eq. (7) with the sent slope
    assert abs(Fraction(float(b[2, 99])) - exact_b) <= abs(exact_b) * Fraction(1, 2 ** 22) + Fraction(1, 2 ** 40)
    # textbook routine
    pa, pb = np.polyfit(x.astype(np.float64), y.astype(np.float64), 1)
    assert abs(ad - pa) <= 1e-5 * max(1.0, abs(pa))
    assert abs(float(b[2, 99]) - pb) <= 1e-3 * max(1.0, abs(pb))


def test_solve_degenerate_bins():
    s = _sums_from_xy([160, 160, 160], [10, 11, 13], c=0, E=5)   # all x equal
    s[9] = _sums_from_xy([32], [200], c=0, E=9)[9]                 # single pixel
    a, b, n, nu = O.solve(s)
    assert a[0, 5] == 0 and b[0, 5] == np.float32(34 / 3)
    assert a[0, 9] == 0 and b[0, 9] == 200
    # unused regions are zero and not counted
    assert nu == 2 and n[0] == 0 and (a[:, 0] == 0).all() and (b[:, 0] == 0).all()


def test_solve_minimises_squared_error():
    # Eq. (5): the sent (a, b) is no worse than nearby pairs
    rng = np.random.default_rng(11)
    x = rng.integers(0, 4081, size=300)
    y = np.clip(x // 20 + rng.integers(-9, 10, size=300), 0, 255)
    a, b, _, _ = O.solve(_sums_from_xy(x, y, c=0, E=1))
    a0, b0 = float(a[0, 1]), float(b[0, 1])

    def F(aa, bb):
        return float(((y - (aa * x + bb)) ** 2).sum())
    f0 = F(a0, b0)
    for da, db in ((1e-4, 0), (-1e-4, 0), (0, 0.05), (0, -0.05)):
        assert f0 <= F(a0 + da, b0 + db) + 1e-6 * f0


# ------------------------------------------------------------------ Eq. (8)


def _half_away(t: float) -> int:
    return int(Decimal(t).quantize(Decimal(1), rounding=ROUND_HALF_UP))


@pytest.mark.parametrize("t", [0.5, 1.5, 2.5, 254.5, 0.49999997, -0.5, -0.49, 255.0, 254.49998, 1e9, -1e9,
                               127.5, 3.4999998, 0.0, 7e-45])
def test_predict_rounding_and_clipping(t):
    # with a = 0 the pre-rounding value is exactly b
    x3 = np.full((3, 1, 1), 1234, np.int32)
    e = np.full((1, 1), 77, np.uint8)
    a = np.zeros((3, 256), np.float32)
    b = np.zeros((3, 256), np.float32)
    b[:, 77] = np.float32(t)
    ms = O.predict(x3, e, a, b)
    expect = min(255, max(0, _half_away(float(np.float32(t)))))
    assert (ms == expect).all()


def test_predict_random_against_decimal_rounding():
    rng = np.random.default_rng(12)
    h, w = 20, 20
    x3 = rng.integers(0, 4081, size=(3, h, w)).astype(np.int32)
    e = rng.integers(0, 256, size=(h, w)).astype(np.uint8)
    a = rng.uniform(-0.2, 0.2, size=(3, 256)).astype(np.float32)
    b = rng.uniform(-60, 300, size=(3, 256)).astype(np.float32)
    ms = O.predict(x3, e, a, b)
    for c in range(3):
        for p in range(0, h * w, 3):
            yy, xx = divmod(p, w)
            E = e[yy, xx]
            t = np.float32(np.float32(a[c, E] * np.float32(x3[c, yy, xx])) + b[c, E])
            assert ms[c, yy, xx] == min(255, max(0, _half_away(float(t))))


@pytest.mark.parametrize("a,x,b,k", [(1.0000001192092896, 4080, -4079.50048828125, 0),
                                     (0.9590728878974915, 2086, -2000.1260986328125, 0),
                                     (0.07105054706335068, 1101, -76.72665405273438, 1),
                                     (0.9138873219490051, 3961, -3612.40771484375, 7),
                                     (0.8200012445449829, 2977, -2340.643798828125, 100),
                                     (1.403257966041565, 1132, -1333.988037109375, 254)])
def test_predict_rounds_the_product_before_adding_b(a, x, b, k):
    # Eq. (8) with 32-bit parameters, every operation an IEEE float32 one:
    # here float32(float32(a x) + b) is exactly k + 1/2 (rounded away from
    # zero to k + 1), while the exact a x + b, and so a fused multiply-add,
    # lies below k + 1/2
    from fractions import Fraction
    a32, b32 = np.float32(a), np.float32(b)
    assert float(a32) == a and float(b32) == b
    t = np.float32(np.float32(a32 * np.float32(x)) + b32)
    assert float(t) == k + 0.5
    assert Fraction(a) * x + Fraction(b) < Fraction(2 * k + 1, 2)
    x3 = np.full((3, 1, 1), x, np.int32)
    e = np.full((1, 1), 9, np.uint8)
    A = np.zeros((3, 256), np.float32)
    B = np.zeros((3, 256), np.float32)
    A[:, 9], B[:, 9] = a32, b32
    assert (O.predict(x3, e, A, B) == k + 1).all()


# ------------------------------------------------------------------ residual / decode


def test_residual_histogram_and_range():
    rng = np.random.default_rng(13)
    m3 = rng.integers(0, 256, size=(3, 9, 10)).astype(np.uint8)
    ms = rng.integers(0, 256, size=(3, 9, 10)).astype(np.uint8)
    r3, hist = O.residual(m3, ms)
    assert np.array_equal(r3, m3.astype(np.int16) - ms.astype(np.int16))
    for c in range(3):
        assert np.array_equal(hist[c], np.bincount(r3[c].reshape(-1) + 255, minlength=511))


@pytest.mark.parametrize("h,w", [(1, 1), (1, 9), (7, 1), (7, 9), (8, 8), (9, 17), (17, 9)])
def test_decode_inverts_encode_for_any_parameters(h, w):
    # M* depends only on (S, E, a, b), so any parameters give a lossless round trip
    rng = np.random.default_rng(h * 100 + w)
    rgbe = synth.tiny_rgbe(h, w, seed=h * w, zero_frac=0.1)
    m3, e = O.rgbe_split(rgbe)
    s3 = rng.integers(0, 256, size=(3, h, w)).astype(np.uint8)
    a = rng.uniform(-1, 1, size=(3, 256)).astype(np.float32)
    b = rng.uniform(-300, 300, size=(3, 256)).astype(np.float32)
    for gf_on in (True, False):
        ms = O.predict(O.gf(s3, gf_on), e, a, b)
        r3, _ = O.residual(m3, ms)
        assert np.array_equal(O.decode(s3, e, r3, a, b, gf_on), rgbe)
