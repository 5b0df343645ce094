"""Pins for the oracle's tone-mapping operator (the base-layer TMO).

The TMO's constants are readings (Reinhard global operator, key 0.18,
BT.709 weights, gamma 2.2); these tests pin the oracle's implementation to
arbitrary-precision values of those definitions, to a float64 textbook
Reinhard operator, and to exact invariants (exposure, gray, zero).
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_2309_11072_gb300 import synth


def test_log2_table_against_arbitrary_precision():
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 120
    lut = O.log2_table()
    for i in range(0, 2048, 3):
        exact = 65536 * mp.log(2048 + i, 2)
        assert abs(exact - int(lut[i])) <= 0.5 + 1e-20


def test_gamma_thresholds_against_arbitrary_precision():
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 120
    t = O.gamma_thresholds()
    assert t[0] == 0
    assert (np.diff(t[1:]) > 0).all()
    for k in range(1, 256):
        exact = mp.power((k - mp.mpf(1) / 2) / 255, mp.mpf(22) / 10)
        # float32 rounding of the exact value: within half an ulp
        ulp = np.spacing(np.float32(t[k]))
        assert abs(exact - mp.mpf(float(t[k]))) <= mp.mpf(float(ulp)) / 2 * (1 + 1e-9)


def test_key_tables_against_arbitrary_precision():
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 120
    kr, wr = O.key_tables()
    for r in range(16):
        for val, base in ((kr[r], mp.mpf("0.18")), (wr[r], mp.mpf(1800))):
            exact = base * mp.power(2, -mp.mpf(r) / 16)
            ulp = np.spacing(np.float32(val))
            assert abs(exact - mp.mpf(float(val))) <= mp.mpf(float(ulp)) / 2 * (1 + 1e-9)


def _log2_lum_exact(words):
    # log2 of 10^4 * Y with Y the BT.709 luminance of the Eq. (3) floats
    f = O.rgbe_to_float(words.reshape(-1))
    y = 0.2126 * f[:, 0] + 0.7152 * f[:, 1] + 0.0722 * f[:, 2]
    nz = (words.reshape(-1) >> 24) > 0
    return np.log2(1e4 * y[nz]), int(nz.sum())


def test_log_average_statistic_within_quantisation_bound():
    img = synth.make_rgbe(96, 128, seed=21, lo=-3, hi=5, highlights=10)
    st = O.lum_stats(img)
    ref, n = _log2_lum_exact(img)
    assert st[1] == n
    # per pixel: Yq truncated to 12 significant bits (< log2(1 + 2^-11)) and a
    # table rounded to 1/65536; the truncation only lowers the estimate
    err = st[0] / 65536.0 - ref.sum()
    assert -n * (np.log2(1 + 2.0 ** -11) + 0.5 / 65536) - 1e-6 <= err <= n * 0.5 / 65536 + 1e-6


def test_log_average_shifts_exactly_with_exposure():
    img = synth.tiny_rgbe(20, 30, seed=4, e_lo=110, e_hi=140, zero_frac=0.1)
    st0 = O.lum_stats(img)
    for k in (-7, 3, 11):
        e = (img >> 24).astype(np.int64)
        shifted = np.where(e > 0, img.astype(np.int64) + (k << 24), img).astype(np.uint32)
        st = O.lum_stats(shifted)
        assert st[1] == st0[1]
        assert st[0] == st0[0] + 65536 * k * st0[1]


@pytest.mark.parametrize("num,n", [(0, 5), (1, 1), (-1, 1), (2047, 1), (2048, 1), (-2048, 1), (-2049, 1),
                                   (123456789, 77), (-987654321, 1234), (4096 * 16 * 5 - 1, 1)])
def test_key_is_round_half_up_of_16_mu(num, n):
    J, r = O.key(np.array([num, n], dtype=np.int64))
    j = 16 * J + r
    assert 0 <= r < 16
    sixteen_mu = Fraction(num, 4096 * n)   # 16 * num / (65536 n)
    assert j - Fraction(1, 2) <= sixteen_mu < j + Fraction(1, 2)


def test_key_of_empty_image():
    assert O.key(np.array([0, 0], dtype=np.int64)) == (0, 0)


def _tmo_image(img):
    st = O.lum_stats(img)
    J, r = O.key(st)
    return O.tmo(img, J, r), J, r


def test_tmo_zero_exponent_gives_black():
    img = synth.tiny_rgbe(9, 11, seed=8, zero_frac=0.3)
    sdr, _, _ = _tmo_image(img)
    z = (img >> 24) == 0
    assert z.any() and (sdr[:, z] == 0).all()


def test_tmo_exposure_invariance():
    # Reinhard's key normalisation: scaling the radiance by 2^k leaves the SDRI unchanged
    img = synth.make_rgbe(48, 64, seed=5, lo=-2, hi=4)
    sdr0, J0, _ = _tmo_image(img)
    for k in (-9, 5):
        shifted = (img.astype(np.int64) + (k << 24)).astype(np.uint32)
        sdr, J, _ = _tmo_image(shifted)
        assert J == J0 + k
        assert np.array_equal(sdr, sdr0)


def test_tmo_gray_is_gray_and_monotone():
    M = np.arange(256, dtype=np.uint32)
    img = (M | (M << 8) | (M << 16) | (np.uint32(130) << 24)).reshape(1, 256)
    sdr = O.tmo(img, J=-7, r=5)
    assert np.array_equal(sdr[0], sdr[1]) and np.array_equal(sdr[1], sdr[2])
    assert (np.diff(sdr[0, 0].astype(int)) >= 0).all()


def test_tmo_close_to_float64_reinhard():
    img = synth.make_rgbe(64, 80, seed=13, lo=-3, hi=5, rects=4, highlights=6)
    sdr, J, r = _tmo_image(img)
    f = O.rgbe_to_float(img.reshape(-1))
    y = 0.2126 * f[:, 0] + 0.7152 * f[:, 1] + 0.0722 * f[:, 2]
    lav = 2.0 ** ((16 * J + r) / 16.0) / 1e4         # log-average the key uses
    nz = y > 0
    L = np.where(nz, 0.18 * y / lav, 0.0)
    Ld = L / (1 + L)
    ref = np.zeros((3, f.shape[0]))
    for c in range(3):
        v = np.where(nz, Ld * f[:, c] / np.where(nz, y, 1), 0.0)
        ref[c] = np.clip(np.floor(255 * np.power(v, 1 / 2.2) + 0.5), 0, 255)
    diff = np.abs(sdr.reshape(3, -1).astype(int) - ref)
    assert diff.max() <= 1
    assert (diff == 0).mean() > 0.99


def test_white_point_operator_without_a_white_point_is_the_plain_operator():
    img = synth.make_rgbe(40, 56, seed=21, lo=-3, hi=5, rects=3, highlights=4)
    sdr, J, r = _tmo_image(img)
    assert np.array_equal(O.tmo_white(img, J, r, np.inf), sdr)


def test_white_point_operator_close_to_float64_reinhard_eq4_and_brighter():
    img = synth.make_rgbe(64, 80, seed=13, lo=-3, hi=5, rects=4, highlights=6)
    sdr, J, r = _tmo_image(img)
    lw = O.white_point(img, J, r)
    f = O.rgbe_to_float(img.reshape(-1))
    y = 0.2126 * f[:, 0] + 0.7152 * f[:, 1] + 0.0722 * f[:, 2]
    lav = 2.0 ** ((16 * J + r) / 16.0) / 1e4
    nz = y > 0
    L = np.where(nz, 0.18 * y / lav, 0.0)
    # the white point is the largest scaled luminance (to float32 rounding of the operator's L)
    assert abs(float(lw) / L.max() - 1.0) < 1e-4
    Ld = L * (1 + L / L.max() ** 2) / (1 + L)
    assert abs(Ld.max() - 1.0) < 1e-12                # the brightest pixel maps to white
    ref = np.zeros((3, f.shape[0]))
    for c in range(3):
        v = np.where(nz, Ld * f[:, c] / np.where(nz, y, 1), 0.0)
        ref[c] = np.clip(np.floor(255 * np.power(v, 1 / 2.2) + 0.5), 0, 255)
    got = O.tmo_white(img, J, r, lw)
    diff = np.abs(got.reshape(3, -1).astype(int) - ref)
    assert diff.max() <= 1
    assert (diff == 0).mean() > 0.99
    assert (got >= sdr).all() and (got > sdr).any()   # the factor 1 + L / L_white^2 only brightens


def test_tmo_equals_the_exact_operator_away_from_the_thresholds():
    """The display code is the number of gamma thresholds ((k - 1/2) / 255)^2.2
    at or below the exact Reinhard value L_d f_c / Y, with f_c the Eq. (3)
    floats, Y their BT.709 luminance, L = 0.18 Y over the log-average
    2^((16 J + r) / 16) / 10^4 the key stands for, and L_d = L / (1 + L).
    The float32 evaluation and the float32 tables move the value by a few
    ulps (below 2^-21 relative), so wherever the exact value is farther than
    2^-19 from every threshold the codes are equal."""
    import bisect
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 80
    img = synth.make_rgbe(36, 44, seed=31, lo=-3, hi=5, rects=3, highlights=4)
    sdr, J, r = _tmo_image(img)
    thr = [mp.power((k - mp.mpf(1) / 2) / 255, mp.mpf(22) / 10) for k in range(1, 256)]
    lavg = mp.power(2, mp.mpf(16 * J + r) / 16) / 10 ** 4
    checked = 0
    words = img.reshape(-1)
    for p, wd in enumerate(words.tolist()):
        E = wd >> 24
        if E == 0:
            continue
        f = [(mp.mpf((wd >> (8 * c)) & 255) + mp.mpf(1) / 2) * mp.power(2, E - 136) for c in range(3)]
        Y = mp.mpf("0.2126") * f[0] + mp.mpf("0.7152") * f[1] + mp.mpf("0.0722") * f[2]
        L = mp.mpf("0.18") * Y / lavg
        Ld = L / (1 + L)
        for c in range(3):
            v = Ld * f[c] / Y
            k = bisect.bisect_right(thr, v)          # thresholds at or below v
            near = min(abs(v - thr[i]) / thr[i] for i in (k - 1, k) if 0 <= i < 255)
            if near < mp.mpf(2) ** -19:
                continue
            assert int(sdr.reshape(3, -1)[c, p]) == k, (p, c)
            checked += 1
    assert checked >= 0.99 * 3 * int(((words >> 24) > 0).sum())
