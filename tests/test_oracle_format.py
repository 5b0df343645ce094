"""Pins for the oracle's Radiance-format functions (Sec. II-A, Eqs. 1-3).

Each check is against exact rational arithmetic or a format invariant,
not against a retyped copy of the oracle's formula.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_2309_11072_gb300 import synth


def _exp_interval_ok(v: Fraction, E: int) -> bool:
    # Eq. (1) read with frexp: 2^(E-129) <= max f < 2^(E-128)
    return Fraction(2) ** (E - 129) <= v < Fraction(2) ** (E - 128)


def test_forward_matches_eq1_eq2_exactly():
    rng = np.random.default_rng(7)
    f = np.exp(rng.uniform(-40, 40, size=(400, 3)))
    words = O.rgbe_from_float(f)
    for p in range(f.shape[0]):
        wd = int(words[p])
        E = wd >> 24
        M = [(wd >> (8 * c)) & 255 for c in range(3)]
        fr = [Fraction(float(x)) for x in f[p]]
        v = max(fr)
        assert _exp_interval_ok(v, E)
        # Eq. (1) with the ceiling agrees away from exact powers of two
        if v.numerator & (v.numerator - 1) or v.denominator & (v.denominator - 1):
            lg_lo = Fraction(2) ** (E - 129)
            assert lg_lo < v  # so ceil(log2 v + 128) == E
        # Eq. (2): M = floor(256 f / 2^(E-128)), exactly
        for c in range(3):
            assert M[c] == (fr[c] * 256 / Fraction(2) ** (E - 128)).__floor__()
        assert 128 <= max(M) <= 255


def test_power_of_two_reading():
    # Eq. (1) literally gives M = 256 at v = 2^k; the reading gives M = 128, E = k + 129
    f = np.array([[1.0, 0.5, 0.25], [2.0 ** -20, 0.0, 0.0]])
    w = O.rgbe_from_float(f)
    assert int(w[0]) >> 24 == 129 and int(w[0]) & 255 == 128
    assert int(w[1]) >> 24 == 109 and int(w[1]) & 255 == 128


def test_zero_and_out_of_range():
    assert O.rgbe_from_float(np.zeros((1, 3)))[0] == 0
    assert O.rgbe_from_float(np.full((1, 3), 1e-33))[0] == 0
    with pytest.raises(ValueError):
        O.rgbe_from_float(np.full((1, 3), 2.0 ** 130))


def test_inverse_eq3_is_interval_midpoint_and_roundtrips():
    words = synth.tiny_rgbe(37, 41, seed=3, e_lo=23, e_hi=255)   # 2^(E-129) >= 1e-32
    f = O.rgbe_to_float(words)
    for p in range(0, words.size, 7):
        wd = int(words.flat[p])
        E = wd >> 24
        for c in range(3):
            M = (wd >> (8 * c)) & 255
            lo = Fraction(M) * Fraction(2) ** (E - 136)
            hi = Fraction(M + 1) * Fraction(2) ** (E - 136)
            assert Fraction(float(f.reshape(-1, 3)[p, c])) == (lo + hi) / 2
    # reversibility of the converter pair for normalised words (Sec. II-A)
    back = O.rgbe_from_float(f.reshape(-1, 3)).reshape(words.shape)
    assert np.array_equal(back, words)


def test_zero_exponent_decodes_to_zero():
    f = O.rgbe_to_float(np.array([0x00FFFFFF, 0], dtype=np.uint32))
    assert (f == 0).all()


def test_generator_packing_agrees_with_eq1_eq2():
    rgb = synth.hdr_image(64, 96, seed=11, lo=-3, hi=5, rects=3, highlights=5)
    assert np.array_equal(synth.pack_radiance(rgb), O.rgbe_from_float(rgb.reshape(-1, 3)).reshape(64, 96))


def test_split_recombines():
    words = synth.tiny_rgbe(13, 17, seed=5, zero_frac=0.2)
    m3, e = O.rgbe_split(words)
    rebuilt = (m3[0].astype(np.uint32) | (m3[1].astype(np.uint32) << 8)
               | (m3[2].astype(np.uint32) << 16) | (e.astype(np.uint32) << 24))
    assert np.array_equal(rebuilt, words)


def test_workload_exponent_ranges():
    # the 8-decade sky workload is scaled so every exponent lies in [100, 150]
    img = synth.make_rgbe(270, 480, seed=3, lo=-3.0, hi=5.0, sky=True)
    e = img >> 24
    assert e.min() >= 100 and e.max() <= 150
