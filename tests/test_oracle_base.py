"""Pins for the oracle's base-layer round trip (fixed-point 8x8 DCT,
quantise, dequantise, inverse DCT; the JPEG base layer of Sec. IV).

References: scipy's orthonormal DCT-II (an independent library routine),
float64 closed forms, and the IJG quality-scaling properties.
"""
import numpy as np
import pytest
from scipy.fft import dct, dctn, idctn

from oracle import oracle as O
from paper_2309_11072_gb300 import synth

lib = O.lib()
import ctypes  # noqa: E402


def _fdct(X):
    X = np.ascontiguousarray(X, dtype=np.int32).reshape(64)
    F = np.empty(64, dtype=np.int32)
    lib.oracle_fdct_block(O._p(X), O._p(F))
    return F.reshape(8, 8)


def _idct(F):
    F = np.ascontiguousarray(F, dtype=np.int32).reshape(64)
    X = np.empty(64, dtype=np.int32)
    lib.oracle_idct_block(O._p(F), O._p(X))
    return X.reshape(8, 8)


def _qdq(F, Q):
    F = np.ascontiguousarray(F, dtype=np.int32).reshape(64)
    Q = np.ascontiguousarray(Q, dtype=np.int32).reshape(64)
    out = np.empty(64, dtype=np.int32)
    lib.oracle_quant_dequant_block(O._p(F), O._p(Q), O._p(out))
    return out.reshape(8, 8)


def test_dct_constants_against_scipy():
    D = O.dct_matrix()
    ref = dct(np.eye(8), type=2, norm="ortho", axis=0) * 4096.0
    assert np.abs(D - ref).max() <= 0.5
    # near-orthogonality of the fixed-point matrix: D D^T ~ 2^24 I
    G = D.astype(np.int64) @ D.T.astype(np.int64)
    assert np.abs(G - (1 << 24) * np.eye(8)).max() < 2 * 4096 * 8 * 0.5


def test_forward_dct_within_one_of_float64():
    rng = np.random.default_rng(1)
    worst = 0
    for _ in range(300):
        X = rng.integers(-128, 128, size=(8, 8))
        F = _fdct(X)
        ref = dctn(X.astype(np.float64), type=2, norm="ortho")
        worst = max(worst, np.abs(F - ref).max())
    assert worst <= 1.0


def test_inverse_dct_within_one_of_float64():
    rng = np.random.default_rng(2)
    worst = 0
    for _ in range(300):
        F = rng.integers(-700, 700, size=(8, 8))
        F[0, 0] = rng.integers(-1024, 1024)
        X = _idct(F)
        ref = idctn(F.astype(np.float64), type=2, norm="ortho")
        worst = max(worst, np.abs(X - ref).max())
    assert worst <= 1.0


def test_dc_of_constant_block_and_zero_ac():
    for c in (-128, -37, 0, 5, 127):
        F = _fdct(np.full((8, 8), c))
        assert abs(F[0, 0] - 8 * c) <= 1
        F[0, 0] = 0
        assert (F == 0).all()


@pytest.mark.parametrize("quality", [1, 10, 25, 49, 50, 51, 75, 90, 99, 100])
def test_quant_table_ijg_rule(quality):
    Q = O.quant_table(quality)
    base = O.quant_table(50)
    assert Q.min() >= 1 and Q.max() <= 255
    if quality == 100:
        assert (Q == 1).all()
    # monotone: higher quality never has a coarser step
    if quality < 100:
        assert (O.quant_table(quality + 1) <= Q).all()
    # T.81 Annex K.1 luminance table at quality 50 (first row and DC)
    assert base[0].tolist() == [16, 11, 10, 16, 24, 40, 51, 61]
    assert base[7, 7] == 99


def test_quality_75_halves_the_table_rounding_halves_up():
    # the IJG rule scales the K.1 steps by 200 - 2Q percent, rounded to the
    # nearest integer with halves up: at Q = 75 that is b / 2, so the odd
    # steps of K.1 (11, 51, 61, ...) become (b + 1) / 2; at Q = 25 it is 2 b
    base = O.quant_table(50)
    assert (base % 2 == 1).sum() >= 10
    assert np.array_equal(O.quant_table(75), (base + 1) // 2)
    assert np.array_equal(O.quant_table(25), np.minimum(2 * base, 255))


def test_quantiser_half_away_from_zero():
    Q = np.full((8, 8), 10, dtype=np.int32)
    F = np.zeros((8, 8), dtype=np.int32)
    vals = [0, 4, 5, 6, 14, 15, 16, -4, -5, -6, -15, -16, 1000, -1000]
    F.flat[:len(vals)] = vals
    out = _qdq(F, Q).flat[:len(vals)]
    expect = [0, 0, 10, 10, 10, 20, 20, 0, -10, -10, -20, -20, 1000, -1000]
    assert list(out) == expect


def test_quality_100_nearly_lossless():
    sdr = np.random.default_rng(3).integers(0, 256, size=(3, 37, 45)).astype(np.uint8)
    s = O.base_roundtrip(sdr, 100)
    assert np.abs(s.astype(int) - sdr).max() <= 1


def test_constant_image_stays_constant():
    for val in (0, 17, 128, 255):
        sdr = np.full((3, 19, 21), val, dtype=np.uint8)
        for q in (10, 50, 90):
            s = O.base_roundtrip(sdr, q)
            assert (s == s[:, :1, :1]).all()
            assert np.abs(s.astype(int) - val).max() <= O.quant_table(q)[0, 0] // 16 + 1


def test_roundtrip_matches_float64_pipeline_where_unambiguous():
    """Integer levels equal the float64 levels wherever the float coefficient
    is more than one unit away from a decision boundary, and the output is
    within one grey level of the float64 inverse of those levels."""
    sdr = synth.make_rgbe(96, 128, seed=9, lo=-2, hi=4)
    st = O.lum_stats(sdr)
    J, r = O.key(st)
    planes = O.tmo(sdr, J, r)
    # coarse qualities: finer steps leave too few blocks far from every boundary
    # (the finer ones are covered by the composition test below)
    for quality in (25, 50):
        Q = O.quant_table(quality).astype(np.float64)
        s = O.base_roundtrip(planes, quality)
        checked = 0
        for c in range(3):
            for by in range(0, 96, 8):
                for bx in range(0, 128, 8):
                    X = planes[c, by:by + 8, bx:bx + 8].astype(np.float64) - 128
                    Ff = dctn(X, type=2, norm="ortho")
                    z = Ff / Q
                    dist = np.abs(np.abs(z) - np.floor(np.abs(z)) - 0.5) * Q
                    if dist.min() <= 1.0:
                        continue
                    lv = np.sign(z) * np.floor(np.abs(z) + 0.5)
                    rec = idctn(lv * Q, type=2, norm="ortho") + 128
                    got = s[c, by:by + 8, bx:bx + 8].astype(np.float64)
                    assert np.abs(got - np.clip(rec, 0, 255)).max() <= 1.0 + 1e-9
                    checked += 1
        assert checked >= 20


def test_roundtrip_is_composition_of_pinned_steps():
    rng = np.random.default_rng(6)
    sdr = rng.integers(0, 256, size=(3, 16, 24)).astype(np.uint8)
    for quality in (30, 85):
        Q = O.quant_table(quality)
        s = O.base_roundtrip(sdr, quality)
        for c in range(3):
            for by in range(0, 16, 8):
                for bx in range(0, 24, 8):
                    X = sdr[c, by:by + 8, bx:bx + 8].astype(np.int32) - 128
                    Y = _idct(_qdq(_fdct(X), Q)) + 128
                    assert np.array_equal(np.clip(Y, 0, 255), s[c, by:by + 8, bx:bx + 8])


def test_ragged_edges_replicate():
    # a ragged image equals the crop of the edge-replicated padded image
    rng = np.random.default_rng(4)
    sdr = rng.integers(0, 256, size=(3, 13, 19)).astype(np.uint8)
    pad = np.pad(sdr, ((0, 0), (0, 3), (0, 5)), mode="edge")
    assert np.array_equal(O.base_roundtrip(sdr, 75), O.base_roundtrip(pad, 75)[:, :13, :19])


def test_bad_quality_rejected():
    with pytest.raises(ValueError):
        O.base_roundtrip(np.zeros((3, 8, 8), np.uint8), 0)
    with pytest.raises(ValueError):
        O.base_roundtrip(np.zeros((3, 8, 8), np.uint8), 101)
