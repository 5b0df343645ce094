"""Whole-encoder pins for the oracle: the reversibility the paper claims
(Sec. I, III-C) and the rate ordering of Table I (SLRME lowers the rate of
the enhancement layer against coding M - S directly)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2309_11072_gb300 import synth
from paper_2309_11072_gb300.metrics import entropy_bits


@pytest.mark.parametrize("quality", [50, 90])
def test_small_workload_is_lossless(quality):
    img = synth.make_rgbe(384, 512, seed=1, lo=-2.0, hi=4.0)
    enc = O.encode(img, quality)
    assert np.array_equal(O.decode(enc["s3"], enc["e"], enc["r3"], enc["a"], enc["b"]), img)
    assert enc["hist"].sum(axis=1).tolist() == [img.size] * 3


def test_all_zero_and_single_exponent_images():
    z = np.zeros((9, 10), np.uint32)
    enc = O.encode(z, 75)
    assert (enc["sdr3"] == 0).all() and enc["n_used"] == 1 and (enc["r3"] == 0).all()
    one = synth.tiny_rgbe(16, 24, seed=2, const_e=131)
    enc = O.encode(one, 75)
    assert enc["n_used"] == 1
    assert np.array_equal(O.decode(enc["s3"], enc["e"], enc["r3"], enc["a"], enc["b"]), one)


def test_every_exponent_value_present():
    img = synth.tiny_rgbe(32, 32, seed=3, e_lo=0, e_hi=255)
    img.flat[:256] = (img.flat[:256] & 0x00FFFFFF) | (np.arange(256, dtype=np.uint32) << 24)
    enc = O.encode(img, 90)
    assert enc["n_used"] == 256
    assert np.array_equal(O.decode(enc["s3"], enc["e"], enc["r3"], enc["a"], enc["b"]), img)


def test_slrme_lowers_residual_entropy():
    # Table I: "with SLRME" < "w/o SLRME" on every image; here by order-0 entropy
    img = synth.make_rgbe(256, 320, seed=17, lo=-3.0, hi=5.0, rects=6, highlights=20)
    enc = O.encode(img, 85)
    h_slr = sum(entropy_bits(h) for h in enc["hist"])
    a = np.full((3, 256), 1 / 16, np.float32)
    b = np.zeros((3, 256), np.float32)
    ms = O.predict(O.gf(enc["s3"], False), enc["e"], a, b)
    assert np.array_equal(ms, enc["s3"])            # w/o SLRME: M* = S exactly
    _, hist_plain = O.residual(enc["m3"], ms)
    h_plain = sum(entropy_bits(h) for h in hist_plain)
    assert h_slr < h_plain


def test_oracle_matches_committed_golden():
    """Regression pin: the oracle still produces the values its generator
    script wrote (tests/golden/make_golden.py, oracle only)."""
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "tiny_codec_q75.json")
    g = json.load(open(path))
    img = np.array(g["rgbe"], np.uint32).reshape(g["h"], g["w"])
    enc = O.encode(img, g["quality"], bool(g["gf_on"]))
    used = np.nonzero(enc["n"])[0]
    assert enc["stats"].tolist() == g["stats"] and (enc["J"], enc["r"]) == (g["J"], g["r"])
    assert enc["sdr3"].reshape(-1).tolist() == g["sdr3"]
    assert enc["s3"].reshape(-1).tolist() == g["s3"]
    assert used.tolist() == g["used"]
    assert enc["sums"][used].tolist() == g["sums_used"]
    assert enc["a"][:, used].view(np.uint32).reshape(-1).tolist() == g["a_bits"]
    assert enc["b"][:, used].view(np.uint32).reshape(-1).tolist() == g["b_bits"]
    assert enc["r3"].reshape(-1).tolist() == g["r3"]


def test_chunked_oracle_equals_the_whole_image_oracle():
    """The chunk-by-chunk run of the oracle (used at 800 M pixels on the GPU)
    gives the whole-image oracle's parameters, histograms, S, x = 16 S* and
    residuals, on 8- and 16-row images with a ragged right edge."""
    import chunked_oracle as K
    from paper_2309_11072_gb300 import synth
    old = K.CHUNK
    K.CHUNK = 64
    try:
        for h, w in [(16, 300), (8, 412), (8, 64)]:
            img = synth.make_rgbe(h, w, seed=9, lo=-3.0, hi=5.0, rects=2, highlights=5)
            J, r = O.key(O.lum_stats(img))
            a, b, cnt, nu = O.solve(K.oracle_sums(img, J, r))
            o = O.encode(img, K.Q)
            assert np.array_equal(a.view(np.uint32), o["a"].view(np.uint32))
            assert np.array_equal(b.view(np.uint32), o["b"].view(np.uint32))
            assert np.array_equal(cnt, o["n"]) and nu == o["n_used"]
            assert np.array_equal(K.oracle_hist(img, J, r, a, b), o["hist"].astype(np.int64))
            for x0, x1 in ((0, 64), (64, 128), ((w - 40) // 8 * 8, w)):
                so, xo, mo, eo = K.oracle_chunk(img, x0, x1, J, r)
                assert np.array_equal(so, o["s3"][:, :, x0:x1]) and np.array_equal(xo, o["x3"][:, :, x0:x1])
                ro, _ = O.residual(mo, O.predict(xo, eo, a, b))
                assert np.array_equal(ro, o["r3"][:, :, x0:x1])
    finally:
        K.CHUNK = old
