"""Pins of the oracle's reversible 5/3 wavelet (JPEG 2000's lossless
transform, which Sec. IV uses for the enhancement layer) and of the segment
form of its rANS coder, against what the mathematics fixes rather than
against the oracle itself:
- the lifting steps approximate the linear 5/3 analysis filter bank,
  (-1, 2, 6, 2, -1) / 8 and (-1, 2, -1) / 2 with whole-sample symmetric
  extension, as computed by scipy, to within their rounding: high-pass
  within 1/2, low-pass within 3/4, and within 9/4 after a 2-D level;
- perfect reconstruction for every size and level count;
- closed forms: a constant plane has only its low-low band (equal to the
  constant), a ramp along the rows has no row high-pass inside the plane;
- the band sizes tile the plane, and the largest magnitude stays within
  the 2x-per-pass bound;
- raw chunks: a chunk holding a value beyond +-255 is stored verbatim."""
import numpy as np
import pytest
from scipy.ndimage import convolve1d

from oracle import oracle as O

H0 = np.array([-1, 2, 6, 2, -1], np.float64) / 8.0
H1 = np.array([-1, 2, -1], np.float64) / 2.0


def _rand(shape, seed, lo=-255, hi=255):
    return np.random.default_rng(seed).integers(lo, hi + 1, size=shape).astype(np.int16)


def _bands(coef_plane, h, w, levels):
    out, at = [], 0
    for bh, bw in O.dwt53_bands(h, w, levels):
        out.append(coef_plane[at:at + bh * bw].reshape(bh, bw))
        at += bh * bw
    assert at == h * w
    return out


@pytest.mark.parametrize("w", [2, 3, 4, 9, 64, 101])
def test_one_dimensional_level_matches_the_linear_filter_bank(w):
    x = _rand((1, 1, w), seed=w)
    c = O.dwt53_forward(x, 1)[0]
    ll, hl, lh, hh = _bands(c, 1, w, 1)
    xf = x[0, 0].astype(np.float64)
    lo = convolve1d(xf, H0, mode="mirror")[0::2]
    hi = convolve1d(xf, H1, mode="mirror")[1::2]
    assert lh.size == 0 and hh.size == 0
    assert np.abs(hl[0] - hi).max() <= 0.5
    assert np.abs(ll[0] - lo).max() <= 0.75
    # the rounding rules themselves: the prediction is floored, so the
    # high-pass value is the exact one or up to 1/2 above it; the update adds
    # (d_l + d_r) / 4 rounded half up, i.e. 1/4 below to 1/2 above it
    d = hl[0].astype(np.float64)
    assert ((d - hi) >= 0).all() and ((d - hi) <= 0.5).all()
    dl = np.concatenate([d[:1], d])[:ll.shape[1]]
    dr = np.concatenate([d, d[-1:]])[:ll.shape[1]]
    upd = ll[0] - (xf[0::2] + (dl + dr) / 4.0)
    assert (upd >= -0.25).all() and (upd <= 0.5).all()


@pytest.mark.parametrize("h,w", [(8, 8), (9, 13), (32, 17)])
def test_two_dimensional_level_matches_the_separable_filter_bank(h, w):
    x = _rand((1, h, w), seed=h * w)
    c = O.dwt53_forward(x, 1)[0]
    ll, hl, lh, hh = _bands(c, h, w, 1)
    xf = x[0].astype(np.float64)
    rl = convolve1d(xf, H0, axis=1, mode="mirror")[:, 0::2]
    rh = convolve1d(xf, H1, axis=1, mode="mirror")[:, 1::2]
    lin = {"ll": convolve1d(rl, H0, axis=0, mode="mirror")[0::2],
           "hl": convolve1d(rh, H0, axis=0, mode="mirror")[0::2],
           "lh": convolve1d(rl, H1, axis=0, mode="mirror")[1::2],
           "hh": convolve1d(rh, H1, axis=0, mode="mirror")[1::2]}
    for name, band in (("ll", ll), ("hl", hl), ("lh", lh), ("hh", hh)):
        assert band.shape == lin[name].shape, name
        assert np.abs(band - lin[name]).max() <= 2.25, name


@pytest.mark.parametrize("h,w", [(1, 1), (1, 7), (7, 1), (2, 2), (3, 5), (16, 16), (33, 65), (100, 37)])
@pytest.mark.parametrize("levels", [0, 1, 2, 3])
def test_perfect_reconstruction(h, w, levels):
    x = _rand((3, h, w), seed=h + 100 * w + levels)
    c = O.dwt53_forward(x, levels)
    assert np.array_equal(O.dwt53_inverse(c, h, w, levels), x)


def test_extreme_values_stay_within_the_growth_bound():
    h, w = 64, 64
    yy, xx = np.mgrid[0:h, 0:w]
    x = np.where((yy + xx) % 2 == 0, 255, -255).astype(np.int16)[None]      # a checkerboard: the worst case
    c = O.dwt53_forward(x, 3)
    assert np.abs(c).max() <= 255 * 64
    assert np.array_equal(O.dwt53_inverse(c, h, w, 3), x)


def test_constant_plane_has_only_its_low_low_band():
    h, w = 23, 41
    x = np.full((1, h, w), -37, np.int16)
    bands = _bands(O.dwt53_forward(x, 3)[0], h, w, 3)
    assert (bands[0] == -37).all()
    for b in bands[1:]:
        assert (b == 0).all()


def test_ramp_along_rows_has_no_interior_row_high_pass():
    h, w = 6, 40
    x = np.tile((np.arange(w) * 3 - 60).astype(np.int16), (h, 1))[None]
    ll, hl, lh, hh = _bands(O.dwt53_forward(x, 1)[0], h, w, 1)
    # a linear signal is predicted exactly from its even neighbours: only the
    # last high-pass value, whose right neighbour is mirrored, can differ
    assert (hl[:, :-1] == 0).all()
    assert (lh == 0).all() and (hh[:, :-1] == 0).all()


def test_band_sizes_tile_the_plane():
    for h, w in [(1, 1), (5, 3), (1536, 2048), (4320, 7680), (17, 1)]:
        dims = O.dwt53_bands(h, w, 3)
        assert len(dims) == 10
        assert sum(a * b for a, b in dims) == h * w


def test_raw_chunks_store_values_beyond_the_alphabet_verbatim():
    lengths = [20000, 5000]
    v = _rand(sum(lengths), seed=5, lo=-40, hi=40)
    v[3] = 300                     # segment 0, chunk 0
    v[20000 + 4999] = -16000       # segment 1, its only chunk
    freq = np.stack([O.rans_table(h) for h in O.segment_hist(v, lengths)])
    words, counts = O.rans_encode_segments(v, lengths, freq)
    chunks, _, _ = O.rans_segment_layout(lengths)
    assert chunks == [3, 1]
    cnt = counts.reshape(-1, 32)
    blocks = words.reshape(-1, 32 * 258)
    assert (cnt[0] == O.RANS_RAW).all() and (cnt[3] == O.RANS_RAW).all()
    assert (cnt[1] != O.RANS_RAW).all() and (cnt[2] != O.RANS_RAW).all()
    assert np.array_equal(blocks[0, :8192].view(np.int16), v[:8192])
    assert np.array_equal(blocks[3, :5000].view(np.int16), v[20000:])
    assert np.array_equal(O.rans_decode_segments(words, counts, lengths, freq), v)


def test_segments_with_their_own_tables_round_trip():
    lengths = [1, 8192, 8193, 0, 31, 30000]
    rng = np.random.default_rng(9)
    parts = [np.clip(np.round(rng.laplace(0, s, size=n)), -255, 255) for n, s in zip(lengths, [1, 2, 9, 3, 40, 0.7])]
    v = np.concatenate(parts).astype(np.int16)
    hist = O.segment_hist(v, lengths)
    freq = np.stack([O.rans_table(h) for h in hist])
    words, counts = O.rans_encode_segments(v, lengths, freq)
    assert np.array_equal(O.rans_decode_segments(words, counts, lengths, freq), v)
    # the three-plane coder is the segment coder over three equal segments
    n = 9000
    r3 = np.clip(np.round(rng.laplace(0, 4, size=3 * n)), -255, 255).astype(np.int16)
    f3 = np.stack([O.rans_table(h) for h in O.segment_hist(r3, [n] * 3)])
    w1, c1 = O.rans_encode(r3, f3)
    w2, c2 = O.rans_encode_segments(r3, [n] * 3, f3)
    assert np.array_equal(w1, w2) and np.array_equal(c1, c2)
