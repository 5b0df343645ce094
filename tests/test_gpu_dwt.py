"""GPU parity of the reversible 5/3 wavelet and of the segment form of the
rANS coder against the oracle: coefficients and per-band histograms bit for
bit, the inverse, tables per band, packed words and counts per chunk, raw
chunks for values beyond the alphabet, and the whole enhancement-layer
chain (residuals -> wavelet -> tables -> bitstream -> residuals) on the
codec's own output."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2309_11072_gb300 import codec, native, synth

pytestmark = pytest.mark.gpu

NRES = 511


def _dev(a: np.ndarray, dtype=None) -> torch.Tensor:
    a = np.ascontiguousarray(a)
    return torch.from_numpy(a.copy()).cuda()


def _gpu_forward(x: np.ndarray, levels: int, hist: bool = True):
    P, h, w = x.shape
    planes = _dev(x.astype(np.int16))
    coef = torch.full((P * h * w,), 0x5A5A, dtype=torch.int16, device="cuda")
    nb = 1 + 3 * levels
    hh = torch.full((P * nb * NRES,), -1, dtype=torch.int32, device="cuda") if hist else None
    ws = torch.empty(max(native.dwt53_workspace_bytes(P, h, w), 256), dtype=torch.uint8, device="cuda")
    native.dwt53_forward(planes, P, h, w, levels, coef, hh, ws)
    torch.cuda.synchronize()
    c = coef.cpu().numpy().reshape(P, h * w)
    return c, (hh.cpu().numpy().view(np.uint32).reshape(P * nb, NRES) if hist else None)


def _gpu_inverse(coef: np.ndarray, P: int, h: int, w: int, levels: int) -> np.ndarray:
    c = _dev(coef.astype(np.int16).reshape(-1))
    out = torch.full((P * h * w,), 0x7777, dtype=torch.int16, device="cuda")
    ws = torch.empty(max(native.dwt53_workspace_bytes(P, h, w), 256), dtype=torch.uint8, device="cuda")
    native.dwt53_inverse(c, P, h, w, levels, out, ws)
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(P, h, w)


def _seg_lengths(h, w, levels, P):
    return [a * b for a, b in O.dwt53_bands(h, w, levels)] * P


@pytest.mark.parametrize("h,w", [(1, 1), (1, 7), (7, 1), (2, 2), (3, 5), (16, 16), (33, 65), (100, 37), (257, 130)])
@pytest.mark.parametrize("levels", [1, 2, 3])
def test_wavelet_bit_exact(h, w, levels):
    x = np.random.default_rng(h * 1000 + w + levels).integers(-255, 256, size=(3, h, w)).astype(np.int16)
    c, hist = _gpu_forward(x, levels)
    oc = O.dwt53_forward(x, levels)
    assert np.array_equal(c, oc)
    assert np.array_equal(hist, O.segment_hist(oc.reshape(-1), _seg_lengths(h, w, levels, 3)))
    assert np.array_equal(_gpu_inverse(oc, 3, h, w, levels), x)


def test_wavelet_of_extreme_values_and_without_histograms():
    h, w = 64, 96
    yy, xx = np.mgrid[0:h, 0:w]
    x = np.stack([np.where((yy + xx) % 2 == 0, 255, -255), np.full((h, w), -255), (xx * 5 - 240) % 511 - 255])
    x = x.astype(np.int16)
    c, _ = _gpu_forward(x, 3, hist=False)
    oc = O.dwt53_forward(x, 3)
    assert np.array_equal(c, oc) and np.abs(oc).max() > 255
    assert np.array_equal(_gpu_inverse(c, 3, h, w, 3), x)


def _gpu_segments(sym: np.ndarray, lengths, freq: np.ndarray):
    s = _dev(sym.astype(np.int16).reshape(-1))
    f = _dev(np.ascontiguousarray(freq, np.uint32).view(np.int32).reshape(-1))
    nw, nc = native.rans_segments_capacity(lengths)
    words = torch.full((max(nw, 8),), 0x5A5A, dtype=torch.int16, device="cuda")
    counts = torch.full((max(nc, 1),), -7, dtype=torch.int32, device="cuda")
    native.rans_encode_segments(s, lengths, f, words, counts)
    back = torch.full_like(s, 0x7777)
    native.rans_decode_segments(words, counts, lengths, f, back)
    torch.cuda.synchronize()
    return (words.cpu().numpy().view(np.uint16)[:nw], counts.cpu().numpy().view(np.uint32)[:nc],
            back.cpu().numpy())


def _blocks_equal(words, counts, ow, oc, lengths):
    """Every chunk's used words (packed streams, or a raw chunk's values) are the oracle's."""
    assert np.array_equal(counts, oc)
    chunks, _, _ = O.rans_segment_layout(lengths)
    b = 0
    for g, n in enumerate(lengths):
        for k in range(chunks[g]):
            m = min(8192, int(n) - 8192 * k)
            cnt = oc[32 * b:32 * (b + 1)]
            used = m if cnt[0] == O.RANS_RAW else int(cnt.astype(np.int64).sum())
            blk = slice(b * 32 * 258, b * 32 * 258 + used)
            assert np.array_equal(words[blk], ow[blk]), (g, k)
            b += 1


def test_segment_coder_bit_exact_with_raw_chunks():
    lengths = [1, 8192, 8193, 0, 31, 30000, 5000]
    rng = np.random.default_rng(17)
    parts = [np.clip(np.round(rng.laplace(0, s, size=n)), -255, 255)
             for n, s in zip(lengths, [1, 2, 9, 3, 40, 0.7, 5])]
    v = np.concatenate(parts).astype(np.int16)
    v[8192 + 1 + 100] = 400              # segment 2, chunk 0: raw
    v[-1] = -9000                        # segment 6: raw
    hist = O.segment_hist(v, lengths)
    h_dev = _dev(hist.view(np.int32).reshape(-1))
    f_dev = torch.empty(len(lengths) * NRES, dtype=torch.int32, device="cuda")
    native.device_status(clear=True)
    native.rans_tables_n(h_dev, len(lengths), f_dev)
    torch.cuda.synchronize()
    freq = f_dev.cpu().numpy().view(np.uint32).reshape(len(lengths), NRES)
    assert np.array_equal(freq, np.stack([O.rans_table(h) for h in hist]))
    words, counts, back = _gpu_segments(v, lengths, freq)
    ow, oc = O.rans_encode_segments(v, lengths, freq)
    _blocks_equal(words, counts, ow, oc, lengths)
    assert np.array_equal(back, v)
    assert np.array_equal(O.rans_decode_segments(words, counts, lengths, freq), v)
    assert native.device_status(clear=True) == 0


def test_segment_all_values_beyond_the_alphabet():
    # a segment whose every value is out of range has an empty table: all its chunks are raw
    lengths = [9000, 100]
    v = np.concatenate([np.full(9000, 1000), np.arange(100) - 50]).astype(np.int16)
    freq = np.stack([O.rans_table(h) for h in O.segment_hist(v, lengths)])
    assert freq[0].sum() == 0
    native.device_status(clear=True)
    words, counts, back = _gpu_segments(v, lengths, freq)
    ow, oc = O.rans_encode_segments(v, lengths, freq)
    _blocks_equal(words, counts, ow, oc, lengths)
    assert np.array_equal(back, v)
    assert native.device_status(clear=True) == 0


@pytest.mark.parametrize("h,w,q", [(96, 160, 75), (1536, 2048, 50)])
def test_enhancement_layer_chain(h, w, q):
    """Residuals of the codec -> 3-level wavelet (GPU) -> per-band tables ->
    bitstream, equal to the oracle's at every step, decoded back to the
    residuals and on to the RGBE words; at 2048x1536, fewer bits than coding
    the residuals directly."""
    levels = 3
    img = synth.make_rgbe(h, w, seed=h + w + q, lo=-3.0, hi=5.0, rects=6)
    c = codec.Codec(h, w, "cuda")
    L = c.encode(torch.from_numpy(img.view(np.int32).reshape(-1).copy()).cuda(), q)
    n = h * w
    nb = 1 + 3 * levels
    coef = torch.empty(3 * n, dtype=torch.int16, device="cuda")
    hist = torch.empty(3 * nb * NRES, dtype=torch.int32, device="cuda")
    ws = torch.empty(native.dwt53_workspace_bytes(3, h, w), dtype=torch.uint8, device="cuda")
    freq = torch.empty(3 * nb * NRES, dtype=torch.int32, device="cuda")
    lengths = _seg_lengths(h, w, levels, 3)
    nw, nc = native.rans_segments_capacity(lengths)
    words = torch.empty(nw, dtype=torch.int16, device="cuda")
    counts = torch.empty(nc, dtype=torch.int32, device="cuda")
    coef_back = torch.empty_like(coef)
    r_back = torch.empty_like(L.r3)
    native.device_status(clear=True)
    native.dwt53_forward(L.r3, 3, h, w, levels, coef, hist, ws)
    native.rans_tables_n(hist, 3 * nb, freq)
    native.rans_encode_segments(coef, lengths, freq, words, counts)
    native.rans_decode_segments(words, counts, lengths, freq, coef_back)
    native.dwt53_inverse(coef_back, 3, h, w, levels, r_back, ws)
    out = c.decode(L.s3, L.e, r_back, L.params)
    torch.cuda.synchronize()
    assert native.device_status(clear=True) == 0
    assert np.array_equal(out.cpu().numpy().view(np.uint32).reshape(h, w), img)
    r3 = L.r3.cpu().numpy().reshape(3, h, w)
    oc = O.dwt53_forward(r3, levels)
    assert np.array_equal(coef.cpu().numpy().reshape(3, n), oc)
    ohist = O.segment_hist(oc.reshape(-1), lengths)
    assert np.array_equal(hist.cpu().numpy().view(np.uint32).reshape(-1, NRES), ohist)
    ofreq = np.stack([O.rans_table(x) for x in ohist])
    assert np.array_equal(freq.cpu().numpy().view(np.uint32).reshape(-1, NRES), ofreq)
    ow, ocnt = O.rans_encode_segments(oc.reshape(-1), lengths, ofreq)
    _blocks_equal(words.cpu().numpy().view(np.uint16), counts.cpu().numpy().view(np.uint32), ow, ocnt, lengths)
    if n < 1 << 20:
        return   # below about a megapixel the 30 bands' stream overhead (32 final states each) dominates
    # the wavelet stage codes the residuals in fewer bits than the plain coder
    plain_f = np.stack([O.rans_table(x) for x in O.segment_hist(r3.reshape(-1), [n] * 3)])
    _, pc = O.rans_encode(r3.reshape(-1), plain_f)
    raw = ocnt == O.RANS_RAW
    bits_dwt = 16.0 * ocnt[~raw].astype(np.int64).sum() + 16.0 * 8192 * raw.sum() / 32
    assert bits_dwt < 16.0 * pc.astype(np.int64).sum()
