"""GPU parity of the base-layer entropy coding against the oracle: the
quantised levels the base kernel writes, bit for bit, and the JPEG baseline
Huffman size of each block and plane, on the codec's own base layer at
ragged and full sizes and on constructed level arrays (long zero runs,
extreme categories), with levels beyond the baseline tables reported."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2309_11072_gb300 import codec, native, synth

pytestmark = pytest.mark.gpu


def _gpu_bits(levels: np.ndarray, h: int, w: int):
    L = torch.from_numpy(np.ascontiguousarray(levels, np.int16).reshape(-1).copy()).cuda()
    bits = torch.full((3,), -1, dtype=torch.int64, device="cuda")
    bh, bw = (h + 7) // 8, (w + 7) // 8
    blk = torch.full((3 * bh * bw,), -1, dtype=torch.int32, device="cuda")
    native.jpeg_huffman_bits(L, h, w, bits, blk)
    torch.cuda.synchronize()
    return bits.cpu().numpy().view(np.uint64), blk.cpu().numpy().view(np.uint32).reshape(3, bh * bw)


@pytest.mark.parametrize("h,w,q", [(8, 8, 50), (13, 21, 75), (33, 130, 10), (96, 136, 90), (1536, 2048, 50)])
def test_levels_and_bits_of_the_base_layer(h, w, q):
    img = synth.make_rgbe(h, w, seed=h * 7 + w, lo=-3.0, hi=5.0, rects=4)
    c = codec.Codec(h, w, "cuda")
    rgbe = torch.from_numpy(img.view(np.int32).reshape(-1).copy()).cuda()
    c.encode(rgbe, q)
    bh, bw = (h + 7) // 8, (w + 7) // 8
    levels = torch.full((3 * bh * bw * 64,), 0x5A5A, dtype=torch.int16, device="cuda")
    s3 = torch.empty_like(c.s3)
    native.device_status(clear=True)
    native.sdri_base_levels(c.m3, c.e, h, w, c.stats, q, s3, levels)
    torch.cuda.synchronize()
    o = O.encode(img, q)
    assert torch.equal(s3, c.s3)                                         # the same round trip
    lv = levels.cpu().numpy().reshape(3, bh * bw, 64)
    assert np.array_equal(lv, O.base_levels(o["sdr3"], q))
    bits, blk = _gpu_bits(lv, h, w)
    obits, oblk = O.jpeg_bits(lv, h, w)
    assert np.array_equal(blk, oblk) and np.array_equal(bits, obits)
    assert native.device_status(clear=True) == 0


def test_constructed_levels_long_runs_and_extreme_categories():
    h, w = 24, 40
    bh, bw = 3, 5
    rng = np.random.default_rng(3)
    lv = np.zeros((3, bh * bw, 64), np.int16)
    # sparse random levels: long zero runs and every size category
    for c in range(3):
        for b in range(bh * bw):
            k = rng.integers(0, 6)
            pos = rng.choice(64, size=k, replace=False)
            mag = (1 << rng.integers(0, 10, size=k)) + rng.integers(0, 2, size=k)
            lv[c, b, pos] = (mag * rng.choice([-1, 1], size=k)).astype(np.int16)
    lv[0, 0, 0] = 2047                     # DC category 11
    lv[0, 1, 0] = 0                        # back down by 2047: category 11 again
    lv[1, 3, 7 * 8 + 7] = 1023             # AC size 10 at the last zigzag position
    native.device_status(clear=True)
    bits, blk = _gpu_bits(lv, h, w)
    obits, oblk = O.jpeg_bits(lv, h, w)
    assert np.array_equal(blk, oblk) and np.array_equal(bits, obits)
    assert native.device_status(clear=True) == 0


def test_levels_beyond_the_baseline_tables_are_reported():
    h, w = 8, 16
    lv = np.zeros((3, 2, 64), np.int16)
    lv[2, 1, 5] = 1024                       # an AC level of size 11
    native.device_status(clear=True)
    _gpu_bits(lv, h, w)
    assert native.device_status(clear=True) == 4
    lv[2, 1, 5] = 0
    lv[0, 0, 0] = 2048                       # a DC difference of category 12
    _gpu_bits(lv, h, w)
    assert native.device_status(clear=True) == 4
