"""GPU parity of the YCbCr 4:2:0 base layer against the oracle: the
decoded SDRI and the levels of the Y, Cb and Cr planes bit for bit, at
ragged sizes (odd heights and widths, chroma planes smaller than a block)
and at 2048x1536, the sizes of their Huffman coding with the luminance and
chrominance tables, and the rest of the codec running on the 4:2:0 layer
(fit, residuals, lossless decode)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2309_11072_gb300 import codec, native, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("h,w,q", [(1, 1, 50), (7, 5, 75), (13, 21, 10), (33, 130, 90), (96, 136, 85),
                                   (1536, 2048, 50)])
def test_420_base_layer_bit_exact(h, w, q):
    img = synth.make_rgbe(h, w, seed=h * 3 + w + q, lo=-3.0, hi=5.0, rects=3)
    c = codec.Codec(h, w, "cuda")
    c.encode(torch.from_numpy(img.view(np.int32).reshape(-1).copy()).cuda(), q)
    nbY, nbC = O.blocks_420(h, w)
    s3 = torch.full_like(c.s3, 77)
    lv = torch.full(((nbY + 2 * nbC) * 64,), 0x5A5A, dtype=torch.int16, device="cuda")
    ws = torch.empty(max(native.sdri_base_420_workspace_bytes(h, w), 256), dtype=torch.uint8, device="cuda")
    native.device_status(clear=True)
    native.sdri_base_roundtrip_420(c.m3, c.e, h, w, c.stats, q, s3, lv, ws)
    bits = torch.full((3,), -1, dtype=torch.int64, device="cuda")
    blk = torch.full((nbY + 2 * nbC,), -1, dtype=torch.int32, device="cuda")
    native.jpeg_huffman_bits_planes(lv, [nbY, nbC, nbC], [0, 1, 1], bits, blk)
    torch.cuda.synchronize()
    o = O.encode(img, q)
    os3, olv = O.base_roundtrip_420(o["sdr3"], q)
    assert np.array_equal(s3.cpu().numpy().reshape(3, h, w), os3)
    assert np.array_equal(lv.cpu().numpy().reshape(-1, 64), olv)
    obits, oblk = O.jpeg_bits_planes(olv, [nbY, nbC, nbC], [0, 1, 1])
    assert np.array_equal(blk.cpu().numpy().view(np.uint32), oblk)
    assert np.array_equal(bits.cpu().numpy().view(np.uint64), obits)
    assert native.device_status(clear=True) == 0


def test_codec_on_the_420_layer_is_lossless_and_matches_the_oracle():
    h, w, q = 96, 160, 75
    img = synth.make_rgbe(h, w, seed=11, lo=-3.0, hi=5.0, rects=4)
    c = codec.Codec(h, w, "cuda")
    rgbe = torch.from_numpy(img.view(np.int32).reshape(-1).copy()).cuda()
    c.encode(rgbe, q)
    ws = torch.empty(native.sdri_base_420_workspace_bytes(h, w), dtype=torch.uint8, device="cuda")
    s3 = torch.empty_like(c.s3)
    native.sdri_base_roundtrip_420(c.m3, c.e, h, w, c.stats, q, s3, None, ws)
    native.slr_fit(s3, c.m3, c.e, h, w, 1, c.sums, c.params)
    native.residual_encode(s3, c.m3, c.e, h, w, 1, c.params, c.r3, c.hist)
    out = c.decode(s3, c.e, c.r3, c.params)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint32).reshape(h, w), img)
    # the oracle's fit and residuals on its own 4:2:0 layer
    o = O.encode(img, q)
    os3, _ = O.base_roundtrip_420(o["sdr3"], q)
    x3 = O.gf(os3, True)
    sums = O.bin_sums(x3, o["m3"], o["e"])
    a, b, n, n_used = O.solve(sums)
    ms = O.predict(x3, o["e"], a, b)
    r3, _ = O.residual(o["m3"], ms)
    assert np.array_equal(c.r3.cpu().numpy().reshape(r3.shape), r3)
