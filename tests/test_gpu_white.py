"""GPU parity of Reinhard's operator with a white point (his Eq. 4 form)
against the oracle: the white point (the largest scaled luminance) bit for
bit, the display codes and the decoded base layer, at ragged and full
sizes, on images with zero-exponent pixels and a single bright pixel; an
infinite white point gives the plain operator."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2309_11072_gb300 import codec, native, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("h,w,q", [(1, 1, 50), (9, 11, 75), (33, 130, 90), (96, 136, 50), (1536, 2048, 75)])
def test_white_point_operator_bit_exact(h, w, q):
    img = synth.make_rgbe(h, w, seed=h + 5 * w, lo=-3.0, hi=5.0, rects=3, highlights=4)
    if h * w > 4:
        flat = img.reshape(-1).copy()
        flat[::7] &= 0x00FFFFFF                       # some pixels with E = 0
        img = flat.reshape(h, w)
    c = codec.Codec(h, w, "cuda")
    c.encode(torch.from_numpy(img.view(np.int32).reshape(-1).copy()).cuda(), q)
    lw = torch.full((1,), -1.0, dtype=torch.float32, device="cuda")
    native.sdri_white_point(c.m3, c.e, h, w, c.stats, lw)
    s3 = torch.empty_like(c.s3)
    sdr3 = torch.empty_like(c.s3)
    native.sdri_base_roundtrip_white(c.m3, c.e, h, w, c.stats, lw, q, s3, sdr3)
    torch.cuda.synchronize()
    J, r = O.key(O.lum_stats(img))
    olw = O.white_point(img, J, r)
    assert lw.cpu().numpy().view(np.uint32)[0] == np.float32(olw).view(np.uint32)
    osdr = O.tmo_white(img, J, r, olw)
    assert np.array_equal(sdr3.cpu().numpy().reshape(3, h, w), osdr)
    assert np.array_equal(s3.cpu().numpy().reshape(3, h, w), O.base_roundtrip(osdr, q))


def test_infinite_white_point_is_the_plain_operator():
    h, w, q = 40, 72, 75
    img = synth.make_rgbe(h, w, seed=3, lo=-3.0, hi=5.0, rects=2)
    c = codec.Codec(h, w, "cuda")
    c.encode(torch.from_numpy(img.view(np.int32).reshape(-1).copy()).cuda(), q)
    lw = torch.full((1,), float("inf"), dtype=torch.float32, device="cuda")
    s3 = torch.empty_like(c.s3)
    sdr_w = torch.empty_like(c.s3)
    sdr_p = torch.empty_like(c.s3)
    native.sdri_base_roundtrip_white(c.m3, c.e, h, w, c.stats, lw, q, s3, sdr_w)
    native.sdri_base_roundtrip(c.m3, c.e, h, w, c.stats, q, torch.empty_like(c.s3), sdr_p)
    torch.cuda.synchronize()
    assert torch.equal(sdr_w, sdr_p) and torch.equal(s3, c.s3)
