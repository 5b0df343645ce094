"""The codec near the size limit of the C ABI (h * w < 2^31): images of
800 M pixels, whose third mantissa plane starts past element 2^31 and whose
residual planes span 4.8 GB, on both the bulk-copy row path (w % 16 == 0)
and the register-window strip path (w % 16 != 0).

The oracle cannot hold such an image whole; it runs column chunk by column
chunk (tests/chunked_oracle.py, exact for these shapes and pinned against the
whole-image oracle on the CPU).  Compared: the luminance statistic, the
parameters (a_E, b_E) and region counts bit for bit, the residual
histograms, the decoded base layer S and the residuals R on sampled column
windows (the first, the middle and the right edge), and the decoded words on
every pixel (Sec. I: lossless).  The batch form is run with such an image in
front of small ones, so every stage addresses images past element 2^31 of
its three-plane buffers."""
import numpy as np
import pytest
import torch

from chunked_oracle import Q, image, oracle_chunk, oracle_hist, oracle_sums
from oracle import oracle as O
from paper_2309_11072_gb300 import codec

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.mark.parametrize("h,w", [(16, 50_000_000), (8, 100_000_004)])
def test_codec_near_the_size_limit(h, w):
    n = h * w
    assert 3 * n > 2 ** 31 and 6 * n > 2 ** 32 and n < 2 ** 31
    img = image(h, w, seed=5)
    O.lib()
    st = O.lum_stats(img)
    J, r = O.key(st)
    a, b, cnt, n_used = O.solve(oracle_sums(img, J, r))
    hist = oracle_hist(img, J, r, a, b)

    c = codec.Codec(h, w, "cuda", gf_on=True)
    rgbe = torch.from_numpy(img.view(np.int32).reshape(-1)).cuda()
    L = c.encode(rgbe, Q)
    out = c.decode(L.s3, L.e, L.r3, L.params)
    torch.cuda.synchronize()
    assert torch.equal(out, rgbe)                         # lossless on every pixel
    del out
    assert np.array_equal(c.stats.cpu().numpy(), st)
    p = codec.params_to_numpy(c.params)
    assert np.array_equal(p["a"].view(np.uint32), a.view(np.uint32))
    assert np.array_equal(p["b"].view(np.uint32), b.view(np.uint32))
    assert np.array_equal(p["n"], cnt) and p["n_used"] == n_used
    assert np.array_equal(c.hist.view(3, 511).cpu().numpy().view(np.uint32).astype(np.int64), hist)
    # S and R on sampled windows: the first columns, the middle, and the last (the right edge)
    s3 = c.s3.view(3, h, w)
    r3 = c.r3.view(3, h, w)
    mid = (w // 2) // 8 * 8
    for x0, x1 in ((0, 4096), (mid, mid + 4096), ((w - 4096) // 8 * 8, w)):
        so, xo, mo, eo = oracle_chunk(img, x0, x1, J, r)
        assert np.array_equal(s3[:, :, x0:x1].cpu().numpy(), so), x0
        ro, _ = O.residual(mo, O.predict(xo, eo, a, b))
        assert np.array_equal(r3[:, :, x0:x1].cpu().numpy(), ro), x0


def test_batch_with_offsets_past_2_to_the_31():
    """The batch form with a 16 x 50,000,000 image first: the images after it
    start past element 800 M of the word planes, so their three-plane
    offsets (3 px_offset) pass 2^31 in every stage.  The large image is
    checked as above (statistic, parameters, histograms, sampled S and R,
    lossless); the small ones after it against the whole-image oracle."""
    from paper_2309_11072_gb300 import batch as B
    h, w = 16, 50_000_000
    big = image(h, w, seed=9)
    small = [synth_small(37, 300, 41), synth_small(8, 1000, 42)]
    imgs = [big] + small
    quals = [Q, 75, 50]
    bc = B.BatchCodec([im.shape for im in imgs], quals)
    assert 3 * bc.offset(1) > 2 ** 31
    bc.load(imgs)
    bc.encode()
    bc.decode()
    torch.cuda.synchronize()
    # the small images: every layer against the oracle
    for i in (1, 2):
        o = O.encode(imgs[i], quals[i], True)
        L = bc.image_layers(i)
        hh, ww = imgs[i].shape
        assert np.array_equal(L["s3"].cpu().numpy(), o["s3"]), i
        p = bc.image_params(i)
        assert np.array_equal(p["a"].view(np.uint32), o["a"].view(np.uint32)), i
        assert np.array_equal(p["b"].view(np.uint32), o["b"].view(np.uint32)), i
        assert np.array_equal(L["r3"].cpu().numpy(), o["r3"]), i
        assert np.array_equal(L["hist"].cpu().numpy().view(np.uint32), o["hist"]), i
        assert np.array_equal(L["out"].cpu().numpy().view(np.uint32), imgs[i]), i
    # the large one: lossless on every pixel, exact statistic, parameters and histograms
    L = bc.image_layers(0)
    rgbe = torch.from_numpy(big.view(np.int32))
    assert torch.equal(L["out"].cpu(), rgbe)
    st = O.lum_stats(big)
    assert np.array_equal(bc.lum_stats()[0], st)
    J, r = O.key(st)
    a, b, cnt, n_used = O.solve(oracle_sums(big, J, r))
    p = bc.image_params(0)
    assert np.array_equal(p["a"].view(np.uint32), a.view(np.uint32))
    assert np.array_equal(p["b"].view(np.uint32), b.view(np.uint32))
    assert np.array_equal(p["n"], cnt) and p["n_used"] == n_used
    hist = oracle_hist(big, J, r, a, b)
    assert np.array_equal(L["hist"].cpu().numpy().view(np.uint32).astype(np.int64), hist)
    mid = (w // 2) // 8 * 8
    for x0, x1 in ((0, 4096), (mid, mid + 4096), ((w - 4096) // 8 * 8, w)):
        so, xo, mo, eo = oracle_chunk(big, x0, x1, J, r)
        assert np.array_equal(L["s3"][:, :, x0:x1].cpu().numpy(), so), x0
        ro, _ = O.residual(mo, O.predict(xo, eo, a, b))
        assert np.array_equal(L["r3"][:, :, x0:x1].cpu().numpy(), ro), x0
    bc.close()


def synth_small(h, w, seed):
    from paper_2309_11072_gb300 import synth
    return synth.make_rgbe(h, w, seed=seed, lo=-3.0, hi=5.0, rects=2, highlights=3)
