"""Batch form on the GPU: many uneven images in one persistent launch per
stage.  Every image must equal the CPU oracle bit for bit, whatever the tile
choice; the autotuner and the captured CUDA graph must not change a result."""
import os

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2309_11072_gb300 import batch as B
from paper_2309_11072_gb300 import synth

pytestmark = pytest.mark.gpu

# widths on and off the 16-element row pitch; two images wider than one
# 2048-column strip of the row stages, with a ragged last strip
SIZES = [(64, 96), (1, 1), (0, 17), (37, 300), (257, 129), (8, 8), (120, 264), (9, 17), (200, 331), (5, 1000),
         (19, 2050), (6, 4111)]
QUALS = [90, 50, 75, 10, 85, 100, 60, 30, 95, 70, 80, 40]


def _images(sizes, seed0=100):
    out = []
    for k, (h, w) in enumerate(sizes):
        if h * w == 0:
            out.append(np.zeros((h, w), np.uint32))
        else:
            out.append(synth.make_rgbe(h, w, seed=seed0 + k, lo=-3.0, hi=5.0, rects=2, highlights=3))
    return out


def _host(t, dt):
    return t.detach().cpu().contiguous().view(torch.uint8).numpy().view(dt)


def _check_against_oracle(bc, imgs, quals, gf_on=True):
    torch.cuda.synchronize()
    gfs = [gf_on] * len(imgs) if isinstance(gf_on, bool) else list(gf_on)
    for i, img in enumerate(imgs):
        h, w = img.shape
        L = bc.image_layers(i)
        if h * w == 0:
            p = bc.image_params(i)
            assert p["n_used"] == 0
            continue
        o = O.encode(img, quals[i], gfs[i])
        assert np.array_equal(_host(L["m3"], np.uint8).reshape(3, h, w), o["m3"]), i
        assert np.array_equal(_host(L["e"], np.uint8).reshape(h, w), o["e"]), i
        assert np.array_equal(_host(L["s3"], np.uint8).reshape(3, h, w), o["s3"]), i
        p = bc.image_params(i)
        assert np.array_equal(p["a"].view(np.uint32), o["a"].view(np.uint32)), i
        assert np.array_equal(p["b"].view(np.uint32), o["b"].view(np.uint32)), i
        assert np.array_equal(p["n"], o["n"]) and p["n_used"] == o["n_used"], i
        assert np.array_equal(_host(L["r3"], np.int16).reshape(3, h, w), o["r3"]), i
        assert np.array_equal(_host(L["hist"], np.uint32).reshape(3, 511), o["hist"]), i
        assert np.array_equal(_host(L["out"], np.uint32).reshape(h, w), img), i


def _snapshot(bc):
    torch.cuda.synchronize()
    return [t.clone() for t in (bc.m3, bc.e, bc.s3, bc.r3, bc.params, bc.hist, bc.out)]


def _same(a, b):
    return all(torch.equal(x, y) for x, y in zip(a, b))


@pytest.mark.parametrize("gf_on", [True, False])
def test_batch_matches_oracle_per_image(gf_on):
    imgs = _images(SIZES)
    bc = B.BatchCodec(SIZES, QUALS, gf_on=gf_on)
    bc.load(imgs)
    bc.encode()
    bc.decode()
    _check_against_oracle(bc, imgs, QUALS, gf_on)


def test_batch_with_mixed_restoration_flags():
    """Images with and without the restoration filter in one batch (the row
    stages then read each image's flag on the device)."""
    imgs = _images(SIZES, seed0=700)
    gfs = [i % 3 != 1 for i in range(len(SIZES))]
    bc = B.BatchCodec(SIZES, QUALS, gf_on=gfs)
    bc.load(imgs)
    bc.encode()
    bc.decode()
    _check_against_oracle(bc, imgs, QUALS, gfs)


def test_batch_without_histograms_gives_the_same_residuals():
    """A batch encode with hist = NULL writes the same residual planes and
    leaves the histogram buffer alone."""
    imgs = _images(SIZES, seed0=800)
    bc = B.BatchCodec(SIZES, QUALS)
    bc.load(imgs)
    bc.encode()
    torch.cuda.synchronize()
    ref = bc.r3.clone()
    bc.r3.zero_()
    bc.hist.fill_(-1)
    bc.bufs.hist = None
    bc.encode()
    torch.cuda.synchronize()
    assert torch.equal(bc.r3, ref)
    assert bool((bc.hist == -1).all())


def test_batch_results_do_not_depend_on_tiles():
    imgs = _images(SIZES, seed0=300)
    bc = B.BatchCodec(SIZES, QUALS)
    bc.load(imgs)
    bc.encode()
    bc.decode()
    ref = _snapshot(bc)
    for kw in (dict(split_ctas_per_sm=1, base_ctas_per_sm=1), dict(split_ctas_per_sm=8, base_ctas_per_sm=3),
               dict(split_ctas_per_sm=2, base_ctas_per_sm=2)):
        bc.set_tiles(**kw)
        for t in (bc.m3, bc.s3, bc.r3, bc.out):
            t.zero_()
        bc.encode()
        bc.decode()
        assert _same(_snapshot(bc), ref), kw


def test_autotune_and_graph_replay_keep_results():
    imgs = _images(SIZES, seed0=500)
    bc = B.BatchCodec(SIZES, QUALS)
    bc.load(imgs)
    bc.encode()
    bc.decode()
    ref = _snapshot(bc)
    tiles = bc.autotune(reps=2)
    assert set(tiles) == {"split_ctas_per_sm", "base_ctas_per_sm"}
    assert 1 <= tiles["split_ctas_per_sm"] <= 8 and 1 <= tiles["base_ctas_per_sm"] <= 3
    bc.encode()
    bc.decode()
    assert _same(_snapshot(bc), ref)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for t in (bc.m3, bc.s3, bc.r3, bc.out):
            t.zero_()
        bc.graph_build(s)
        bc.graph_launch(s)
        bc.graph_launch(s)
    s.synchronize()
    assert _same(_snapshot(bc), ref)
    bc.close()


def _oracle_all(imgs, quals, gf_on=True):
    """The CPU oracle's encoding of every image, one thread per image (the
    oracle's C calls release the GIL, so the images run on separate cores)."""
    from concurrent.futures import ThreadPoolExecutor
    O.lib()
    gfs = [gf_on] * len(imgs) if isinstance(gf_on, bool) else list(gf_on)
    with ThreadPoolExecutor(max_workers=max(1, min(len(imgs), os.cpu_count() or 1))) as ex:
        return list(ex.map(lambda k: None if imgs[k].size == 0 else O.encode(imgs[k], quals[k], gfs[k]),
                           range(len(imgs))))


def _check_all(bc, imgs, quals, gf_on=True):
    """Every layer of every image against the oracle, bit for bit."""
    torch.cuda.synchronize()
    ref = _oracle_all(imgs, quals, gf_on)
    for i, (img, o) in enumerate(zip(imgs, ref)):
        h, w = img.shape
        p = bc.image_params(i)
        if o is None:
            assert p["n_used"] == 0, i
            continue
        L = bc.image_layers(i)
        assert np.array_equal(_host(L["m3"], np.uint8).reshape(3, h, w), o["m3"]), i
        assert np.array_equal(_host(L["e"], np.uint8).reshape(h, w), o["e"]), i
        assert np.array_equal(_host(L["s3"], np.uint8).reshape(3, h, w), o["s3"]), i
        assert np.array_equal(p["a"].view(np.uint32), o["a"].view(np.uint32)), i
        assert np.array_equal(p["b"].view(np.uint32), o["b"].view(np.uint32)), i
        assert np.array_equal(p["n"], o["n"]) and p["n_used"] == o["n_used"], i
        assert np.array_equal(_host(L["r3"], np.int16).reshape(3, h, w), o["r3"]), i
        assert np.array_equal(_host(L["hist"], np.uint32).reshape(3, 511), o["hist"]), i
        assert np.array_equal(_host(L["out"], np.uint32).reshape(h, w), img), i


def test_batch_ctas_that_cross_image_boundaries():
    """200 small images (1 to 128 rows): the row stages split the batch's
    rows into one contiguous range per CTA (two CTAs per SM), about 40 rows
    each, so most CTAs change image in the middle of the launch (flushing
    their shared bins and histograms to one image and loading the next
    one's parameters) and some cover several short images; the images
    alternate irregularly between restoration on and off.  Every image must
    still equal the oracle."""
    rng = np.random.default_rng(77)
    sizes = [(int(rng.integers(1, 129)), int(rng.integers(1, 257))) for _ in range(200)]
    quals = [int(q) for q in rng.choice([30, 50, 75, 90, 100], size=len(sizes))]
    gfs = [bool(g) for g in rng.random(len(sizes)) < 0.7]
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    imgs = _images(sizes, seed0=900)
    bc = B.BatchCodec(sizes, quals, gf_on=gfs)
    rows_per_cta = bc.plan.tile_rows / (2 * sms)
    assert rows_per_cta < 64 and min(h for h, _ in sizes) < rows_per_cta / 4
    bc.load(imgs)
    bc.set_tiles(split_ctas_per_sm=1, base_ctas_per_sm=1)
    bc.encode()
    bc.decode()
    _check_all(bc, imgs, quals, gfs)
    bc.close()


@pytest.mark.slow
def test_batch_workload_64_uneven_images():
    """The 64-image uneven workload (about 174 MP): every layer of every image
    against the oracle, with the tiles the autotuner picks."""
    wl = synth.workload_batch()
    imgs = synth.make_workload_images(wl)
    quals = list(wl.qualities) * len(wl.sizes)
    bc = B.BatchCodec(wl.sizes, quals)
    bc.load(imgs)
    bc.autotune(reps=1)
    bc.encode()
    bc.decode()
    _check_all(bc, imgs, quals)
    bc.close()
