"""Batch form on the GPU: many uneven images in one persistent launch per
stage.  Every image must equal the CPU oracle bit for bit, whatever the tile
choice; the autotuner and the captured CUDA graph must not change a result."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2309_11072_gb300 import batch as B
from paper_2309_11072_gb300 import synth

pytestmark = pytest.mark.gpu

SIZES = [(64, 96), (1, 1), (0, 17), (37, 300), (257, 129), (8, 8), (120, 264), (9, 17), (200, 331), (5, 1000)]
QUALS = [90, 50, 75, 10, 85, 100, 60, 30, 95, 70]


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
    for i, img in enumerate(imgs):
        h, w = img.shape
        L = bc.image_layers(i)
        if h * w == 0:
            p = bc.image_params(i)
            assert p["n_used"] == 0
            continue
        o = O.encode(img, quals[i], gf_on)
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


def test_batch_results_do_not_depend_on_tiles():
    imgs = _images(SIZES, seed0=300)
    bc = B.BatchCodec(SIZES, QUALS)
    bc.load(imgs)
    bc.encode()
    bc.decode()
    ref = _snapshot(bc)
    for kw in (dict(strip_rows=4, fit_ctas_per_sm=1, res_ctas_per_sm=1, split_ctas_per_sm=1, base_ctas_per_sm=1),
               dict(strip_rows=16, fit_ctas_per_sm=2, res_ctas_per_sm=2, split_ctas_per_sm=8, base_ctas_per_sm=3),
               dict(strip_rows=8, fit_ctas_per_sm=1, res_ctas_per_sm=2, split_ctas_per_sm=2, base_ctas_per_sm=2)):
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
    assert tiles["strip_rows"] in (4, 8, 16)
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


@pytest.mark.slow
def test_batch_workload_64_uneven_images():
    wl = synth.workload_batch()
    imgs = synth.make_workload_images(wl)
    bc = B.BatchCodec(wl.sizes, wl.qualities * len(wl.sizes))
    bc.load(imgs)
    bc.encode()
    bc.decode()
    torch.cuda.synchronize()
    out = _host(bc.out, np.uint32)
    for i, img in enumerate(imgs):
        h, w = img.shape
        o = bc.offset(i)
        assert np.array_equal(out[o:o + h * w].reshape(h, w), img), i
    # oracle parity, image by image, on the three smallest images
    small = sorted(range(len(imgs)), key=lambda i: imgs[i].size)[:3]
    sub = [imgs[i] for i in small]
    for k, i in enumerate(small):
        L = bc.image_layers(i)
        h, w = sub[k].shape
        o = O.encode(sub[k], wl.qualities[0])
        assert np.array_equal(_host(L["s3"], np.uint8).reshape(3, h, w), o["s3"])
        assert np.array_equal(_host(L["r3"], np.int16).reshape(3, h, w), o["r3"])
        p = bc.image_params(i)
        assert np.array_equal(p["a"].view(np.uint32), o["a"].view(np.uint32))
