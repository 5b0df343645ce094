"""Learned estimator vs the regression, at workload scale, on one GPU.

Trains the integer CNN with the library's own kernels on crops of synthetic
images coded by the batch encoder, exports the integer network, then codes
held-out images with both estimators and picks, per image, the one whose
residuals cost fewer bits.  The training set cycles through three kinds:
512x512 fBm over 6 decades; 512x512 fBm over 8 decades with rectangles and
highlights (the 2048x1536 benchmark image's generator); and 1024x1024 fBm
over 8 decades with a smooth sky band in the top third (the 7680x4320
benchmark image's generator).  Two held-out sets are coded: 2048x1536
images of the second kind (seeds 20000 and up) and 3840x2160 images of the
third (seeds 30000 and up).  Synthesis runs in a pool of spawned processes
before the GPU is touched.

    python -m paper_2309_11072_gb300.learned_eval --train 2000 --test 200 \\
        --test-sky 8 --steps 6000 --json out.json --weights weights.npz
"""
from __future__ import annotations

import argparse
import json
import os
import time
from concurrent.futures import ProcessPoolExecutor
from multiprocessing import get_context

import numpy as np

from . import synth


def _train_spec(i: int):
    k = i % 3
    if k == 0:
        return (512, 512, 10000 + i, -2.0, 4.0, 0, 0, False)
    if k == 1:
        return (512, 512, 10000 + i, -3.0, 5.0, 40, 200, False)
    return (1024, 1024, 10000 + i, -3.0, 5.0, 0, 0, True)


def _test_spec(i: int):
    return (1536, 2048, 20000 + i, -3.0, 5.0, 40, 200, False)


def _sky_spec(i: int):
    return (2160, 3840, 30000 + i, -3.0, 5.0, 0, 0, True)


def _make(spec):
    h, w, seed, lo, hi, rects, highlights, sky = spec
    return synth.make_rgbe(h, w, seed=seed, lo=lo, hi=hi, rects=rects, highlights=highlights, sky=sky)


def make_all(specs, pool):
    return list(pool.map(_make, specs, chunksize=4))


def _code_and_pick(timgs, first, quality, net_dev, Bm, Lr, torch, entropy_bits):
    """Both estimators on a list of held-out images; one row per image."""
    dev = torch.device("cuda")
    rows, ms, px = [], 0.0, 0
    tb = Bm.BatchCodec([im.shape for im in timgs], [quality] * len(timgs))
    tb.load(timgs)
    tb.encode()
    tb.decode()
    tkeys = tb.keys()
    for i, img in enumerate(timgs):
        L = tb.dense_layers(i)
        h, w = img.shape
        r3 = torch.empty(3 * h * w, dtype=torch.int16, device=dev)
        hist = torch.empty(3 * 511, dtype=torch.int32, device=dev)
        out = torch.empty(h * w, dtype=torch.int32, device=dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        Lr.cnn_residual_encode(L["s3"], L["m3"], L["e"], h, w, tkeys[i], net_dev, L["params"], 1, r3, hist)
        e1.record()
        Lr.cnn_residual_decode(L["s3"], L["e"], r3, h, w, tkeys[i], net_dev, L["params"], 1, out)
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
        px += h * w
        lossless = bool(np.array_equal(out.cpu().numpy().view(np.uint32).reshape(h, w), img)) and \
            bool(np.array_equal(L["out"].cpu().numpy().view(np.uint32).reshape(h, w), img))
        hs = L["hist"].cpu().numpy().view(np.uint32).reshape(3, 511)
        hc = hist.cpu().numpy().view(np.uint32).reshape(3, 511)
        pk = Lr.pick_image(hs, tb.image_params(i)["n_used"], hc, h * w)
        rows.append(dict(image=first + i, bits_slr=pk.bits_slr, bits_cnn=pk.bits_cnn, pick_cnn=pk.use_cnn,
                         bits=pk.bits, lossless=lossless,
                         h0_slr=[entropy_bits(x) for x in hs], h0_cnn=[entropy_bits(x) for x in hc]))
    tb.close()
    return rows, ms, px


def _summary(rows):
    mean = lambda k: float(np.mean([r[k] for r in rows])) if rows else None
    return dict(images=len(rows), mean_bits_slr=mean("bits_slr"), mean_bits_cnn=mean("bits_cnn"),
                mean_bits_pick=mean("bits"),
                gain_bits=(mean("bits_slr") - mean("bits")) if rows else None,
                fraction_cnn_picked=float(np.mean([r["pick_cnn"] for r in rows])) if rows else None,
                all_lossless=all(r["lossless"] for r in rows))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--test", type=int, default=200)
    ap.add_argument("--test-sky", type=int, default=8)
    ap.add_argument("--steps", type=int, default=6000)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--crop", type=int, default=64)
    ap.add_argument("--quality", type=int, default=90)
    ap.add_argument("--chunk", type=int, default=20, help="test images coded per batch")
    ap.add_argument("--workers", type=int, default=min(16, os.cpu_count() or 1))
    ap.add_argument("--json", default=None)
    ap.add_argument("--weights", default=None)
    args = ap.parse_args(argv)

    # every image is made before the GPU is touched (the pool's processes are spawned)
    t0 = time.perf_counter()
    with ProcessPoolExecutor(max_workers=args.workers, mp_context=get_context("spawn")) as pool:
        imgs = make_all([_train_spec(i) for i in range(args.train)], pool)
        test_imgs = make_all([_test_spec(i) for i in range(args.test)], pool)
        sky_imgs = make_all([_sky_spec(i) for i in range(args.test_sky)], pool)
    t_gen = time.perf_counter() - t0

    import torch

    from . import batch as Bm
    from . import learned as Lr
    from .metrics import entropy_bits

    bc = Bm.BatchCodec([im.shape for im in imgs], [args.quality] * len(imgs))
    bc.load(imgs)
    del imgs
    bc.encode()
    torch.cuda.synchronize()
    keys = bc.keys()
    history = []
    t0 = time.perf_counter()
    tr = Lr.train(bc, keys, steps=args.steps, B=args.batch, H=args.crop, W=args.crop, seed=0,
                  log_every=max(1, args.steps // 20), history=history)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    theta = tr.theta.cpu().numpy()
    net = Lr.export_int_net(theta)
    net_dev = Lr.upload_net(net)
    bc.close()
    del bc, tr
    torch.cuda.empty_cache()

    rows, cnn_ms, cnn_px = [], 0.0, 0
    for start in range(0, args.test, args.chunk):
        r, ms, px = _code_and_pick(test_imgs[start:start + args.chunk], start, args.quality, net_dev, Bm, Lr, torch,
                                   entropy_bits)
        rows += r
        cnn_ms += ms
        cnn_px += px
        torch.cuda.empty_cache()
    sky_rows = []
    for start in range(0, args.test_sky, 4):
        r, ms, px = _code_and_pick(sky_imgs[start:start + 4], start, args.quality, net_dev, Bm, Lr, torch,
                                   entropy_bits)
        sky_rows += r
        torch.cuda.empty_cache()

    gflop = 2 * 5616 * cnn_px / 1e9
    summary = dict(train_images=args.train, test_images=args.test, test_sky_images=args.test_sky, steps=args.steps,
                   batch=args.batch, crop=args.crop, quality=args.quality,
                   train_kinds="512x512 fBm 6 decades; 512x512 fBm 8 decades + 40 rectangles + 200 highlights; "
                               "1024x1024 fBm 8 decades + sky band (cycling)",
                   test_kind="2048x1536 fBm 8 decades + 40 rectangles + 200 highlights, seeds 20000+",
                   test_sky_kind="3840x2160 fBm 8 decades + sky band, seeds 30000+",
                   loss_history=history, seconds_generate=round(t_gen, 1), seconds_train=round(t_train, 1),
                   held_out=_summary(rows), held_out_sky=_summary(sky_rows),
                   cnn_encode_mpix_s=round(cnn_px / (cnn_ms * 1e-3) / 1e6, 1) if cnn_ms else None,
                   cnn_encode_tflops_algorithmic=round(gflop / (cnn_ms * 1e-3) / 1e3, 2) if cnn_ms else None,
                   images=rows, images_sky=sky_rows)
    print(json.dumps({k: v for k, v in summary.items() if k not in ("images", "images_sky", "loss_history")}),
          flush=True)
    if args.json:
        with open(args.json, "w") as fh:
            json.dump(summary, fh)
    if args.weights:
        np.savez(args.weights, theta=theta, **{f"w{l}": net["w"][l] for l in range(4)},
                 **{f"b{l}": net["b"][l] for l in range(4)}, **{f"m{l}": net["m"][l] for l in range(4)},
                 sh=np.asarray(net["sh"], np.int32))


if __name__ == "__main__":
    main()
