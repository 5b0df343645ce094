"""Learned estimator vs the regression, at workload scale, on one GPU.

Trains the integer CNN with the library's own kernels on crops of synthetic
512x512 images coded by the batch encoder (half with 6 decades of fBm
luminance, half with 8 decades plus rectangles and highlights), exports the
integer network, then codes held-out 2048x1536 images (8 decades,
rectangles, highlights) with both estimators and picks, per image, the one
whose residuals cost fewer bits.

    python -m paper_2309_11072_gb300.learned_eval --train 2000 --test 200 \\
        --steps 4000 --json out.json --weights weights.npz
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import batch as Bm
from . import learned as Lr
from . import synth
from .metrics import entropy_bits


def train_images(n: int, size: int = 512):
    for i in range(n):
        if i % 2 == 0:
            yield synth.make_rgbe(size, size, seed=10000 + i, lo=-2.0, hi=4.0)
        else:
            yield synth.make_rgbe(size, size, seed=10000 + i, lo=-3.0, hi=5.0, rects=40, highlights=200)


def test_images(start: int, n: int):
    for i in range(start, start + n):
        yield synth.make_rgbe(1536, 2048, seed=20000 + i, lo=-3.0, hi=5.0, rects=40, highlights=200)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--test", type=int, default=200)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--crop", type=int, default=64)
    ap.add_argument("--quality", type=int, default=90)
    ap.add_argument("--chunk", type=int, default=20, help="test images coded per batch")
    ap.add_argument("--json", default=None)
    ap.add_argument("--weights", default=None)
    args = ap.parse_args(argv)
    dev = torch.device("cuda")

    t0 = time.perf_counter()
    imgs = list(train_images(args.train))
    t_gen = time.perf_counter() - t0
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
    del bc, tr
    torch.cuda.empty_cache()

    rows = []
    cnn_ms, cnn_px = 0.0, 0
    for start in range(0, args.test, args.chunk):
        n = min(args.chunk, args.test - start)
        timgs = list(test_images(start, n))
        tb = Bm.BatchCodec([im.shape for im in timgs], [args.quality] * n)
        tb.load(timgs)
        tb.encode()
        tb.decode()
        tkeys = tb.keys()
        for i, img in enumerate(timgs):
            L = tb.image_layers(i)
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
            cnn_ms += e0.elapsed_time(e1)
            cnn_px += h * w
            lossless = bool(np.array_equal(out.cpu().numpy().view(np.uint32).reshape(h, w), img)) and \
                bool(np.array_equal(L["out"].cpu().numpy().view(np.uint32).reshape(h, w), img))
            hs = L["hist"].cpu().numpy().view(np.uint32).reshape(3, 511)
            hc = hist.cpu().numpy().view(np.uint32).reshape(3, 511)
            pk = Lr.pick_image(hs, tb.image_params(i)["n_used"], hc, h * w)
            rows.append(dict(image=start + i, bits_slr=pk.bits_slr, bits_cnn=pk.bits_cnn, pick_cnn=pk.use_cnn,
                             bits=pk.bits, lossless=lossless,
                             h0_slr=[entropy_bits(x) for x in hs], h0_cnn=[entropy_bits(x) for x in hc]))
        tb.close()
        del tb, timgs
        torch.cuda.empty_cache()

    mean = lambda k: float(np.mean([r[k] for r in rows]))
    gflop = 2 * 5616 * cnn_px / 1e9
    summary = dict(train_images=args.train, test_images=args.test, steps=args.steps, batch=args.batch,
                   crop=args.crop, quality=args.quality, loss_history=history,
                   seconds_generate_train=round(t_gen, 1), seconds_train=round(t_train, 1),
                   mean_bits_slr=mean("bits_slr"), mean_bits_cnn=mean("bits_cnn"), mean_bits_pick=mean("bits"),
                   gain_bits=mean("bits_slr") - mean("bits"),
                   fraction_cnn_picked=float(np.mean([r["pick_cnn"] for r in rows])),
                   all_lossless=all(r["lossless"] for r in rows),
                   cnn_encode_mpix_s=round(cnn_px / (cnn_ms * 1e-3) / 1e6, 1),
                   cnn_encode_tflops_algorithmic=round(gflop / (cnn_ms * 1e-3) / 1e3, 2), images=rows)
    print(json.dumps({k: v for k, v in summary.items() if k != "images"}), flush=True)
    if args.json:
        with open(args.json, "w") as fh:
            json.dump(summary, fh)
    if args.weights:
        np.savez(args.weights, theta=theta, **{f"w{l}": net["w"][l] for l in range(4)},
                 **{f"b{l}": net["b"][l] for l in range(4)}, **{f"m{l}": net["m"][l] for l in range(4)},
                 sh=np.asarray(net["sh"], np.int32))


if __name__ == "__main__":
    main()
