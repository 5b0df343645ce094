"""A minimal driver of the five coder calls for profilers (ncu).

Builds one benchmark image, runs rgbe_split, sdri_base_roundtrip, slr_fit,
residual_encode and residual_decode once to warm up, then once more (the
launches to capture), and checks that the decoded words equal the input and
that no kernel's bounded wait gave up.  It holds only the one codec's
buffers on the device (about 0.7 GB at 7680x4320), so a profiler that saves
and restores device memory between its passes stays quick.  With
`--workload batch64` it runs the batch form's encode and decode over the
64-image uneven workload (about 3.8 GB of batch planes) twice instead, with
the batch's default grid sizes.  With `--call cnn` it codes the image, then
runs the learned estimator's cnn_residual_encode twice with the shipped
network and its decoder once, and checks that decoding is lossless.

    python -m paper_2309_11072_gb300.profile_calls --workload 8k
    ncu --set full --clock-control none -k regex:"k_fit_tile|k_rows_tile|k_base" -s 4 -c 4 \\
        -o prof python -m paper_2309_11072_gb300.profile_calls --workload 8k
"""
from __future__ import annotations

import argparse

import numpy as np
import torch

from . import codec, native, synth


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", choices=["8k", "2k", "batch64"], default="8k")
    ap.add_argument("--quality", type=int, default=90)
    ap.add_argument("--call", choices=["coder", "cnn"], default="coder")
    args = ap.parse_args(argv)
    if args.workload == "batch64":
        return batch_main()
    wl = synth.workload_8k() if args.workload == "8k" else synth.workload_2k()
    (h, w), = wl.sizes
    img = synth.make_workload_images(wl)[0]
    rgbe = torch.from_numpy(img.view(np.int32).reshape(-1).copy()).cuda()
    c = codec.Codec(h, w, "cuda", gf_on=True)
    st = torch.cuda.current_stream()
    for _ in range(2):
        native.rgbe_split(rgbe, h, w, c.m3, c.e, c.stats, st)
        native.sdri_base_roundtrip(c.m3, c.e, h, w, c.stats, args.quality, c.s3, None, st)
        native.slr_fit(c.s3, c.m3, c.e, h, w, 1, c.sums, c.params, st)
        native.residual_encode(c.s3, c.m3, c.e, h, w, 1, c.params, c.r3, c.hist, st)
        native.residual_decode(c.s3, c.e, c.r3, h, w, 1, c.params, c.out, st)
        c.check()
    if not torch.equal(c.out, rgbe):
        raise SystemExit("decoded words differ from the input")
    if args.call == "cnn":
        from . import learned as Lr
        net = Lr.upload_net(Lr.load_net(Lr.default_weights()))
        J = native.rgbe_key_scale(c.stats.cpu().numpy())[0]
        r3 = torch.empty_like(c.r3)
        hist = torch.empty_like(c.hist)
        for _ in range(2):
            Lr.cnn_residual_encode(c.s3, c.m3, c.e, h, w, J, net, c.params, 1, r3, hist, st)
        c.out.zero_()
        Lr.cnn_residual_decode(c.s3, c.e, r3, h, w, J, net, c.params, 1, c.out, st)
        c.check()
        if not torch.equal(c.out, rgbe):
            raise SystemExit("the learned estimator's decode differs from the input")
    print(f"ok {w}x{h} q{args.quality} {args.call}")


def batch_main():
    from . import batch
    wl = synth.workload_batch()
    imgs = synth.make_workload_images(wl)
    bc = batch.BatchCodec(wl.sizes, list(wl.qualities) * len(wl.sizes))
    bc.load(imgs)
    for _ in range(2):
        bc.encode()
        bc.decode()
        native.check_device_status("profile_calls")
    for i, img in enumerate(imgs):
        if not np.array_equal(bc.image_layers(i)["out"].cpu().numpy().view(np.uint32), img):
            raise SystemExit(f"image {i}: decoded words differ from the input")
    print(f"ok {wl.name}: {len(imgs)} images")


if __name__ == "__main__":
    main()
