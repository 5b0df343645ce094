"""Writes tests/golden/tiny_codec_q75.json from the CPU oracle only.

The input is a fixed 11x13 array of RGBE words built from integer
arithmetic (no FFT, so it is identical on every machine); the expected
values are the oracle's intermediates at quality 75 with the Gaussian
restoration on.  Run from the repository root:
    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O  # noqa: E402


def tiny_input():
    h, w = 11, 13
    y, x = np.mgrid[0:h, 0:w]
    E = 118 + (3 * y + 2 * x) // 7                     # exponent regions in diagonal bands
    R = (128 + (37 * x + 11 * y) % 128)
    G = (60 + 5 * x * y) % 256
    B = (200 - 7 * x + 3 * y) % 256
    E[0, 0] = 0
    R[0, 0] = G[0, 0] = B[0, 0] = 0
    return (R | (G << 8) | (B << 16) | (E << 24)).astype(np.uint32)


def main():
    img = tiny_input()
    enc = O.encode(img, 75, True)
    used = np.nonzero(enc["n"])[0]
    out = {
        "source": "oracle/slrme_oracle.c via tests/golden/make_golden.py",
        "quality": 75, "gf_on": 1, "h": 11, "w": 13,
        "rgbe": img.reshape(-1).tolist(),
        "stats": enc["stats"].tolist(), "J": enc["J"], "r": enc["r"],
        "sdr3": enc["sdr3"].reshape(-1).tolist(),
        "s3": enc["s3"].reshape(-1).tolist(),
        "used": used.tolist(),
        "sums_used": enc["sums"][used].tolist(),
        "a_bits": enc["a"][:, used].view(np.uint32).reshape(-1).tolist(),
        "b_bits": enc["b"][:, used].view(np.uint32).reshape(-1).tolist(),
        "r3": enc["r3"].reshape(-1).tolist(),
    }
    with open(os.path.join(HERE, "tiny_codec_q75.json"), "w") as fh:
        json.dump(out, fh, separators=(",", ":"))


if __name__ == "__main__":
    main()
