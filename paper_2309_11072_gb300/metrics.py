"""Host-side rate metrics for the enhancement layer.

The paper codes the residual planes with JPEG 2000 lossless (Sec. IV); this
project reports the order-0 entropy of the residual histograms instead (the
histograms come from the encoder kernel), plus the side information of
Sec. III-C: one 32-bit slope and one 32-bit intercept per channel and used
exponent region, and a 256-bit map of the used regions.
"""
from __future__ import annotations

import math
from typing import Sequence


def entropy_bits(hist: Sequence[int]) -> float:
    """Order-0 entropy in bits per symbol of one histogram."""
    tot = float(sum(int(v) for v in hist))
    if tot <= 0:
        return 0.0
    h = 0.0
    for v in hist:
        v = int(v)
        if v:
            p = v / tot
            h -= p * math.log2(p)
    return h


def enhancement_bits_per_pixel(hist3, n_used: int, n_px: int, flag_bits: int = 0) -> float:
    """Sum over the three residual planes of H0, plus side information per pixel."""
    side = 256 + 3 * 64 * int(n_used) + int(flag_bits)
    return sum(entropy_bits(h) for h in hist3) + side / float(n_px)


def reduction_pct(reference: float, ours: float) -> float:
    """Relative reduction of ``ours`` against ``reference``, in percent."""
    if reference <= 0:
        raise ValueError("reference must be positive")
    return 100.0 * (reference - ours) / reference
