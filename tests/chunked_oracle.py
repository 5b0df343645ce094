"""The CPU oracle run column chunk by column chunk, for images too large to
hold whole (test infrastructure: the size-limit GPU test and its CPU pin).

Exact for images of 8 or 16 rows and chunk widths that are multiples of 8:
every 8x8 block of the base round trip (Sec. II-B) lies in one chunk (a
chunk is coded with the whole blocks around it), the 3x3 restoration filter
(Sec. III-B) needs one neighbouring column, which each chunk carries on both
sides, and the exponent-binned sums of Eqs. 9-10 and the residual
histograms add over disjoint pixel sets.  The tone mapping uses the whole
image's key.  Only the oracle computes here."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from oracle import oracle as O
from paper_2309_11072_gb300 import synth

CHUNK = 1 << 19          # columns per oracle chunk (a multiple of 8)
Q = 90


def image(h, w, seed):
    """h x w words: a seeded h x 100,000 scene repeated along the rows."""
    tile = synth.make_rgbe(h, 100_000, seed=seed, lo=-3.0, hi=5.0, rects=4, highlights=20)
    reps = -(-w // tile.shape[1])
    return np.ascontiguousarray(np.tile(tile, (1, reps))[:, :w])


def oracle_chunk(img, x0, x1, J, r):
    """The oracle's S, x = 16 S*, mantissas and exponents of columns x0 .. x1 - 1."""
    h, w = img.shape
    a0, a1 = max(x0 - 8, 0), min(x1 + 8, w)           # whole 8x8 blocks around the chunk
    words = np.ascontiguousarray(img[:, a0:a1])
    s3 = O.base_roundtrip(O.tmo(words, J, r), Q)
    x3 = O.gf(s3, True)
    sl = slice(x0 - a0, x1 - a0)
    m3, e = O.rgbe_split(np.ascontiguousarray(img[:, x0:x1]))
    return s3[:, :, sl], np.ascontiguousarray(x3[:, :, sl]), m3, e


def chunks(w):
    edges = list(range(0, w, CHUNK)) + [w]
    return list(zip(edges[:-1], edges[1:]))


def _pool():
    return ThreadPoolExecutor(max_workers=max(1, min(16, os.cpu_count() or 1)))


def oracle_sums(img, J, r):
    def one(ch):
        _, x3, m3, e = oracle_chunk(img, ch[0], ch[1], J, r)
        return O.bin_sums(x3, m3, e)

    with _pool() as ex:
        return sum(ex.map(one, chunks(img.shape[1])))


def oracle_hist(img, J, r, a, b):
    def one(ch):
        _, x3, m3, e = oracle_chunk(img, ch[0], ch[1], J, r)
        return O.residual(m3, O.predict(x3, e, a, b))[1].astype(np.int64)

    with _pool() as ex:
        return sum(ex.map(one, chunks(img.shape[1])))


