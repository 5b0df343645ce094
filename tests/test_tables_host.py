"""The library's constant tables (csrc/tables.inc, written by
csrc/gen_tables.py) against the oracle's own, independently built tables,
and the display-code lookup the base kernel does with them (one bucket
word and one integer comparison) against the oracle's threshold count, at
every threshold and its neighbouring float32 values."""
import os
import re
import struct

import numpy as np

from oracle import oracle as O

INC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2309_11072_gb300", "csrc",
                   "tables.inc")


def _table(name: str) -> np.ndarray:
    text = open(INC).read()
    m = re.search(r"\b" + name + r"\[(\d+)\]\s*=\s*\{(.*?)\};", text, re.S)
    assert m, name
    vals = [int(v.rstrip("u"), 0) for v in re.findall(r"-?0x[0-9a-fA-F]+u?|-?\d+", m.group(2))]
    assert len(vals) == int(m.group(1))
    return np.array(vals, dtype=np.int64)


def _bits(a) -> np.ndarray:
    return np.asarray(a, np.float32).view(np.uint32).astype(np.int64)


def test_tables_equal_the_oracles():
    assert np.array_equal(_table("kLog2Lut"), O.log2_table().astype(np.int64))
    assert np.array_equal(_table("kGammaBits"), _bits(O.gamma_thresholds()))
    kr, wr = O.key_tables()
    assert np.array_equal(_table("kKrBits"), _bits(kr))
    assert np.array_equal(_table("kWrBits"), _bits(wr))


def _display_code(v: np.ndarray, code: np.ndarray) -> np.ndarray:
    # the kernel's lookup: the float bits clamped to the below / above
    # buckets, the entry of their high half, then (bits + word) >> 16 mod
    # 2^32: the bucket's start plus one where the low bits reach the
    # threshold's
    bits = np.clip(np.asarray(v, np.float32).view(np.int32).astype(np.int64), 0x357F0000, 0x3F800000)
    e = code[(bits >> 16) - 0x357F].astype(np.int64)
    return ((bits + e) & 0xFFFFFFFF) >> 16


def test_display_code_lookup_equals_the_threshold_count():
    code = _table("kGammaCode")
    t = O.gamma_thresholds()
    tb = t[1:].view(np.uint32).astype(np.int64)
    near = (tb[:, None] + np.arange(-3, 4)[None, :]).reshape(-1)
    rng = np.random.default_rng(22)
    v = np.concatenate([near.astype(np.uint32).view(np.float32),
                        np.array([0.0, 1e-45, 1e-38, 2.0 ** -20, 1.0, 1.5, 3e38], np.float32),
                        rng.uniform(0, 1.2, 200_000).astype(np.float32),
                        (2.0 ** rng.uniform(-30, 1, 200_000)).astype(np.float32)])
    want = np.searchsorted(t[1:], v, side="right")        # #{k in 1..255 : v >= t[k]}
    assert np.array_equal(_display_code(v, code), want)
