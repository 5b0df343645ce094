"""Pins of the oracle's base-layer entropy coding (JPEG baseline Huffman
coding of the quantised DCT levels, T.81 Annex F.1.2 with the Annex K.3
luminance tables; Sec. IV codes the base layer with JPEG), against what the
standard and the mathematics fix rather than against the oracle itself:
- the code lengths form complete prefix codes but for the all-ones code
  the standard reserves (Kraft sums 1 - 2^-9 and 1 - 2^-16) over exactly
  the valid symbols;
- the zigzag order of T.81 Figure A.6;
- the levels dequantise to the pinned base round trip;
- the cost of blocks whose coding follows by hand from the rules: empty
  blocks, DC prediction across block rows, runs that need ZRL codes, the
  largest categories."""
import numpy as np
import pytest

from oracle import oracle as O

ZIGZAG_A6 = [0, 1, 8, 16, 9, 2, 3, 10, 17, 24, 32, 25, 18, 11, 4, 5, 12, 19, 26, 33, 40, 48, 41, 34, 27, 20, 13, 6,
             7, 14, 21, 28, 35, 42, 49, 56, 57, 50, 43, 36, 29, 22, 15, 23, 30, 37, 44, 51, 58, 59, 52, 45, 38, 31, 39,
             46, 53, 60, 61, 54, 47, 55, 62, 63]


def test_code_lengths_are_complete_prefix_codes_over_the_valid_symbols():
    dc = [O.jpeg_dc_len(c) for c in range(12)]
    assert sum(2.0 ** -l for l in dc) == 1.0 - 2.0 ** -9
    assert O.jpeg_dc_len(12) == 0
    valid = {0x00, 0xF0} | {(r << 4) | s for r in range(16) for s in range(1, 11)}
    lens = {sym: O.jpeg_ac_len(sym) for sym in range(256)}
    assert {s for s, l in lens.items() if l > 0} == valid and len(valid) == 162
    assert sum(2.0 ** -lens[s] for s in valid) == 1.0 - 2.0 ** -16
    assert max(lens.values()) == 16


def test_zigzag_is_figure_a6():
    zz = O.zigzag()
    assert list(zz) == ZIGZAG_A6
    for a, b in zip(zz[:-1], zz[1:]):        # every step moves to a neighbouring coefficient
        assert abs(a // 8 - b // 8) <= 1 and abs(a % 8 - b % 8) <= 1


@pytest.mark.parametrize("h,w,q", [(8, 8, 50), (13, 21, 75), (40, 24, 10), (9, 17, 100)])
def test_levels_dequantise_to_the_base_round_trip(h, w, q):
    rng = np.random.default_rng(h * w + q)
    sdr = rng.integers(0, 256, size=(3, h, w)).astype(np.uint8)
    L = O.base_levels(sdr, q)
    Q = O.quant_table(q)          # [v][u]
    bh, bw = (h + 7) // 8, (w + 7) // 8
    s_rt = O.base_roundtrip(sdr, q)
    # rebuild S from the levels with the oracle's own (pinned) inverse transform
    import ctypes
    out = np.zeros((3, h, w), np.uint8)
    for c in range(3):
        for b in range(bh * bw):
            by, bx = divmod(b, bw)
            F = (L[c, b].reshape(8, 8).T.astype(np.int32) * Q).reshape(-1)   # back to [v][u]
            X = np.zeros(64, np.int32)
            O.lib().oracle_idct_block(O._p(np.ascontiguousarray(F)), O._p(X))
            blk = np.clip(X.reshape(8, 8) + 128, 0, 255)
            hh, ww = min(8, h - 8 * by), min(8, w - 8 * bx)
            out[c, 8 * by:8 * by + hh, 8 * bx:8 * bx + ww] = blk[:hh, :ww]
    assert np.array_equal(out, s_rt)


def test_constant_planes_have_only_dc_levels():
    sdr = np.stack([np.full((16, 16), v, np.uint8) for v in (128, 255, 0)])
    L = O.base_levels(sdr, 100)
    assert (L[:, :, 1:] == 0).all()
    assert (L[0, :, 0] == 0).all() and (L[1, :, 0] == 8 * 127).all() and (L[2, :, 0] == -8 * 128).all()


def _blocks(*blocks):
    """Levels of one plane (the others zero) from per-block {natural index (v*8+u): level} maps."""
    L = np.zeros((3, len(blocks), 64), np.int16)
    for b, d in enumerate(blocks):
        for nat, lv in d.items():
            v, u = divmod(nat, 8)
            L[0, b, u * 8 + v] = lv
    return L


def test_hand_worked_block_costs():
    # one row of 4 blocks (h = 8, w = 32)
    L = _blocks({}, {0: 5}, {0: 5, 1: -1}, {0: 4, 63: 1})
    bits, blk = O.jpeg_bits(L, 8, 32)
    assert blk[0, 0] == 2 + 4                    # DC diff 0 (2 bits), EOB (4)
    assert blk[0, 1] == 3 + 3 + 4                # diff 5: category 3 (3-bit code + 3 bits), EOB
    assert blk[0, 2] == 2 + 2 + 1 + 4            # diff 0; zigzag 1 = -1: symbol 0x01 (2) + 1 bit; EOB
    # diff -1 (category 1: 3 + 1); 62 zeros then a 1 in the last position:
    # three ZRL codes (11 bits each), symbol 0xE1 (16) + 1 bit, no EOB
    assert blk[0, 3] == 3 + 1 + 3 * 11 + 16 + 1
    assert bits[0] == blk[0].sum() and bits[1] == 4 * 6 and bits[2] == 4 * 6


def test_dc_prediction_runs_across_block_rows_and_zrl_boundaries():
    # 2 x 2 blocks: raster order (0,0), (0,1), (1,0), (1,1)
    L = _blocks({0: 100}, {0: 100}, {0: -100}, {0: -100, ZIGZAG_A6[17]: 3})
    _, blk = O.jpeg_bits(L, 16, 16)
    assert blk[0, 0] == 5 + 7 + 4                # diff 100: category 7 (a 5-bit code) + 7 bits, EOB
    assert blk[0, 1] == 2 + 4
    assert blk[0, 2] == 6 + 8 + 4                # diff -200 after the first row: category 8 (6 bits) + 8 bits
    # a 3 after exactly 16 zeros: one ZRL (11), then symbol 0x02 (2) + 2 bits, EOB
    assert blk[0, 3] == 2 + 11 + 2 + 2 + 4


def test_largest_categories_and_their_limits():
    L = _blocks({0: 2047}, {0: 2047, 1: 1023})
    _, blk = O.jpeg_bits(L, 8, 16)
    assert blk[0, 0] == 9 + 11 + 4               # category 11
    assert blk[0, 1] == 2 + 16 + 10 + 4          # diff 0; symbol 0x0A (16) + 10 bits; EOB
    with pytest.raises(ValueError):
        O.jpeg_bits(_blocks({0: 2048}), 8, 8)
    with pytest.raises(ValueError):
        O.jpeg_bits(_blocks({1: 1024}), 8, 8)
