"""Pins of the oracle's YCbCr 4:2:0 base layer (the colour handling of a
default JPEG encoder, which codes the base layer in Sec. IV) and of the
chrominance Huffman tables, against what the standards and the mathematics
fix rather than against the oracle itself:
- the colour transform is T.871's (JFIF) equations to within rounding, and
  maps greys to (v, 128, 128) exactly; the inverse undoes it to within the
  roundings of both directions;
- a grey image takes the luminance path only: its 4:2:0 layer equals the
  pinned 4:4:4 round trip of its plane;
- constant colours keep DC levels only, and chroma constant over 2x2
  pixels survives the subsampling exactly at Q = 100;
- the chrominance code lengths form complete prefix codes but for the
  reserved all-ones code, over exactly the valid symbols, and price
  hand-worked blocks;
- K.2's chrominance table at Q = 50."""
import numpy as np
import pytest

from oracle import oracle as O


def test_chroma_code_lengths_are_complete_prefix_codes():
    dc = [O.jpeg_dc_len_c(c) for c in range(12)]
    assert sum(2.0 ** -l for l in dc) == 1.0 - 2.0 ** -11
    valid = {0x00, 0xF0} | {(r << 4) | s for r in range(16) for s in range(1, 11)}
    lens = {sym: O.jpeg_ac_len_c(sym) for sym in range(256)}
    assert {s for s, l in lens.items() if l > 0} == valid
    assert sum(2.0 ** -lens[s] for s in valid) == 1.0 - 2.0 ** -16


def test_chroma_quantiser_at_q50_is_annex_k2():
    q = O.quant_table_chroma(50)
    assert list(q[0]) == [17, 18, 24, 47, 99, 99, 99, 99]
    assert list(q[:, 0]) == [17, 18, 24, 47, 99, 99, 99, 99]
    assert (q[4:] == 99).all() and (O.quant_table_chroma(100) == 1).all()
    # the IJG rule at Q = 75: half of each step, halves rounded up (17 -> 9, 47 -> 24, 99 -> 50)
    assert np.array_equal(O.quant_table_chroma(75), (q + 1) // 2)


def test_colour_transform_is_t871_within_rounding():
    rng = np.random.default_rng(1)
    rgb = rng.integers(0, 256, size=(3, 4000)).astype(np.uint8)
    ycc = O.rgb_to_ycc(rgb).astype(np.float64)
    r, g, b = rgb.astype(np.float64)
    y = 0.299 * r + 0.587 * g + 0.114 * b
    cb = -0.299 / 1.772 * r - 0.587 / 1.772 * g + 0.5 * b + 128
    cr = 0.5 * r - 0.587 / 1.402 * g - 0.114 / 1.402 * b + 128
    # rounding to an integer (1/2) plus three 16-bit weights, each within half a unit of 65536 c
    bound = 0.5 + 3 * 0.5 * 255 / 65536
    for got, want in ((ycc[0], y), (ycc[1], np.clip(cb, 0, 255)), (ycc[2], np.clip(cr, 0, 255))):
        assert np.abs(got - want).max() <= bound
    grey = np.tile(np.arange(256, dtype=np.uint8), (3, 1))
    assert np.array_equal(O.rgb_to_ycc(grey), np.stack([np.arange(256), np.full(256, 128), np.full(256, 128)]))
    # T.871's weight 1/2 is exact: pure blue has Cb = 128 + B / 2 and pure red
    # Cr = 128 + R / 2, halves rounded up, clamped to 255
    v = np.arange(256)
    blue = np.stack([np.zeros(256), np.zeros(256), v]).astype(np.uint8)
    red = np.stack([v, np.zeros(256), np.zeros(256)]).astype(np.uint8)
    assert np.array_equal(O.rgb_to_ycc(blue)[1], np.minimum(128 + (v + 1) // 2, 255))
    assert np.array_equal(O.rgb_to_ycc(red)[2], np.minimum(128 + (v + 1) // 2, 255))


def test_inverse_colour_transform_is_t871_within_rounding():
    # every (Cb, Cr) pair at five luma values against T.871's real-valued
    # inverse; the bound is the rounding to an integer plus the 16-bit
    # weights, each within half a unit of 65536 c, over |Cb - 128|, |Cr - 128| <= 128
    cb, cr = [a.reshape(-1) for a in np.meshgrid(np.arange(256), np.arange(256))]
    for y in (0, 61, 128, 200, 255):
        ycc = np.stack([np.full(cb.size, y), cb, cr]).astype(np.uint8)
        rgb = O.ycc_to_rgb(ycc).astype(np.float64)
        dcb, dcr = cb - 128.0, cr - 128.0
        want = (y + 1.402 * dcr, y - 0.344136 * dcb - 0.714136 * dcr, y + 1.772 * dcb)
        for got, exact, nw in zip(rgb, want, (1, 2, 1)):
            assert np.abs(got - np.clip(exact, 0, 255)).max() <= 0.5 + nw * 0.5 * 128 / 65536
    # neutral chroma leaves the luma as it is
    grey = np.stack([np.arange(256), np.full(256, 128), np.full(256, 128)]).astype(np.uint8)
    assert np.array_equal(O.ycc_to_rgb(grey), np.tile(np.arange(256, dtype=np.uint8), (3, 1)))


def test_chroma_subsampling_rounds_the_2x2_mean_half_up():
    # rows alternate black and (0, 0, 2): Y = 0 and Cr = 128 for both, Cb = 128
    # and 129, so every 2x2 chroma mean is 128.5, taken half up to 129; the
    # subsampled planes are constant, and at Q = 100 (every step 1) a constant
    # block's only level is its DC, 8 (m - 128)
    h, w = 16, 32
    rgb = np.zeros((3, h, w), np.uint8)
    rgb[2, 1::2] = 2
    ycc = O.rgb_to_ycc(rgb.reshape(3, -1)).reshape(3, h, w)
    assert (ycc[0] == 0).all() and (ycc[2] == 128).all()
    assert (ycc[1, 0::2] == 128).all() and (ycc[1, 1::2] == 129).all()
    _, lv = O.base_roundtrip_420(rgb, 100)
    nbY, nbC = O.blocks_420(h, w)
    cb_blocks, cr_blocks = lv[nbY:nbY + nbC], lv[nbY + nbC:]
    assert (cb_blocks[:, 0] == 8 * (129 - 128)).all() and (cb_blocks[:, 1:] == 0).all()
    assert (cr_blocks == 0).all()


def test_grey_images_take_the_luminance_path_only():
    rng = np.random.default_rng(2)
    for h, w, q in [(8, 8, 50), (13, 21, 75), (30, 17, 10)]:
        plane = rng.integers(0, 256, size=(h, w)).astype(np.uint8)
        grey = np.stack([plane] * 3)
        s3, lv = O.base_roundtrip_420(grey, q)
        ref = O.base_roundtrip(grey, q)                 # 4:4:4, every plane with the luminance table
        assert np.array_equal(s3, ref)
        nbY, nbC = O.blocks_420(h, w)
        # chroma is 128 everywhere: its levels are all zero
        assert (lv[nbY:] == 0).all()


def test_constant_colours_and_blocky_chroma():
    s3, lv = O.base_roundtrip_420(np.stack([np.full((16, 24), v, np.uint8) for v in (200, 30, 90)]), 50)
    assert (lv[:, 1:] == 0).all()
    # colour constant on 2x2 pixels loses nothing to the subsampling: at Q = 100 every plane's round
    # trip is within 1 (the 4:4:4 pin), each transform rounds by 1/2, so with the inverse weights
    # (1.402, 0.344 + 0.714, 1.772) R and B stay within 4 and G within 3 of the input
    rng = np.random.default_rng(3)
    small = rng.integers(40, 216, size=(3, 8, 12)).astype(np.uint8)
    img = small.repeat(2, axis=1).repeat(2, axis=2)
    s3, _ = O.base_roundtrip_420(img, 100)
    err = np.abs(s3.astype(int) - img.astype(int)).max(axis=(1, 2))
    assert err[0] <= 4 and err[1] <= 3 and err[2] <= 4
    # a colour edge inside a 2x2 cell is averaged away: chroma cannot follow it
    edge = np.zeros((3, 16, 16), np.uint8)
    edge[0, :, 1::2] = 255
    s_edge, _ = O.base_roundtrip_420(edge, 100)
    assert np.abs(s_edge[0].astype(int)[:, 1::2] - 255).max() > 40


def test_hand_worked_chroma_block_costs():
    # one luminance and one chroma plane of two blocks each
    lv = np.zeros((4, 64), np.int16)
    lv[2, 0] = 3                      # chroma block 0: DC diff 3 (category 2)
    lv[3, 0] = 3                      # chroma block 1: diff 0; zigzag 1 = 1: symbol 0x01
    lv[3, 8] = 1
    bits, blk = O.jpeg_bits_planes(lv, [2, 2], [0, 1])
    assert list(blk[:2]) == [2 + 4, 2 + 4]              # luminance: DC 0 (2), EOB (4)
    assert blk[2] == 2 + 2 + 2                           # chroma DC category 2: 2-bit code + 2; EOB 2 bits
    assert blk[3] == 2 + 2 + 1 + 2                       # chroma DC 0 (2), 0x01 (2) + 1, EOB (2)
    assert list(bits) == [12, 13]
