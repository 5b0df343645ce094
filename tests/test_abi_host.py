"""CPU-only checks of the CUDA library: it builds for sm_103a, loads,
exports every entry point declared in include/*.h, rejects bad arguments
before touching the GPU, and its host-built constant tables equal the
oracle's (built independently) and the closed forms they come from."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest
from scipy.fft import dct

from oracle import oracle as O
from paper_2309_11072_gb300 import native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M):
            if m.group(1) not in ("if", "defined", "sizeof"):
                names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    lib = native.lib()
    names = _declared_functions()
    assert "rgbe_split" in names and "residual_decode" in names and len(names) >= 9
    for name in names:
        assert hasattr(lib, name), f"missing export {name}"


def test_library_is_built_for_sm_103a():
    from paper_2309_11072_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)
    assert os.path.exists(native.library_path())


def test_host_tables_equal_oracle_tables():
    t = native.host_tables(75)
    assert np.array_equal(t["log2_lut"], O.log2_table())
    assert np.array_equal(t["gamma"].view(np.uint32), O.gamma_thresholds().view(np.uint32))
    kr, wr = O.key_tables()
    assert np.array_equal(t["kr"].view(np.uint32), kr.view(np.uint32))
    assert np.array_equal(t["wr"].view(np.uint32), wr.view(np.uint32))
    for q in (1, 25, 50, 75, 90, 100):
        assert np.array_equal(native.host_tables(q)["quant"], O.quant_table(q))


def test_library_dct_constants_against_scipy():
    d = native.host_tables()["dct"]
    ref = np.round(dct(np.eye(8), type=2, norm="ortho", axis=0) * 4096.0)
    assert np.array_equal(d, ref.astype(np.int32))


@pytest.mark.parametrize("num,n", [(0, 0), (5, 1), (-1, 1), (-2049, 3), (10 ** 15, 77777), (-(10 ** 14), 12345)])
def test_key_scale_matches_oracle(num, n):
    assert native.rgbe_key_scale([num, n]) == O.key(np.array([num, n], np.int64))


def test_bad_arguments_rejected_before_any_gpu_work():
    L = native.lib()
    EINVAL = -1
    assert L.rgbe_split(None, 4, 4, None, None, None, None) == EINVAL
    assert L.rgbe_split(None, -1, 4, None, None, None, None) == EINVAL
    assert L.rgbe_split(None, 65536, 32768, None, None, None, None) == EINVAL     # h*w = 2^31
    assert L.sdri_base_roundtrip(1, 1, 8, 8, 1, 0, 1, None, None) == EINVAL       # quality 0
    assert L.sdri_base_roundtrip(1, 1, 8, 8, 1, 101, 1, None, None) == EINVAL     # quality 101
    assert "quality" in native.last_error()
    assert L.slr_fit(1, 1, 1, 8, 8, 2, 1, 1, None) == EINVAL                      # gf_on 2
    assert L.slr_fit(1, 1, 1, 8, 8, 1, None, 1, None) == EINVAL                   # no workspace
    assert L.residual_encode(None, 1, 1, 8, 8, 1, 1, 1, None, None) == EINVAL
    assert L.residual_decode(1, 1, 1, 8, 8, 1, None, 1, None) == EINVAL
    assert L.rgbe_key_scale(None, None, None) == EINVAL
    buf = (ctypes.c_int64 * 2)(0, -5)
    J, r = ctypes.c_int32(), ctypes.c_int32()
    assert L.rgbe_key_scale(ctypes.addressof(buf), ctypes.addressof(J), ctypes.addressof(r)) == EINVAL
    assert native.slr_fit_workspace_bytes() == 256 * 13 * 8


def test_misaligned_typed_pointers_rejected():
    # typed buffers must be naturally aligned; the check runs before any launch
    L = native.lib()
    EINVAL = -1
    assert L.rgbe_split(0x1001, 4, 4, 0x2000, 0x3000, 0x4000, None) == EINVAL      # uint32 words at odd address
    assert L.rgbe_split(0x1000, 4, 4, 0x2000, 0x3000, 0x4004, None) == EINVAL      # int64 stats at 4 mod 8
    assert L.sdri_base_roundtrip(0x1000, 0x2000, 8, 8, 0x3002, 50, 0x4000, None, None) == EINVAL
    assert L.slr_fit(0x1000, 0x2000, 0x3000, 8, 8, 1, 0x4004, 0x5000, None) == EINVAL
    assert L.slr_fit(0x1000, 0x2000, 0x3000, 8, 8, 1, 0x4000, 0x5002, None) == EINVAL
    assert L.residual_encode(0x1000, 0x2000, 0x3000, 8, 8, 1, 0x4000, 0x5001, None, None) == EINVAL
    assert L.residual_encode(0x1000, 0x2000, 0x3000, 8, 8, 1, 0x4000, 0x5000, 0x6002, None) == EINVAL
    assert L.residual_decode(0x1000, 0x2000, 0x3001, 8, 8, 1, 0x4000, 0x5000, None) == EINVAL
    assert L.residual_decode(0x1000, 0x2000, 0x3000, 8, 8, 1, 0x4000, 0x5002, None) == EINVAL
    assert "aligned" in native.last_error()


def test_params_layout_roundtrip():
    from paper_2309_11072_gb300 import codec
    rng = np.random.default_rng(0)
    a = rng.standard_normal((3, 256)).astype(np.float32)
    b = rng.standard_normal((3, 256)).astype(np.float32)
    n = rng.integers(0, 5, 256).astype(np.int32)
    import torch
    p = codec.params_to_numpy(torch.from_numpy(codec.params_from_numpy(a, b, n)))
    assert np.array_equal(p["a"], a) and np.array_equal(p["b"], b) and np.array_equal(p["n"], n)
    assert p["n_used"] == int((n > 0).sum())


def test_batch_struct_layouts_and_argument_checks():
    import ctypes as C
    from paper_2309_11072_gb300 import batch as B
    # the sizes the library's static_asserts fix
    assert C.sizeof(B.BatchImage) == 32 and C.sizeof(B.BatchTiles) == 8
    assert C.sizeof(B.BatchPlan) == 72 and C.sizeof(B.BatchBuffers) == 64
    L = B._lib()
    assert L.slrme_batch_workspace_bytes(0) == 0
    assert L.slrme_batch_workspace_bytes(64) > 64 * 256 * 13 * 8
    imgs = (B.BatchImage * 2)(B.BatchImage(8, 8, 90, 1, 0, 0, 0), B.BatchImage(8, 8, 0, 1, 0, 0, 0))   # quality 0
    plan = B.BatchPlan()
    assert L.slrme_batch_plan_init(C.addressof(plan), C.addressof(imgs), 2, 0x100000, None) == -1
    assert "quality" in native.last_error()
    assert L.slrme_batch_plan_init(C.addressof(plan), C.addressof(imgs), 2, 0x100010, None) == -1   # unaligned
    assert L.slrme_batch_plan_init(C.addressof(plan), C.addressof(imgs), 65536, 0x100000, None) == -1
    assert "at most 65535" in native.last_error()
    assert L.slrme_batch_graph_launch(C.addressof(plan), None) == -1


def test_rans_capacity_matches_the_oracle_layout():
    for n in (0, 1, 31, 8192, 8193, 2048 * 1536, 7680 * 4320):
        _, nw, nc = O.rans_layout(n)
        assert native.rans_words_capacity(n) == nw
        assert native.rans_counts_capacity(n) == nc
    assert native.rans_words_capacity(-5) == 0 and native.rans_counts_capacity(-5) == 0


def test_rans_bad_arguments_rejected_before_any_gpu_work():
    L = native.lib()
    EINVAL = -1
    assert L.rans_tables(None, 64, None) == EINVAL
    assert L.rans_tables(66, 64, None) == EINVAL                     # hist3 not 4-byte aligned
    assert L.rans_encode(None, 10, 64, 64, 64, None) == EINVAL
    assert L.rans_encode(64, 10, 64, 72, 64, None) == EINVAL          # words not 16-byte aligned
    assert L.rans_encode(65, 10, 64, 64, 64, None) == EINVAL          # r3 not 2-byte aligned
    assert L.rans_encode(64, -1, 64, 64, 64, None) == EINVAL
    assert L.rans_encode(64, 1 << 31, 64, 64, 64, None) == EINVAL
    assert L.rans_decode(64, 66, 10, 64, 64, None) == EINVAL          # counts not 4-byte aligned
    assert L.rans_decode(72, 64, 10, 64, 64, None) == EINVAL          # words not 16-byte aligned
    assert L.rans_decode(64, 64, 10, 64, None, None) == EINVAL
    assert "rans_decode" in native.last_error()
    assert L.rans_encode(None, 0, None, None, None, None) == 0        # empty planes: nothing to do


def test_dwt_band_sizes_and_segment_capacities_match_the_oracle():
    for h, w in [(1, 1), (1, 7), (7, 1), (5, 3), (33, 65), (1536, 2048), (4320, 7680)]:
        for levels in (1, 2, 3):
            assert native.dwt53_bands(h, w, levels) == O.dwt53_bands(h, w, levels)
    for lengths in ([1], [8192, 8193, 0, 31], [n for n in range(0, 64 * 100, 100)]):
        _, nw, nc = O.rans_segment_layout(lengths)
        assert native.rans_segments_capacity(lengths) == (nw, nc)


def test_dwt_and_segment_bad_arguments_rejected_before_any_gpu_work():
    L = native.lib()
    EINVAL = -1
    import numpy as np
    assert L.dwt53_forward(64, 3, 8, 8, 0, 128, None, 256, None) == EINVAL        # levels 0
    assert L.dwt53_forward(64, 3, 8, 8, 4, 128, None, 256, None) == EINVAL        # levels 4
    assert L.dwt53_forward(64, 3, 65536, 8, 1, 128, None, 256, None) == EINVAL    # h > 65535
    assert L.dwt53_forward(64, 3, 8, 8, 1, 128, None, 272, None) == EINVAL        # ws not 256-byte aligned
    assert L.dwt53_forward(65, 3, 8, 8, 1, 128, None, 256, None) == EINVAL        # planes misaligned
    assert L.dwt53_inverse(64, 0, 8, 8, 1, 128, 256, None) == EINVAL              # no planes
    assert L.dwt53_bands(8, 8, 0, 64) == EINVAL
    ln = np.array([10, -1], np.int64)
    assert L.rans_encode_segments(64, 2, ln.ctypes.data, 64, 64, 64, None) == EINVAL    # negative length
    ln = np.zeros(65, np.int64)
    assert L.rans_encode_segments(64, 65, ln.ctypes.data, 64, 64, 64, None) == EINVAL   # too many segments
    ln = np.array([100], np.int64)
    assert L.rans_decode_segments(72, 64, 1, ln.ctypes.data, 64, 64, None) == EINVAL    # words misaligned
    assert L.rans_tables_n(64, 0, 64, None) == EINVAL
    assert L.rans_segments_words_capacity(0, ln.ctypes.data) == 0


def test_base_levels_and_jpeg_bits_reject_bad_arguments():
    L = native.lib()
    EINVAL = -1
    assert L.sdri_base_levels(64, 64, 8, 8, 64, 0, 64, 64, None) == EINVAL      # quality 0
    assert L.sdri_base_levels(64, 64, 8, 8, 64, 50, 64, None, None) == EINVAL   # no levels
    assert L.sdri_base_levels(64, 64, 8, 8, 64, 50, 64, 72, None) == EINVAL     # levels not 16-byte aligned
    assert L.jpeg_huffman_bits(64, 8, 8, None, None, None) == EINVAL           # no bits3
    assert L.jpeg_huffman_bits(64, 8, 8, 68, None, None) == EINVAL             # bits3 not 8-byte aligned
    assert L.jpeg_huffman_bits(64, -1, 8, 64, None, None) == EINVAL


def test_420_and_plane_bits_reject_bad_arguments():
    import numpy as np
    L = native.lib()
    EINVAL = -1
    assert L.sdri_base_roundtrip_420(64, 64, 8, 8, 64, 0, 64, None, 256, None) == EINVAL    # quality 0
    assert L.sdri_base_roundtrip_420(64, 64, 8, 8, 64, 50, 64, None, None, None) == EINVAL  # no workspace
    assert L.sdri_base_roundtrip_420(64, 64, 8, 8, 64, 50, 64, 72, 256, None) == EINVAL    # levels misaligned
    assert L.sdri_base_roundtrip_420(64, 64, 131071, 8, 64, 50, 64, None, 256, None) == EINVAL
    nb = np.array([4, 1], np.int64)
    ch = np.array([0, 2], np.int32)
    assert L.jpeg_huffman_bits_planes(64, 2, nb.ctypes.data, ch.ctypes.data, 64, None, None) == EINVAL  # class 2
    ch = np.array([0, 1], np.int32)
    assert L.jpeg_huffman_bits_planes(64, 5, nb.ctypes.data, ch.ctypes.data, 64, None, None) == EINVAL  # 5 planes
    assert L.jpeg_huffman_bits_planes(64, 2, nb.ctypes.data, ch.ctypes.data, 68, None, None) == EINVAL  # bits
    assert native.sdri_base_420_workspace_bytes(1536, 2048) == 1536 * 2048 + 2 * 768 * 1024


def test_white_point_calls_reject_bad_arguments():
    L = native.lib()
    EINVAL = -1
    assert L.sdri_white_point(64, 64, 8, 8, 64, None, None) == EINVAL            # no output
    assert L.sdri_white_point(64, 64, 8, 8, 66, 64, None) == EINVAL              # stats misaligned
    assert L.sdri_base_roundtrip_white(64, 64, 8, 8, 64, None, 50, 64, None, None) == EINVAL   # no white point
    assert L.sdri_base_roundtrip_white(64, 64, 8, 8, 64, 64, 0, 64, None, None) == EINVAL     # quality 0
