"""slr_fit_noalloc: the fit for callers that cannot allocate device memory.

Such callers (a plugin whose host application owns all device memory, a
service that allocates nothing after start-up, C code that only receives
device pointers) cannot hand slr_fit its bin_sums workspace; this entry point
keeps the sums in the library's static device array instead.  The test calls
it through the C ABI twice in a row on different images and checks each
result against slr_fit with a caller workspace.  The tolerance is the one
every parity test here uses: bit-exact.  The second call also shows that the
shared array is cleared between calls.  This file is collected last so that
a run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest
import torch

from paper_2309_11072_gb300 import codec, native, synth

pytestmark = pytest.mark.gpu


def _planes(h, w, seed, quality):
    """Decoded SDRI, mantissa and exponent planes of a synthetic image, on the GPU."""
    img = synth.make_rgbe(h, w, seed=seed, lo=-3.0, hi=5.0, rects=4, highlights=8)
    c = codec.Codec(h, w, "cuda")
    c.encode(torch.from_numpy(img.view(np.int32).reshape(-1).copy()).cuda(), quality)
    return c


def _fit_both(c, gf_on):
    with_ws = torch.zeros(native.PARAMS_BYTES // 4, dtype=torch.int32, device="cuda")
    without = torch.full((native.PARAMS_BYTES // 4,), -1, dtype=torch.int32, device="cuda")
    sums = torch.empty(native.slr_fit_workspace_bytes() // 8, dtype=torch.int64, device="cuda")
    native.slr_fit(c.s3, c.m3, c.e, c.h, c.w, gf_on, sums, with_ws)
    native.slr_fit_noalloc(c.s3, c.m3, c.e, c.h, c.w, gf_on, without)
    torch.cuda.synchronize()
    return codec.params_to_numpy(with_ws), codec.params_to_numpy(without)


def test_noalloc_fit_matches_workspace_fit_twice_in_a_row():
    assert torch.cuda.is_available()
    native.lib()
    first = _planes(300, 412, seed=31, quality=75)      # ragged width: scalar paths
    second = _planes(256, 512, seed=32, quality=90)     # vector paths, other regions
    for c, gf_on in ((first, 1), (second, 0)):
        ref, got = _fit_both(c, gf_on)
        assert got["n_used"] == ref["n_used"] > 0
        assert np.array_equal(got["n"], ref["n"])
        assert np.array_equal(got["a"].view(np.uint32), ref["a"].view(np.uint32))
        assert np.array_equal(got["b"].view(np.uint32), ref["b"].view(np.uint32))


def test_noalloc_fit_rejects_oversized_image():
    L = native.lib()
    params = torch.zeros(native.PARAMS_BYTES // 4, dtype=torch.int32, device="cuda")
    rc = L.slr_fit_noalloc(1, 1, 1, 65536, 32768, 1, params.data_ptr(), None)    # h*w = 2^31
    assert rc == -1 and "supported size" in native.last_error()
