"""ctypes binding of the C ABI in ``include/slrme.h``.

Argument marshalling only: each function takes torch CUDA tensors (or raw
device addresses) and forwards pointers, sizes and the stream to the entry
point of the same name in ``_build/libslrme.so``.  A non-zero status raises
``SlrmeError`` with the library's message.  There is no fallback: if the
library cannot be loaded the call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
HEADER = os.path.join(ROOT, "include", "slrme.h")

SLRME_NBIN, SLRME_NSUM, SLRME_NRES = 256, 13, 511
PARAMS_BYTES = 7184


class SlrmeError(RuntimeError):
    def __init__(self, name: str, code: int, msg: str):
        super().__init__(f"{name} failed with status {code}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib: Optional[ctypes.CDLL] = None

_vp, _i32, _i64, _sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
_SIGS = {
    "rgbe_split": [_vp, _i32, _i32, _vp, _vp, _vp, _vp],
    "rgbe_key_scale": [_vp, _vp, _vp],
    "sdri_base_roundtrip": [_vp, _vp, _i32, _i32, _vp, _i32, _vp, _vp, _vp],
    "slr_fit": [_vp, _vp, _vp, _i32, _i32, _i32, _vp, _vp, _vp],
    "slr_fit_noalloc": [_vp, _vp, _vp, _i32, _i32, _i32, _vp, _vp],
    "residual_encode": [_vp, _vp, _vp, _i32, _i32, _i32, _vp, _vp, _vp, _vp],
    "residual_decode": [_vp, _vp, _vp, _i32, _i32, _i32, _vp, _vp, _vp],
    "slrme_host_tables": [_vp, _vp, _vp, _vp, _i32, _vp, _vp],
    "slrme_device_status": [_vp, _i32],
    "slrme_wait_probe": [_i32, _i32, _vp],
    "rans_tables": [_vp, _vp, _vp],
    "rans_encode": [_vp, _i64, _vp, _vp, _vp, _vp],
    "rans_decode": [_vp, _vp, _i64, _vp, _vp, _vp],
    "rans_tables_n": [_vp, _i32, _vp, _vp],
    "rans_encode_segments": [_vp, _i32, _vp, _vp, _vp, _vp, _vp],
    "rans_decode_segments": [_vp, _vp, _i32, _vp, _vp, _vp, _vp],
    "sdri_base_levels": [_vp, _vp, _i32, _i32, _vp, _i32, _vp, _vp, _vp],
    "jpeg_huffman_bits": [_vp, _i32, _i32, _vp, _vp, _vp],
    "jpeg_huffman_bits_planes": [_vp, _i32, _vp, _vp, _vp, _vp, _vp],
    "sdri_white_point": [_vp, _vp, _i32, _i32, _vp, _vp, _vp],
    "sdri_base_roundtrip_white": [_vp, _vp, _i32, _i32, _vp, _vp, _i32, _vp, _vp, _vp],
    "sdri_base_roundtrip_420": [_vp, _vp, _i32, _i32, _vp, _i32, _vp, _vp, _vp, _vp],
    "dwt53_bands": [_i32, _i32, _i32, _vp],
    "dwt53_forward": [_vp, _i32, _i32, _i32, _i32, _vp, _vp, _vp, _vp],
    "dwt53_inverse": [_vp, _i32, _i32, _i32, _i32, _vp, _vp, _vp],
}


def library_path() -> str:
    from . import build
    return build.LIB_PATH


def lib() -> ctypes.CDLL:
    """Load the CUDA library (building it first if the sources are newer)."""
    global _lib
    with _lock:
        if _lib is None:
            from . import build
            path = build.build()
            L = ctypes.CDLL(path)
            for name, args in _SIGS.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int
            L.slrme_last_error.restype = ctypes.c_char_p
            L.slrme_last_error.argtypes = []
            L.slr_fit_workspace_bytes.restype = ctypes.c_size_t
            L.slr_fit_workspace_bytes.argtypes = []
            for name in ("rans_words_capacity", "rans_counts_capacity"):
                fn = getattr(L, name)
                fn.restype = ctypes.c_int64
                fn.argtypes = [_i64]
            for name in ("rans_segments_words_capacity", "rans_segments_counts_capacity"):
                fn = getattr(L, name)
                fn.restype = ctypes.c_int64
                fn.argtypes = [_i32, _vp]
            L.sdri_base_420_workspace_bytes.restype = ctypes.c_size_t
            L.sdri_base_420_workspace_bytes.argtypes = [_i32, _i32]
            L.dwt53_workspace_bytes.restype = ctypes.c_size_t
            L.dwt53_workspace_bytes.argtypes = [_i32, _i32, _i32]
            _lib = L
    return _lib


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_contiguous():
        raise ValueError("the library takes dense planes: pass a contiguous tensor")
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(name: str, code: int) -> None:
    if code != 0:
        raise SlrmeError(name, code, lib().slrme_last_error().decode())


def last_error() -> str:
    return lib().slrme_last_error().decode()


# ---------------------------------------------------------------- entry points

def rgbe_split(rgbe, h: int, w: int, m3, e, lum_stats, stream=None) -> None:
    _check("rgbe_split", lib().rgbe_split(_ptr(rgbe), h, w, _ptr(m3), _ptr(e), _ptr(lum_stats), _stream(stream)))


def rgbe_key_scale(lum_stats_host) -> tuple:
    """Host helper: (J, r) from a host (CPU) pair of int64 statistics."""
    buf = (ctypes.c_int64 * 2)(int(lum_stats_host[0]), int(lum_stats_host[1]))
    J, r = ctypes.c_int32(), ctypes.c_int32()
    _check("rgbe_key_scale", lib().rgbe_key_scale(ctypes.addressof(buf), ctypes.addressof(J), ctypes.addressof(r)))
    return J.value, r.value


def sdri_base_roundtrip(m3, e, h: int, w: int, lum_stats, quality: int, s_dec3, sdr3=None, stream=None) -> None:
    _check("sdri_base_roundtrip", lib().sdri_base_roundtrip(_ptr(m3), _ptr(e), h, w, _ptr(lum_stats), quality,
                                                            _ptr(s_dec3), _ptr(sdr3), _stream(stream)))


def slr_fit(s_dec3, m3, e, h: int, w: int, gf_on: int, bin_sums, params, stream=None) -> None:
    _check("slr_fit", lib().slr_fit(_ptr(s_dec3), _ptr(m3), _ptr(e), h, w, int(gf_on), _ptr(bin_sums),
                                    _ptr(params), _stream(stream)))


def slr_fit_noalloc(s_dec3, m3, e, h: int, w: int, gf_on: int, params, stream=None) -> None:
    """slr_fit without a caller workspace: the library's static device scratch
    holds the bin sums (for callers that cannot allocate device memory)."""
    _check("slr_fit_noalloc", lib().slr_fit_noalloc(_ptr(s_dec3), _ptr(m3), _ptr(e), h, w, int(gf_on),
                                                    _ptr(params), _stream(stream)))


def slr_fit_workspace_bytes() -> int:
    return int(lib().slr_fit_workspace_bytes())


def residual_encode(s_dec3, m3, e, h: int, w: int, gf_on: int, params, r3, hist=None, stream=None) -> None:
    _check("residual_encode", lib().residual_encode(_ptr(s_dec3), _ptr(m3), _ptr(e), h, w, int(gf_on),
                                                    _ptr(params), _ptr(r3), _ptr(hist), _stream(stream)))


def residual_decode(s_dec3, e, r3, h: int, w: int, gf_on: int, params, rgbe_out, stream=None) -> None:
    _check("residual_decode", lib().residual_decode(_ptr(s_dec3), _ptr(e), _ptr(r3), h, w, int(gf_on),
                                                    _ptr(params), _ptr(rgbe_out), _stream(stream)))


def rans_words_capacity(n: int) -> int:
    return int(lib().rans_words_capacity(int(n)))


def rans_counts_capacity(n: int) -> int:
    return int(lib().rans_counts_capacity(int(n)))


def rans_tables(hist3, freq3, stream=None) -> None:
    _check("rans_tables", lib().rans_tables(_ptr(hist3), _ptr(freq3), _stream(stream)))


def rans_encode(r3, n: int, freq3, words, counts, stream=None) -> None:
    _check("rans_encode", lib().rans_encode(_ptr(r3), int(n), _ptr(freq3), _ptr(words), _ptr(counts),
                                            _stream(stream)))


def rans_decode(words, counts, n: int, freq3, r3, stream=None) -> None:
    _check("rans_decode", lib().rans_decode(_ptr(words), _ptr(counts), int(n), _ptr(freq3), _ptr(r3),
                                            _stream(stream)))


def sdri_base_levels(m3, e, h: int, w: int, lum_stats, quality: int, s_dec3, levels3, stream=None) -> None:
    _check("sdri_base_levels", lib().sdri_base_levels(_ptr(m3), _ptr(e), h, w, _ptr(lum_stats), quality, _ptr(s_dec3),
                                                      _ptr(levels3), _stream(stream)))


def jpeg_huffman_bits(levels3, h: int, w: int, bits3, block_bits=None, stream=None) -> None:
    _check("jpeg_huffman_bits", lib().jpeg_huffman_bits(_ptr(levels3), h, w, _ptr(bits3), _ptr(block_bits),
                                                        _stream(stream)))


def sdri_white_point(m3, e, h: int, w: int, lum_stats, l_white, stream=None) -> None:
    _check("sdri_white_point", lib().sdri_white_point(_ptr(m3), _ptr(e), h, w, _ptr(lum_stats), _ptr(l_white),
                                                      _stream(stream)))


def sdri_base_roundtrip_white(m3, e, h: int, w: int, lum_stats, l_white, quality: int, s_dec3, sdr3=None,
                              stream=None) -> None:
    _check("sdri_base_roundtrip_white", lib().sdri_base_roundtrip_white(_ptr(m3), _ptr(e), h, w, _ptr(lum_stats),
                                                                        _ptr(l_white), quality, _ptr(s_dec3),
                                                                        _ptr(sdr3), _stream(stream)))


def jpeg_huffman_bits_planes(levels, nblocks, chroma, bits, block_bits=None, stream=None) -> None:
    import numpy as np
    nb = np.ascontiguousarray(nblocks, dtype=np.int64)
    ch = np.ascontiguousarray(chroma, dtype=np.int32)
    _check("jpeg_huffman_bits_planes", lib().jpeg_huffman_bits_planes(_ptr(levels), int(nb.size), nb.ctypes.data,
                                                                      ch.ctypes.data, _ptr(bits), _ptr(block_bits),
                                                                      _stream(stream)))


def sdri_base_420_workspace_bytes(h: int, w: int) -> int:
    return int(lib().sdri_base_420_workspace_bytes(int(h), int(w)))


def sdri_base_roundtrip_420(m3, e, h: int, w: int, lum_stats, quality: int, s_dec3, levels, ws, stream=None) -> None:
    _check("sdri_base_roundtrip_420", lib().sdri_base_roundtrip_420(_ptr(m3), _ptr(e), h, w, _ptr(lum_stats), quality,
                                                                    _ptr(s_dec3), _ptr(levels), _ptr(ws),
                                                                    _stream(stream)))


def _lengths(lengths):
    """The segment lengths as a host int64 array (kept alive by the caller's reference)."""
    import numpy as np
    return np.ascontiguousarray(np.asarray(lengths, dtype=np.int64).reshape(-1))


def rans_segments_capacity(lengths) -> tuple:
    """(uint16 words, uint32 counts) of a run of segments."""
    ln = _lengths(lengths)
    return (int(lib().rans_segments_words_capacity(int(ln.size), ln.ctypes.data)),
            int(lib().rans_segments_counts_capacity(int(ln.size), ln.ctypes.data)))


def rans_tables_n(hist, ntables: int, freq, stream=None) -> None:
    _check("rans_tables_n", lib().rans_tables_n(_ptr(hist), int(ntables), _ptr(freq), _stream(stream)))


def rans_encode_segments(sym, lengths, freq, words, counts, stream=None) -> None:
    ln = _lengths(lengths)
    _check("rans_encode_segments", lib().rans_encode_segments(_ptr(sym), int(ln.size), ln.ctypes.data, _ptr(freq),
                                                              _ptr(words), _ptr(counts), _stream(stream)))


def rans_decode_segments(words, counts, lengths, freq, sym, stream=None) -> None:
    ln = _lengths(lengths)
    _check("rans_decode_segments", lib().rans_decode_segments(_ptr(words), _ptr(counts), int(ln.size),
                                                              ln.ctypes.data, _ptr(freq), _ptr(sym),
                                                              _stream(stream)))


def dwt53_bands(h: int, w: int, levels: int) -> list:
    """(rows, columns) of each band of a plane in output order."""
    import numpy as np
    dims = np.zeros(2 * 10, np.int32)
    nb = lib().dwt53_bands(int(h), int(w), int(levels), dims.ctypes.data)
    if nb < 0:
        raise SlrmeError("dwt53_bands", nb, last_error())
    return [(int(dims[2 * b]), int(dims[2 * b + 1])) for b in range(nb)]


def dwt53_workspace_bytes(nplanes: int, h: int, w: int) -> int:
    return int(lib().dwt53_workspace_bytes(int(nplanes), int(h), int(w)))


def dwt53_forward(planes, nplanes: int, h: int, w: int, levels: int, coef, hist, ws, stream=None) -> None:
    _check("dwt53_forward", lib().dwt53_forward(_ptr(planes), int(nplanes), int(h), int(w), int(levels), _ptr(coef),
                                                _ptr(hist), _ptr(ws), _stream(stream)))


def dwt53_inverse(coef, nplanes: int, h: int, w: int, levels: int, planes, ws, stream=None) -> None:
    _check("dwt53_inverse", lib().dwt53_inverse(_ptr(coef), int(nplanes), int(h), int(w), int(levels), _ptr(planes),
                                                _ptr(ws), _stream(stream)))


def device_status(clear: bool = True) -> int:
    """The library's device status word (0 = fine); see include/slrme.h."""
    v = ctypes.c_int(-1)
    _check("slrme_device_status", lib().slrme_device_status(ctypes.addressof(v), int(clear)))
    return v.value


# Code of the SlrmeError raised for a non-zero device status word (the library
# reports a bounded wait that gave up through slrme_device_status, not as the
# return code of a call: the call had already returned when the wait ran).
DEVICE_STATUS_ERROR = -4


def check_device_status(where: str) -> None:
    """Waits for the device, then reads and clears the library's status word;
    raises SlrmeError if a kernel's bounded wait gave up since the last check
    (the outputs of the calls since then are then incomplete)."""
    import torch
    torch.cuda.synchronize()
    st = device_status(clear=True)
    if st != 0:
        raise SlrmeError(where, DEVICE_STATUS_ERROR, f"device status word {st:#x}: a kernel's bounded wait gave up; "
                                    "the outputs of the calls since the last check are incomplete")


def wait_probe(max_spins: int, arrive: bool, stream=None) -> None:
    """Launches the library's bounded-wait self-test (see slrme_wait_probe)."""
    _check("slrme_wait_probe", lib().slrme_wait_probe(int(max_spins), int(bool(arrive)), _stream(stream)))


def host_tables(quality: int = 50) -> dict:
    """The library's own constant tables (host code, no GPU)."""
    import numpy as np
    lut = np.empty(2048, np.int32)
    gam = np.empty(256, np.float32)
    kr = np.empty(16, np.float32)
    wr = np.empty(16, np.float32)
    q = np.empty(64, np.int32)
    d = np.empty(64, np.int32)
    _check("slrme_host_tables", lib().slrme_host_tables(lut.ctypes.data, gam.ctypes.data, kr.ctypes.data,
                                                        wr.ctypes.data, quality, q.ctypes.data, d.ctypes.data))
    return dict(log2_lut=lut, gamma=gam, kr=kr, wr=wr, quant=q.reshape(8, 8), dct=d.reshape(8, 8))
