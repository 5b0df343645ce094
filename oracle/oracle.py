"""Python face of the CPU oracle (``slrme_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  The product path never imports this
module.  Every function is a thin numpy <-> C marshalling wrapper; the
arithmetic, with its citations to the paper, lives in the C file.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "slrme_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, IEEE arithmetic, no contraction).
    SLRME_ORACLE_LIB names an already built library to load instead (the
    mutation tests load deliberately broken copies of the oracle this way)."""
    alt = os.environ.get("SLRME_ORACLE_LIB")
    if alt:
        return alt
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _lib.oracle_i128_to_double_parts.restype = ctypes.c_double
            _lib.oracle_i128_to_double_parts.argtypes = [ctypes.c_int64, ctypes.c_uint64]
            _lib.oracle_rgbe_from_float.restype = ctypes.c_int
            _lib.oracle_base_roundtrip.restype = ctypes.c_int
            _lib.oracle_rans_table.restype = ctypes.c_int
            _lib.oracle_rans_encode.restype = ctypes.c_int
            _lib.oracle_rans_encode.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_void_p]
            _lib.oracle_rans_decode.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                                ctypes.c_void_p]
            _lib.oracle_rans_encode_segments.restype = ctypes.c_int
            _lib.oracle_rans_encode_segments.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            _lib.oracle_rans_decode_segments.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            _lib.oracle_white_point.restype = ctypes.c_float
            _lib.oracle_white_point.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32]
            _lib.oracle_tmo_white.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                              ctypes.c_float, ctypes.c_void_p]
            _lib.oracle_base_levels.restype = ctypes.c_int
            _lib.oracle_jpeg_bits.restype = ctypes.c_int
            _lib.oracle_jpeg_ac_len.restype = ctypes.c_int
            _lib.oracle_jpeg_dc_len.restype = ctypes.c_int
            _lib.oracle_jpeg_ac_len_c.restype = ctypes.c_int
            _lib.oracle_jpeg_dc_len_c.restype = ctypes.c_int
            _lib.oracle_jpeg_bits_planes.restype = ctypes.c_int
            _lib.oracle_base_roundtrip_420.restype = ctypes.c_int
            _lib.oracle_rgb_to_ycc.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
            _lib.oracle_dwt53_bands.restype = ctypes.c_int
            _lib.oracle_dwt53_forward.restype = ctypes.c_int
            _lib.oracle_dwt53_inverse.restype = ctypes.c_int
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
    return ctypes.c_void_p(a.ctypes.data)


NBIN, NSUM, NRES = 256, 13, 511


# ---------------------------------------------------------------- format
def rgbe_from_float(f: np.ndarray) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty(f.shape[:-1], dtype=np.uint32)
    rc = lib().oracle_rgbe_from_float(_p(f), ctypes.c_int64(out.size), _p(out))
    if rc != 0:
        raise ValueError("exponent outside [1, 255]")
    return out


def rgbe_to_float(rgbe: np.ndarray) -> np.ndarray:
    rgbe = np.ascontiguousarray(rgbe, dtype=np.uint32)
    out = np.empty(rgbe.shape + (3,), dtype=np.float64)
    lib().oracle_rgbe_to_float(_p(rgbe), ctypes.c_int64(rgbe.size), _p(out))
    return out


def rgbe_split(rgbe: np.ndarray):
    rgbe = np.ascontiguousarray(rgbe, dtype=np.uint32)
    m3 = np.empty((3,) + rgbe.shape, dtype=np.uint8)
    e = np.empty(rgbe.shape, dtype=np.uint8)
    lib().oracle_rgbe_split(_p(rgbe), ctypes.c_int64(rgbe.size), _p(m3), _p(e))
    return m3, e


# ---------------------------------------------------------------- tables
def log2_table() -> np.ndarray:
    t = np.empty(2048, dtype=np.int32)
    lib().oracle_log2_table(_p(t))
    return t


def gamma_thresholds() -> np.ndarray:
    t = np.empty(256, dtype=np.float32)
    lib().oracle_gamma_thresholds(_p(t))
    return t


def key_tables():
    kr = np.empty(16, dtype=np.float32)
    wr = np.empty(16, dtype=np.float32)
    lib().oracle_key_tables(_p(kr), _p(wr))
    return kr, wr


def quant_table(quality: int) -> np.ndarray:
    q = np.empty(64, dtype=np.int32)
    lib().oracle_quant_table(ctypes.c_int(quality), _p(q))
    return q.reshape(8, 8)


def dct_matrix() -> np.ndarray:
    d = np.empty(64, dtype=np.int32)
    lib().oracle_dct_matrix(_p(d))
    return d.reshape(8, 8)


# ---------------------------------------------------------------- base layer
def lum_stats(rgbe: np.ndarray) -> np.ndarray:
    rgbe = np.ascontiguousarray(rgbe, dtype=np.uint32)
    st = np.zeros(2, dtype=np.int64)
    lib().oracle_lum_stats(_p(rgbe), ctypes.c_int64(rgbe.size), _p(st))
    return st


def key(stats: np.ndarray):
    stats = np.ascontiguousarray(stats, dtype=np.int64)
    J = ctypes.c_int32()
    r = ctypes.c_int32()
    lib().oracle_key(_p(stats), ctypes.byref(J), ctypes.byref(r))
    return J.value, r.value


def tmo(rgbe: np.ndarray, J: int, r: int) -> np.ndarray:
    rgbe = np.ascontiguousarray(rgbe, dtype=np.uint32)
    sdr3 = np.empty((3,) + rgbe.shape, dtype=np.uint8)
    lib().oracle_tmo(_p(rgbe), ctypes.c_int64(rgbe.size), ctypes.c_int32(J), ctypes.c_int32(r), _p(sdr3))
    return sdr3


def white_point(rgbe: np.ndarray, J: int, r: int) -> np.float32:
    """The largest scaled luminance L of the image (the white point of the operator's Eq. 4 form)."""
    rgbe = np.ascontiguousarray(rgbe, dtype=np.uint32)
    return np.float32(lib().oracle_white_point(_p(rgbe), ctypes.c_int64(rgbe.size), ctypes.c_int32(J),
                                               ctypes.c_int32(r)))


def tmo_white(rgbe: np.ndarray, J: int, r: int, l_white: float) -> np.ndarray:
    """Display codes of Reinhard's operator with white point l_white (float32)."""
    rgbe = np.ascontiguousarray(rgbe, dtype=np.uint32)
    sdr3 = np.empty((3,) + rgbe.shape, dtype=np.uint8)
    lib().oracle_tmo_white(_p(rgbe), ctypes.c_int64(rgbe.size), ctypes.c_int32(J), ctypes.c_int32(r),
                           ctypes.c_float(l_white), _p(sdr3))
    return sdr3


def base_roundtrip(sdr3: np.ndarray, quality: int) -> np.ndarray:
    sdr3 = np.ascontiguousarray(sdr3, dtype=np.uint8)
    _, h, w = sdr3.shape
    s3 = np.empty_like(sdr3)
    rc = lib().oracle_base_roundtrip(_p(sdr3), ctypes.c_int(h), ctypes.c_int(w), ctypes.c_int(quality), _p(s3))
    if rc != 0:
        raise ValueError("quality must be in [1, 100]")
    return s3


# ---------------------------------------------------------------- SLRME
def gf(s3: np.ndarray, gf_on: bool = True) -> np.ndarray:
    s3 = np.ascontiguousarray(s3, dtype=np.uint8)
    _, h, w = s3.shape
    x3 = np.empty((3, h, w), dtype=np.int32)
    lib().oracle_gf(_p(s3), ctypes.c_int(h), ctypes.c_int(w), ctypes.c_int(int(gf_on)), _p(x3))
    return x3


def bin_sums(x3: np.ndarray, m3: np.ndarray, e: np.ndarray) -> np.ndarray:
    x3 = np.ascontiguousarray(x3, dtype=np.int32)
    m3 = np.ascontiguousarray(m3, dtype=np.uint8)
    e = np.ascontiguousarray(e, dtype=np.uint8)
    sums = np.empty((NBIN, NSUM), dtype=np.int64)
    lib().oracle_bin_sums(_p(x3), _p(m3), _p(e), ctypes.c_int64(e.size), _p(sums))
    return sums


def i128_to_double(v: int) -> float:
    lo = v & ((1 << 64) - 1)
    hi = v >> 64
    return lib().oracle_i128_to_double_parts(ctypes.c_int64(hi), ctypes.c_uint64(lo))


def solve(sums: np.ndarray):
    """Returns (a[3,256] f32, b[3,256] f32, n[256] i32, n_used)."""
    sums = np.ascontiguousarray(sums, dtype=np.int64)
    a = np.empty((3, NBIN), dtype=np.float32)
    b = np.empty((3, NBIN), dtype=np.float32)
    n = np.empty(NBIN, dtype=np.int32)
    nu = ctypes.c_int32()
    lib().oracle_solve(_p(sums), _p(a), _p(b), _p(n), ctypes.byref(nu))
    return a, b, n, nu.value


def predict(x3: np.ndarray, e: np.ndarray, a: np.ndarray, b: np.ndarray) -> np.ndarray:
    x3 = np.ascontiguousarray(x3, dtype=np.int32)
    e = np.ascontiguousarray(e, dtype=np.uint8)
    a = np.ascontiguousarray(a, dtype=np.float32)
    b = np.ascontiguousarray(b, dtype=np.float32)
    ms = np.empty(x3.shape, dtype=np.uint8)
    lib().oracle_predict(_p(x3), _p(e), ctypes.c_int64(e.size), _p(a), _p(b), _p(ms))
    return ms


def residual(m3: np.ndarray, mstar3: np.ndarray):
    m3 = np.ascontiguousarray(m3, dtype=np.uint8)
    mstar3 = np.ascontiguousarray(mstar3, dtype=np.uint8)
    r3 = np.empty(m3.shape, dtype=np.int16)
    hist = np.empty((3, NRES), dtype=np.uint32)
    lib().oracle_residual(_p(m3), _p(mstar3), ctypes.c_int64(m3[0].size), _p(r3), _p(hist))
    return r3, hist


def decode(s3: np.ndarray, e: np.ndarray, r3: np.ndarray, a: np.ndarray, b: np.ndarray,
           gf_on: bool = True) -> np.ndarray:
    s3 = np.ascontiguousarray(s3, dtype=np.uint8)
    e = np.ascontiguousarray(e, dtype=np.uint8)
    r3 = np.ascontiguousarray(r3, dtype=np.int16)
    a = np.ascontiguousarray(a, dtype=np.float32)
    b = np.ascontiguousarray(b, dtype=np.float32)
    _, h, w = s3.shape
    out = np.empty((h, w), dtype=np.uint32)
    lib().oracle_decode(_p(s3), _p(e), _p(r3), ctypes.c_int(h), ctypes.c_int(w), ctypes.c_int(int(gf_on)),
                        _p(a), _p(b), _p(out))
    return out


# ---------------------------------------------------------------- pipeline
def encode(rgbe: np.ndarray, quality: int, gf_on: bool = True) -> dict:
    """Whole encoder (Fig. 2, bottom): split, TMO, base round trip, SLRME fit,
    prediction and residual.  Returns every intermediate."""
    rgbe = np.ascontiguousarray(rgbe, dtype=np.uint32)
    m3, e = rgbe_split(rgbe)
    st = lum_stats(rgbe)
    J, r = key(st)
    sdr3 = tmo(rgbe, J, r)
    s3 = base_roundtrip(sdr3, quality)
    x3 = gf(s3, gf_on)
    sums = bin_sums(x3, m3, e)
    a, b, n, n_used = solve(sums)
    ms = predict(x3, e, a, b)
    r3, hist = residual(m3, ms)
    return dict(m3=m3, e=e, stats=st, J=J, r=r, sdr3=sdr3, s3=s3, x3=x3, sums=sums,
                a=a, b=b, n=n, n_used=n_used, mstar3=ms, r3=r3, hist=hist)


def entropy_bits(hist: np.ndarray) -> float:
    """Order-0 entropy (bits per symbol) of one histogram, float64."""
    h = np.asarray(hist, dtype=np.float64)
    tot = h.sum()
    if tot == 0:
        return 0.0
    p = h[h > 0] / tot
    return float(-(p * np.log2(p)).sum())


# ---------------------------------------------------------------- enhancement-layer coder (rANS)
RANS_CHUNK, RANS_LANES, RANS_CAP = 8192, 32, 8192 // 32 + 2


def rans_table(counts: np.ndarray) -> np.ndarray:
    """Frequency table (total 2^14) of one channel from its residual histogram."""
    c = np.ascontiguousarray(counts, dtype=np.uint32).reshape(NRES)
    f = np.zeros(NRES, np.uint32)
    lib().oracle_rans_table(_p(c), _p(f))
    return f


def rans_layout(n: int):
    chunks = (n + RANS_CHUNK - 1) // RANS_CHUNK
    return chunks, 3 * chunks * RANS_LANES * RANS_CAP, 3 * chunks * RANS_LANES


def rans_encode(r3: np.ndarray, freq3: np.ndarray):
    """Words ([3][chunks] blocks of 32 x 258 uint16, each chunk's streams packed from the start of
    its block) and counts ([3][chunks][32]) of the residual planes; the rest of a block is 0."""
    r = np.ascontiguousarray(r3, dtype=np.int16).reshape(-1)
    n = r.size // 3
    _, nw, nc = rans_layout(n)
    words = np.zeros(nw, np.uint16)
    counts = np.zeros(nc, np.uint32)
    f = np.ascontiguousarray(freq3, dtype=np.uint32).reshape(3 * NRES)
    rc = lib().oracle_rans_encode(_p(r), n, _p(f), _p(words), _p(counts))
    if rc != 0:
        raise ValueError("a residual has a zero frequency in its channel's table")
    return words, counts


def rans_decode(words: np.ndarray, counts: np.ndarray, n: int, freq3: np.ndarray) -> np.ndarray:
    out = np.zeros(3 * n, np.int16)
    f = np.ascontiguousarray(freq3, dtype=np.uint32).reshape(3 * NRES)
    lib().oracle_rans_decode(_p(np.ascontiguousarray(words, dtype=np.uint16)),
                             _p(np.ascontiguousarray(counts, dtype=np.uint32)), n, _p(f), _p(out))
    return out


RANS_RAW = 0xFFFFFFFF


def rans_segment_layout(lengths):
    """Chunks per segment and the words / counts sizes of a run of segments."""
    chunks = [(int(n) + RANS_CHUNK - 1) // RANS_CHUNK for n in lengths]
    total = sum(chunks)
    return chunks, total * RANS_LANES * RANS_CAP, total * RANS_LANES


def rans_encode_segments(sym: np.ndarray, lengths, freq: np.ndarray):
    """Words and counts of a run of segments (segment g: `lengths[g]` symbols, table freq[g]);
    chunks with a value outside -255..255 are stored raw."""
    v = np.ascontiguousarray(sym, dtype=np.int16).reshape(-1)
    ln = np.ascontiguousarray(lengths, dtype=np.int64)
    assert v.size == int(ln.sum())
    _, nw, nc = rans_segment_layout(ln)
    words = np.zeros(nw, np.uint16)
    counts = np.zeros(nc, np.uint32)
    f = np.ascontiguousarray(freq, dtype=np.uint32).reshape(-1)
    assert f.size == NRES * ln.size
    rc = lib().oracle_rans_encode_segments(_p(v), int(ln.size), _p(ln), _p(f), _p(words), _p(counts))
    if rc != 0:
        raise ValueError("a value has a zero frequency in its segment's table")
    return words, counts


def rans_decode_segments(words: np.ndarray, counts: np.ndarray, lengths, freq: np.ndarray) -> np.ndarray:
    ln = np.ascontiguousarray(lengths, dtype=np.int64)
    out = np.zeros(int(ln.sum()), np.int16)
    f = np.ascontiguousarray(freq, dtype=np.uint32).reshape(-1)
    lib().oracle_rans_decode_segments(_p(np.ascontiguousarray(words, dtype=np.uint16)),
                                      _p(np.ascontiguousarray(counts, dtype=np.uint32)), int(ln.size), _p(ln),
                                      _p(f), _p(out))
    return out


def segment_hist(sym: np.ndarray, lengths) -> np.ndarray:
    """Histogram (511 bins, value + 255) of the values inside -255..255 of each segment."""
    v = np.asarray(sym, dtype=np.int64).reshape(-1)
    out, at = [], 0
    for n in lengths:
        seg = v[at:at + int(n)]
        seg = seg[(seg >= -255) & (seg <= 255)] + 255
        out.append(np.bincount(seg, minlength=NRES))
        at += int(n)
    return np.array(out, dtype=np.uint32).reshape(len(out), NRES)


DWT_MAX_LEVELS = 3


def dwt53_bands(h: int, w: int, levels: int):
    """(rows, columns) of each band in output order: LL_L, then HL, LH, HH from level L down to 1."""
    dims = np.zeros(2 * (1 + 3 * DWT_MAX_LEVELS), np.int32)
    nb = lib().oracle_dwt53_bands(ctypes.c_int(h), ctypes.c_int(w), ctypes.c_int(levels), _p(dims))
    return [(int(dims[2 * b]), int(dims[2 * b + 1])) for b in range(nb)]


def dwt53_forward(planes: np.ndarray, levels: int) -> np.ndarray:
    """Reversible 5/3 transform of each plane ([P][h][w] int16) into its subband-major order ([P][h*w])."""
    x = np.ascontiguousarray(planes, dtype=np.int16)
    P, h, w = x.shape
    out = np.zeros((P, h * w), np.int16)
    for c in range(P):
        rc = lib().oracle_dwt53_forward(_p(x[c]), ctypes.c_int(h), ctypes.c_int(w), ctypes.c_int(levels),
                                        _p(out[c]))
        if rc != 0:
            raise ValueError("levels must be in 0..3")
    return out


def dwt53_inverse(coef: np.ndarray, h: int, w: int, levels: int) -> np.ndarray:
    cf = np.ascontiguousarray(coef, dtype=np.int16).reshape(-1, h * w)
    out = np.zeros((cf.shape[0], h, w), np.int16)
    for c in range(cf.shape[0]):
        rc = lib().oracle_dwt53_inverse(_p(cf[c]), ctypes.c_int(h), ctypes.c_int(w), ctypes.c_int(levels),
                                        _p(out[c]))
        if rc != 0:
            raise ValueError("levels must be in 0..3")
    return out


# ---------------------------------------------------------------- base-layer entropy coding (JPEG baseline)
def base_levels(sdr3: np.ndarray, quality: int) -> np.ndarray:
    """Quantised levels of the base round trip: [3][bh*bw][64] int16, coefficient (v, u) at u*8 + v."""
    s = np.ascontiguousarray(sdr3, dtype=np.uint8)
    _, h, w = s.shape
    bh, bw = (h + 7) // 8, (w + 7) // 8
    out = np.zeros((3, bh * bw, 64), np.int16)
    if lib().oracle_base_levels(_p(s), ctypes.c_int(h), ctypes.c_int(w), ctypes.c_int(quality), _p(out)) != 0:
        raise ValueError("quality must be in 1..100")
    return out


def jpeg_bits(levels3: np.ndarray, h: int, w: int):
    """Entropy-coded bits per plane ([3] uint64) and per block ([3][bh*bw] uint32)."""
    L = np.ascontiguousarray(levels3, dtype=np.int16)
    bh, bw = (h + 7) // 8, (w + 7) // 8
    bits = np.zeros(3, np.uint64)
    blk = np.zeros((3, bh * bw), np.uint32)
    if lib().oracle_jpeg_bits(_p(L), ctypes.c_int(h), ctypes.c_int(w), _p(bits), _p(blk)) != 0:
        raise ValueError("a category exceeds the baseline Huffman tables")
    return bits, blk


def zigzag() -> np.ndarray:
    zz = np.zeros(64, np.int32)
    lib().oracle_zigzag(_p(zz))
    return zz


def jpeg_ac_len(sym: int) -> int:
    return int(lib().oracle_jpeg_ac_len(ctypes.c_int(sym)))


def jpeg_dc_len(cat: int) -> int:
    return int(lib().oracle_jpeg_dc_len(ctypes.c_int(cat)))


def jpeg_ac_len_c(sym: int) -> int:
    return int(lib().oracle_jpeg_ac_len_c(ctypes.c_int(sym)))


def jpeg_dc_len_c(cat: int) -> int:
    return int(lib().oracle_jpeg_dc_len_c(ctypes.c_int(cat)))


def jpeg_bits_planes(levels: np.ndarray, nblocks, chroma):
    """Bits per plane and per block of planes with nblocks[p] blocks each, plane p with the chrominance
    tables when chroma[p] (else luminance); levels: the planes' blocks one after another, 64 levels each."""
    L = np.ascontiguousarray(levels, dtype=np.int16).reshape(-1)
    nb = np.ascontiguousarray(nblocks, dtype=np.int64)
    ch = np.ascontiguousarray(chroma, dtype=np.int32)
    assert L.size == 64 * int(nb.sum())
    bits = np.zeros(nb.size, np.uint64)
    blk = np.zeros(int(nb.sum()), np.uint32)
    if lib().oracle_jpeg_bits_planes(_p(L), ctypes.c_int(nb.size), _p(nb), _p(ch), _p(bits), _p(blk)) != 0:
        raise ValueError("a category exceeds the baseline Huffman tables")
    return bits, blk


def quant_table_chroma(quality: int) -> np.ndarray:
    q = np.zeros(64, np.int32)
    lib().oracle_quant_table_chroma(ctypes.c_int(quality), _p(q))
    return q.reshape(8, 8)


def rgb_to_ycc(rgb3: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(rgb3, dtype=np.uint8)
    out = np.zeros_like(x)
    lib().oracle_rgb_to_ycc(_p(x), x[0].size, _p(out))
    return out


def ycc_to_rgb(ycc3: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(ycc3, dtype=np.uint8)
    out = np.zeros_like(x)
    lib().oracle_ycc_to_rgb(_p(x), ctypes.c_int64(x[0].size), _p(out))
    return out


def blocks_420(h: int, w: int):
    """Blocks of the Y plane and of each chroma plane of the 4:2:0 base layer."""
    hc, wc = (h + 1) // 2, (w + 1) // 2
    return ((h + 7) // 8) * ((w + 7) // 8), ((hc + 7) // 8) * ((wc + 7) // 8)


def base_roundtrip_420(sdr3: np.ndarray, quality: int):
    """The YCbCr 4:2:0 base layer: decoded RGB planes and the levels (Y blocks, Cb blocks, Cr blocks)."""
    x = np.ascontiguousarray(sdr3, dtype=np.uint8)
    _, h, w = x.shape
    nbY, nbC = blocks_420(h, w)
    s3 = np.zeros_like(x)
    lv = np.zeros((nbY + 2 * nbC, 64), np.int16)
    if lib().oracle_base_roundtrip_420(_p(x), ctypes.c_int(h), ctypes.c_int(w), ctypes.c_int(quality), _p(s3),
                                       _p(lv)) != 0:
        raise ValueError("quality must be in 1..100")
    return s3, lv
