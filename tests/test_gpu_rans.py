"""GPU parity of the enhancement-layer rANS coder against the oracle: the
frequency tables, every word and count of the bitstream bit for bit, the
lossless decode, cross-decoding (GPU words by the oracle and the reverse),
and the corrupt-input reports through the device status word."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2309_11072_gb300 import codec, native, synth

pytestmark = pytest.mark.gpu

NRES = 511
STATUS_RANS = 2


def _gpu_tables(hist3: np.ndarray) -> np.ndarray:
    h = torch.from_numpy(np.ascontiguousarray(hist3, np.uint32).view(np.int32).reshape(-1).copy()).cuda()
    f = torch.full((3 * NRES,), -1, dtype=torch.int32, device="cuda")
    native.rans_tables(h, f)
    torch.cuda.synchronize()
    return f.cpu().numpy().view(np.uint32).reshape(3, NRES)


def _oracle_tables(hist3: np.ndarray) -> np.ndarray:
    return np.stack([O.rans_table(hist3[c]) for c in range(3)])


def _hist(r3: np.ndarray, n: int) -> np.ndarray:
    r = r3.reshape(3, n).astype(np.int64) + 255
    return np.stack([np.bincount(r[c], minlength=NRES) for c in range(3)]).astype(np.uint32)


def _used(words: np.ndarray, counts: np.ndarray) -> np.ndarray:
    """The packed words of every chunk block (the rest of a block is not part of the stream)."""
    blocks = words.reshape(-1, 32 * 258)
    per_block = counts.reshape(-1, 32).astype(np.int64).sum(axis=1)
    return np.concatenate([blocks[b, :per_block[b]] for b in range(blocks.shape[0])])


def _gpu_encode(r3: np.ndarray, n: int, freq3: np.ndarray):
    r = torch.from_numpy(np.ascontiguousarray(r3, np.int16).reshape(-1).copy()).cuda()
    f = torch.from_numpy(np.ascontiguousarray(freq3, np.uint32).view(np.int32).reshape(-1).copy()).cuda()
    nw, nc = native.rans_words_capacity(n), native.rans_counts_capacity(n)
    words = torch.full((nw,), 0x5A5A, dtype=torch.int16, device="cuda")
    counts = torch.full((nc,), -1, dtype=torch.int32, device="cuda")
    native.rans_encode(r, n, f, words, counts)
    torch.cuda.synchronize()
    return words.cpu().numpy().view(np.uint16), counts.cpu().numpy().view(np.uint32)


def _gpu_decode(words: np.ndarray, counts: np.ndarray, n: int, freq3: np.ndarray) -> np.ndarray:
    w = torch.from_numpy(np.ascontiguousarray(words, np.uint16).view(np.int16).copy()).cuda()
    c = torch.from_numpy(np.ascontiguousarray(counts, np.uint32).view(np.int32).copy()).cuda()
    f = torch.from_numpy(np.ascontiguousarray(freq3, np.uint32).view(np.int32).reshape(-1).copy()).cuda()
    out = torch.full((3 * n,), 0x7777, dtype=torch.int16, device="cuda")
    native.rans_decode(w, c, n, f, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _check_roundtrip(r3: np.ndarray, n: int):
    native.device_status(clear=True)
    hist = _hist(r3, n)
    freq = _gpu_tables(hist)
    assert np.array_equal(freq, _oracle_tables(hist))
    words, counts = _gpu_encode(r3, n, freq)
    ow, oc = O.rans_encode(r3.reshape(-1), freq)
    assert np.array_equal(counts, oc)
    assert np.array_equal(_used(words, counts), _used(ow, oc))
    assert np.array_equal(_gpu_decode(words, counts, n, freq), r3.reshape(-1))
    assert native.device_status(clear=True) == 0
    return words, counts, freq


def _laplace(n: int, seed: int, scale: float = 3.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.clip(np.round(rng.laplace(0.0, scale, size=3 * n)), -255, 255).astype(np.int16)


@pytest.mark.parametrize("n", [1, 31, 32, 33, 255, 8191, 8192, 8193, 20000, 3 * 8192 + 77])
def test_laplace_residuals_bit_exact(n):
    _check_roundtrip(_laplace(n, seed=n), n)


def test_every_symbol_present_forces_excess_removal():
    # all 511 symbols, most of them rare: many entries are raised to 1 and the
    # excess is taken from the peak
    n = 40000
    rng = np.random.default_rng(11)
    r = _laplace(n, seed=12, scale=1.5)
    r[rng.choice(3 * n, size=3 * NRES, replace=False)] = np.tile(np.arange(-255, 256, dtype=np.int16), 3)
    _check_roundtrip(r, n)


def test_uniform_residuals_use_the_whole_alphabet():
    n = 30000
    r = np.random.default_rng(13).integers(-255, 256, size=3 * n).astype(np.int16)
    _check_roundtrip(r, n)


def test_single_symbol_planes():
    n = 10000
    r = np.concatenate([np.zeros(n), np.full(n, -255), np.full(n, 255)]).astype(np.int16)
    words, counts, freq = _check_roundtrip(r, n)
    assert (freq.max(axis=1) == 16384).all()
    assert (counts == 2).all()


def test_tables_against_oracle_on_adversarial_histograms():
    rng = np.random.default_rng(21)
    cases = []
    h = np.zeros((3, NRES), np.uint32)
    h[0, 255] = 1
    h[1, :] = 1                                   # 511 equal counts: excess on ties
    h[2, [0, 510]] = [7, 7]                       # two-way tie for the shortfall
    cases.append(h)
    for _ in range(20):
        h = np.zeros((3, NRES), np.uint32)
        for c in range(3):
            k = int(rng.integers(1, NRES + 1))
            idx = rng.choice(NRES, size=k, replace=False)
            h[c, idx] = rng.integers(1, int(rng.choice([3, 100, 10 ** 6, 2 ** 31])), size=k, dtype=np.int64)
        cases.append(h)
    h = np.zeros((3, NRES), np.uint32)
    h[:, 255] = 2 ** 32 - 1
    h[:, 254] = 1
    cases.append(h)
    for h in cases:
        g = _gpu_tables(h)
        assert np.array_equal(g, _oracle_tables(h))
        assert ((g.sum(axis=1) == 16384) | (h.sum(axis=1, dtype=np.uint64) == 0)).all()


def test_empty_histogram_gives_empty_table():
    h = np.zeros((3, NRES), np.uint32)
    h[1, 3] = 5
    g = _gpu_tables(h)
    assert (g[0] == 0).all() and (g[2] == 0).all() and g[1, 3] == 16384


def test_cross_decode_with_oracle():
    n = 12345
    r = _laplace(n, seed=31, scale=6.0)
    hist = _hist(r, n)
    freq = _oracle_tables(hist)
    ow, oc = O.rans_encode(r, freq)
    assert np.array_equal(_gpu_decode(ow, oc, n, freq), r)
    words, counts = _gpu_encode(r, n, freq)
    assert np.array_equal(O.rans_decode(words, counts, n, freq), r)


@pytest.mark.parametrize("h,w,q", [(64, 96, 75), (1536, 2048, 90)])
def test_codec_residuals_roundtrip(h, w, q):
    """The enhancement layer of real codec output: tables from the residual
    kernel's histograms, bitstream equal to the oracle's, decode back to R and
    on to the RGBE words."""
    img = synth.make_rgbe(h, w, seed=h + w, lo=-3.0, hi=5.0, rects=6)
    c = codec.Codec(h, w, "cuda")
    L = c.encode(torch.from_numpy(img.view(np.int32).reshape(-1).copy()).cuda(), q)
    n = h * w
    freq = torch.empty(3 * NRES, dtype=torch.int32, device="cuda")
    native.rans_tables(L.hist.reshape(-1), freq)
    words = torch.empty(native.rans_words_capacity(n), dtype=torch.int16, device="cuda")
    counts = torch.empty(native.rans_counts_capacity(n), dtype=torch.int32, device="cuda")
    native.device_status(clear=True)
    native.rans_encode(L.r3, n, freq, words, counts)
    r_back = torch.empty_like(L.r3)
    native.rans_decode(words, counts, n, freq, r_back)
    out = c.decode(L.s3, L.e, r_back, L.params)
    torch.cuda.synchronize()
    assert native.device_status(clear=True) == 0
    assert np.array_equal(out.cpu().numpy().view(np.uint32).reshape(h, w), img)
    r3 = L.r3.cpu().numpy()
    hist = L.hist.cpu().numpy().view(np.uint32).reshape(3, NRES)
    f_or = _oracle_tables(hist)
    assert np.array_equal(freq.cpu().numpy().view(np.uint32).reshape(3, NRES), f_or)
    ow, oc = O.rans_encode(r3, f_or)
    assert np.array_equal(counts.cpu().numpy().view(np.uint32), oc)
    assert np.array_equal(_used(words.cpu().numpy().view(np.uint16), oc), _used(ow, oc))
    # the coded size is close to the zeroth-order entropy of the histograms:
    # at most 32 bits of final state and one partly used word per stream over it
    bits = 16.0 * oc.astype(np.float64).sum()
    h0 = sum(O.entropy_bits(hist[ch]) * n for ch in range(3))
    assert bits < h0 * 1.01 + 48 * len(oc)


def test_residual_without_frequency_is_reported():
    n = 9000
    r = _laplace(n, seed=41)
    freq = _oracle_tables(_hist(r, n))
    r_bad = r.copy()
    r_bad[5000] = 200
    assert freq[0, 200 + 255] == 0
    native.device_status(clear=True)
    words, counts = _gpu_encode(r_bad, n, freq)
    assert native.device_status(clear=True) == STATUS_RANS
    # chunk 0, stream 5000 % 32 of plane 0 could not be coded; all others are exact
    bad = 5000 % 32
    assert counts[bad] == 0
    ow, oc = O.rans_encode(r, freq)
    keep = np.ones(counts.size, bool)
    keep[bad] = False
    assert np.array_equal(counts[keep], oc[keep])
    # the blocks of the other chunks are the oracle's
    nb = counts.size // 32
    for b in range(1, nb):
        sl = slice(b * 32, (b + 1) * 32)
        w_gpu = words.reshape(nb, -1)[b, :int(counts[sl].sum())]
        w_or = ow.reshape(nb, -1)[b, :int(oc[sl].sum())]
        assert np.array_equal(w_gpu, w_or)


def test_corrupt_streams_and_tables_are_reported():
    n = 9000
    r = _laplace(n, seed=43)
    freq = _oracle_tables(_hist(r, n))
    words, counts = O.rans_encode(r, freq)
    native.device_status(clear=True)
    bad_counts = counts.copy()
    bad_counts[7] = 300                                      # beyond the region
    _gpu_decode(words, bad_counts, n, freq)
    assert native.device_status(clear=True) == STATUS_RANS
    bad_counts = counts.copy()
    bad_counts[40] = 2                                        # truncated stream
    _gpu_decode(words, bad_counts, n, freq)
    assert native.device_status(clear=True) == STATUS_RANS
    bad_freq = freq.copy()
    bad_freq[1, 255] += 1                                     # total M + 1
    _gpu_decode(words, counts, n, bad_freq)
    assert native.device_status(clear=True) == STATUS_RANS
    _gpu_encode(r, n, bad_freq)
    assert native.device_status(clear=True) == STATUS_RANS
    big = freq.copy()
    big[2, :] = 0
    big[2, 255] = 2 ** 32 - 16384                             # entries above M whose 32-bit sum wraps to M
    big[2, 256] = 2 * 16384
    _gpu_decode(words, counts, n, big)
    assert native.device_status(clear=True) == STATUS_RANS
    # the good stream still decodes afterwards
    assert np.array_equal(_gpu_decode(words, counts, n, freq), r)
    assert native.device_status(clear=True) == 0
