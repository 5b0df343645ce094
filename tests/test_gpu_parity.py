"""Bit-exact parity of every C-ABI entry point against the CPU oracle.

Each stage is fed the oracle's own inputs for that stage (so a mismatch is
localised), then the chained encoder/decoder is compared on the workload
sizes, ragged sizes, empty images, edge-case exponent layouts and
misaligned buffers (scalar paths).  All comparisons are exact: the codec
is integer work plus float32/float64 steps both sides take identically.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2309_11072_gb300 import codec, native, synth

pytestmark = pytest.mark.gpu

DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    native.lib()
    yield
    torch.cuda.synchronize()


def dev(a: np.ndarray, dtype=None, offset: int = 0) -> torch.Tensor:
    """Upload a C-contiguous numpy array; offset > 0 places it at a misaligned address."""
    a = np.ascontiguousarray(a)
    raw = a.reshape(-1).view(np.uint8)
    if offset:
        buf = torch.empty(raw.size + offset, dtype=torch.uint8, device=DEV)
        buf[offset:].copy_(torch.from_numpy(raw.copy()))
        return buf[offset:]
    t = torch.from_numpy(a.reshape(-1).copy())
    if dtype is not None:
        t = t.view(dtype)
    return t.to(DEV)


def host(t: torch.Tensor, np_dtype) -> np.ndarray:
    return t.detach().cpu().contiguous().view(torch.uint8).numpy().view(np_dtype)


def empty_bytes(nbytes: int, offset: int = 0) -> torch.Tensor:
    buf = torch.empty(max(1, nbytes + offset), dtype=torch.uint8, device=DEV)
    return buf[offset:offset + nbytes]


SIZES = [(1, 1), (1, 9), (7, 1), (7, 9), (8, 8), (9, 17), (17, 9), (16, 256), (33, 65), (100, 37),
         (37, 300), (64, 264), (129, 513)]


def make_img(h, w, kind, seed):
    if kind == "scene":
        return synth.make_rgbe(h, w, seed=seed, lo=-3.0, hi=5.0, rects=2, highlights=3)
    if kind == "noise":          # exponents change at every pixel: per-pixel run path
        return synth.tiny_rgbe(h, w, seed=seed, e_lo=0, e_hi=255, zero_frac=0.05)
    if kind == "flat":           # one exponent region
        return synth.tiny_rgbe(h, w, seed=seed, const_e=128)
    if kind == "zero":
        return np.zeros((h, w), np.uint32)
    raise ValueError(kind)


# ------------------------------------------------------------------ per stage

def run_split(img, offset=0):
    """offset > 0: words 4 bytes past a 16-byte boundary (naturally aligned, not
    vector aligned) and byte planes `offset` bytes past one."""
    h, w = img.shape
    n = h * w
    m3 = empty_bytes(3 * n, offset)
    e = empty_bytes(n, offset)
    st = torch.empty(2, dtype=torch.int64, device=DEV)
    native.rgbe_split(dev(img.view(np.uint8), offset=4) if offset else dev(img, torch.int32),
                      h, w, m3, e, st)
    torch.cuda.synchronize()
    return host(m3, np.uint8).reshape(3, h, w), host(e, np.uint8).reshape(h, w), st.cpu().numpy()


@pytest.mark.parametrize("h,w", SIZES)
@pytest.mark.parametrize("kind", ["scene", "noise", "zero"])
def test_split_parity(h, w, kind):
    img = make_img(h, w, kind, seed=h * 1000 + w)
    m3, e, st = run_split(img)
    om3, oe = O.rgbe_split(img)
    assert np.array_equal(m3, om3) and np.array_equal(e, oe)
    assert np.array_equal(st, O.lum_stats(img))


@pytest.mark.parametrize("offset", [1, 3])
def test_split_misaligned(offset):
    img = make_img(24, 40, "scene", seed=5)
    m3, e, st = run_split(img, offset)
    om3, oe = O.rgbe_split(img)
    assert np.array_equal(m3, om3) and np.array_equal(e, oe) and np.array_equal(st, O.lum_stats(img))


def run_base(m3, e, stats, quality, offset=0):
    h, w = e.shape
    n = h * w
    s3 = empty_bytes(3 * n, offset)
    sdr3 = empty_bytes(3 * n, offset)
    native.sdri_base_roundtrip(dev(m3, offset=offset), dev(e, offset=offset), h, w,
                               dev(stats.astype(np.int64)), quality, s3, sdr3)
    torch.cuda.synchronize()
    return host(s3, np.uint8).reshape(3, h, w), host(sdr3, np.uint8).reshape(3, h, w)


@pytest.mark.parametrize("h,w", SIZES)
@pytest.mark.parametrize("quality", [10, 50, 90, 100])
def test_base_parity(h, w, quality):
    img = make_img(h, w, "scene", seed=h + 7 * w)
    om3, oe = O.rgbe_split(img)
    st = O.lum_stats(img)
    J, r = O.key(st)
    osdr = O.tmo(img, J, r)
    os3 = O.base_roundtrip(osdr, quality)
    s3, sdr3 = run_base(om3, oe, st, quality)
    assert np.array_equal(sdr3, osdr)
    assert np.array_equal(s3, os3)


@pytest.mark.parametrize("kind", ["noise", "zero", "flat"])
def test_base_parity_edge_images(kind):
    img = make_img(40, 56, kind, seed=9)
    om3, oe = O.rgbe_split(img)
    st = O.lum_stats(img)
    J, r = O.key(st)
    s3, sdr3 = run_base(om3, oe, st, 75)
    assert np.array_equal(sdr3, O.tmo(img, J, r))
    assert np.array_equal(s3, O.base_roundtrip(O.tmo(img, J, r), 75))


def test_base_misaligned():
    img = make_img(24, 48, "scene", seed=3)
    om3, oe = O.rgbe_split(img)
    st = O.lum_stats(img)
    J, r = O.key(st)
    s3, sdr3 = run_base(om3, oe, st, 60, offset=5)
    osdr = O.tmo(img, J, r)
    assert np.array_equal(sdr3, osdr) and np.array_equal(s3, O.base_roundtrip(osdr, 60))


def run_fit(s3, m3, e, gf_on, offset=0):
    h, w = e.shape
    sums = torch.empty(256 * 13, dtype=torch.int64, device=DEV)
    params = torch.empty(native.PARAMS_BYTES // 4, dtype=torch.int32, device=DEV)
    native.slr_fit(dev(s3, offset=offset), dev(m3, offset=offset), dev(e, offset=offset), h, w, gf_on, sums, params)
    torch.cuda.synchronize()
    return sums.cpu().numpy().reshape(256, 13), codec.params_to_numpy(params)


def _check_params(p, a, b, n, nu):
    assert np.array_equal(p["a"].view(np.uint32), a.view(np.uint32))
    assert np.array_equal(p["b"].view(np.uint32), b.view(np.uint32))
    assert np.array_equal(p["n"], n) and p["n_used"] == nu


@pytest.mark.parametrize("h,w", SIZES)
@pytest.mark.parametrize("kind", ["scene", "noise"])
@pytest.mark.parametrize("gf_on", [0, 1])
def test_fit_parity(h, w, kind, gf_on):
    img = make_img(h, w, kind, seed=3 * h + w)
    rng = np.random.default_rng(h * w)
    om3, oe = O.rgbe_split(img)
    s3 = rng.integers(0, 256, size=(3, h, w)).astype(np.uint8) if kind == "noise" else \
        O.base_roundtrip(O.tmo(img, *O.key(O.lum_stats(img))), 80)
    sums, p = run_fit(s3, om3, oe, gf_on)
    osums = O.bin_sums(O.gf(s3, bool(gf_on)), om3, oe)
    assert np.array_equal(sums, osums)
    _check_params(p, *O.solve(osums))


def test_fit_misaligned_and_degenerate():
    img = make_img(30, 64, "flat", seed=4)
    om3, oe = O.rgbe_split(img)
    s3 = np.full((3, 30, 64), 77, np.uint8)            # D_xx = 0 in the only region
    sums, p = run_fit(s3, om3, oe, 1, offset=3)
    osums = O.bin_sums(O.gf(s3), om3, oe)
    assert np.array_equal(sums, osums)
    _check_params(p, *O.solve(osums))
    assert p["n_used"] == 1 and p["a"][0, 128] == 0


def run_residual(s3, m3, e, a, b, gf_on, offset=0):
    h, w = e.shape
    n = h * w
    r3 = empty_bytes(2 * 3 * n, 2 * offset).view(torch.int16) if not offset else \
        torch.empty(3 * n + 1, dtype=torch.int16, device=DEV)[1:]
    hist = torch.empty(3 * 511, dtype=torch.int32, device=DEV)
    params = dev(codec.params_from_numpy(a, b), torch.int32)
    native.residual_encode(dev(s3, offset=offset), dev(m3, offset=offset), dev(e, offset=offset), h, w, gf_on,
                           params, r3, hist)
    torch.cuda.synchronize()
    return host(r3, np.int16).reshape(3, h, w), host(hist, np.uint32).reshape(3, 511)


@pytest.mark.parametrize("h,w", [(9, 17), (33, 64), (20, 2064)])
def test_residual_without_histograms(h, w):
    """hist = NULL: the same residuals, nothing counted (a width that is a
    multiple of 16 takes the bulk-copy row kernels, the others the strip
    kernels)."""
    img = make_img(h, w, "noise", seed=h + 7 * w)
    rng = np.random.default_rng(h * w)
    om3, oe = O.rgbe_split(img)
    s3 = rng.integers(0, 256, size=(3, h, w)).astype(np.uint8)
    a, b = _random_params(w)
    n = h * w
    r3 = torch.empty(3 * n, dtype=torch.int16, device=DEV)
    params = dev(codec.params_from_numpy(a, b), torch.int32)
    native.residual_encode(dev(s3), dev(om3), dev(oe), h, w, 1, params, r3, None)
    torch.cuda.synchronize()
    or3, _ = O.residual(om3, O.predict(O.gf(s3), oe, a, b))
    assert np.array_equal(host(r3, np.int16).reshape(3, h, w), or3)


def _random_params(seed):
    rng = np.random.default_rng(seed)
    return (rng.uniform(-0.2, 0.2, (3, 256)).astype(np.float32),
            rng.uniform(-80, 330, (3, 256)).astype(np.float32))


@pytest.mark.parametrize("h,w", SIZES)
@pytest.mark.parametrize("gf_on", [0, 1])
def test_residual_parity(h, w, gf_on):
    img = make_img(h, w, "noise", seed=h * 31 + w)
    rng = np.random.default_rng(w)
    om3, oe = O.rgbe_split(img)
    s3 = rng.integers(0, 256, size=(3, h, w)).astype(np.uint8)
    a, b = _random_params(h + w)
    r3, hist = run_residual(s3, om3, oe, a, b, gf_on)
    ms = O.predict(O.gf(s3, bool(gf_on)), oe, a, b)
    or3, ohist = O.residual(om3, ms)
    assert np.array_equal(r3, or3) and np.array_equal(hist, ohist)


def test_residual_misaligned():
    img = make_img(16, 64, "scene", seed=8)
    om3, oe = O.rgbe_split(img)
    s3 = np.random.default_rng(1).integers(0, 256, size=(3, 16, 64)).astype(np.uint8)
    a, b = _random_params(5)
    r3, hist = run_residual(s3, om3, oe, a, b, 1, offset=1)
    or3, ohist = O.residual(om3, O.predict(O.gf(s3), oe, a, b))
    assert np.array_equal(r3, or3) and np.array_equal(hist, ohist)


@pytest.mark.parametrize("h,w", SIZES)
@pytest.mark.parametrize("gf_on", [0, 1])
def test_decode_parity_any_params(h, w, gf_on):
    img = make_img(h, w, "noise", seed=h + w * 13)
    rng = np.random.default_rng(h * 7)
    om3, oe = O.rgbe_split(img)
    s3 = rng.integers(0, 256, size=(3, h, w)).astype(np.uint8)
    a, b = _random_params(w)
    r3, _ = O.residual(om3, O.predict(O.gf(s3, bool(gf_on)), oe, a, b))
    out = torch.empty(h * w, dtype=torch.int32, device=DEV)
    native.residual_decode(dev(s3), dev(oe), dev(r3, torch.int16), h, w, gf_on,
                           dev(codec.params_from_numpy(a, b), torch.int32), out)
    torch.cuda.synchronize()
    got = host(out, np.uint32).reshape(h, w)
    assert np.array_equal(got, O.decode(s3, oe, r3, a, b, bool(gf_on)))
    assert np.array_equal(got, img)


@pytest.mark.parametrize("w", [64, 72])
def test_prediction_ties_round_half_away(w):
    # slopes and intercepts that put a * x + b exactly on .5 for many x: the
    # residuals (and the decoder) follow Eq. 8's round half away from zero
    h = 40
    img = make_img(h, w, "noise", seed=w)
    om3, oe = O.rgbe_split(img)
    s3 = np.random.default_rng(w).integers(0, 256, size=(3, h, w)).astype(np.uint8)
    a = np.zeros((3, 256), np.float32)
    b = np.zeros((3, 256), np.float32)
    a[0], b[0] = 1.0 / 32.0, 0.0          # x = 16 (2k + 1): t = k + 0.5
    a[1], b[1] = 1.0 / 16.0, 0.5          # every x: t = S* + 0.5 on integer S*
    a[2], b[2] = 1.0 / 64.0, 0.25         # x = 16 (2k + 1): t = k / 2 + 0.5 (every other one a tie)
    for gf_on in (0, 1):
        x3 = O.gf(s3, bool(gf_on))
        ms = O.predict(x3, oe, a, b)
        r3, hist = run_residual(s3, om3, oe, a, b, gf_on)
        or3, ohist = O.residual(om3, ms)
        assert np.array_equal(r3, or3) and np.array_equal(hist, ohist)
        out = torch.empty(h * w, dtype=torch.int32, device=DEV)
        native.residual_decode(dev(s3), dev(oe), dev(or3, torch.int16), h, w, gf_on,
                               dev(codec.params_from_numpy(a, b), torch.int32), out)
        torch.cuda.synchronize()
        assert np.array_equal(host(out, np.uint32).reshape(h, w), img)


# ------------------------------------------------------------------ chained

def encode_gpu(img, quality, gf_on=True):
    h, w = img.shape
    c = codec.Codec(h, w, DEV, gf_on=gf_on, keep_sdr=True)
    L = c.encode(dev(img, torch.int32), quality)
    out = c.decode(L.s3, L.e, L.r3, L.params)
    torch.cuda.synchronize()
    res = dict(m3=host(c.m3, np.uint8).reshape(3, h, w), e=host(c.e, np.uint8).reshape(h, w),
               stats=c.stats.cpu().numpy(), sdr3=host(c.sdr3, np.uint8).reshape(3, h, w),
               s3=host(c.s3, np.uint8).reshape(3, h, w), sums=c.sums.cpu().numpy().reshape(256, 13),
               r3=host(c.r3, np.int16).reshape(3, h, w), hist=host(c.hist, np.uint32).reshape(3, 511),
               out=host(out, np.uint32).reshape(h, w), bpp=c.bits_per_pixel())
    res.update(codec.params_to_numpy(c.params))
    return res


def assert_matches_oracle(img, quality, gf_on=True):
    g = encode_gpu(img, quality, gf_on)
    o = O.encode(img, quality, gf_on)
    for k in ("m3", "e", "stats", "sdr3", "s3", "sums", "r3", "hist"):
        assert np.array_equal(g[k], o[k]), k
    _check_params(g, o["a"], o["b"], o["n"], o["n_used"])
    assert np.array_equal(g["out"], img), "decode(encode(x)) != x"
    return g, o


@pytest.mark.parametrize("h,w", [(0, 0), (0, 7), (5, 0)])
def test_empty_images(h, w):
    c = codec.Codec(h, w, DEV)
    rgbe = torch.empty(0, dtype=torch.int32, device=DEV)
    L = c.encode(rgbe, 75)
    c.decode(L.s3, L.e, L.r3, L.params)
    torch.cuda.synchronize()
    p = codec.params_to_numpy(c.params)
    assert p["n_used"] == 0 and (p["n"] == 0).all()
    assert c.stats.cpu().tolist() == [0, 0] and int(c.hist.sum()) == 0


@pytest.mark.parametrize("h,w", [(1, 1), (9, 17), (129, 513), (263, 389)])
@pytest.mark.parametrize("gf_on", [True, False])
def test_pipeline_ragged(h, w, gf_on):
    assert_matches_oracle(make_img(h, w, "scene", seed=h * w), 85, gf_on)


@pytest.mark.parametrize("kind", ["noise", "flat", "zero"])
def test_pipeline_edge_images(kind):
    assert_matches_oracle(make_img(96, 136, kind, seed=2), 70)


def test_pipeline_every_exponent():
    img = synth.tiny_rgbe(64, 64, seed=3, e_lo=0, e_hi=255)
    img.flat[:256] = (img.flat[:256] & 0x00FFFFFF) | (np.arange(256, dtype=np.uint32) << 24)
    g, _ = assert_matches_oracle(img, 90)
    assert g["n_used"] == 256


def test_pipeline_small_workload():
    wl = synth.workload_small()
    img = synth.make_workload_images(wl)[0]
    assert_matches_oracle(img, 90)


@pytest.mark.slow
@pytest.mark.parametrize("quality", [50, 75, 90])
def test_pipeline_2k_workload_full_size(quality):
    wl = synth.workload_2k()
    img = synth.make_workload_images(wl)[0]
    g, _ = assert_matches_oracle(img, quality)
    assert 0 < g["bpp"] < 24


@pytest.mark.slow
def test_pipeline_8k_workload_full_size():
    wl = synth.workload_8k()
    img = synth.make_workload_images(wl)[0]
    g, o = assert_matches_oracle(img, 90)
    e = g["e"]
    assert e.min() >= 100 and e.max() <= 150


def _device_status():
    import ctypes
    v = ctypes.c_int(-1)
    L = native.lib()
    assert L.slrme_device_status(ctypes.addressof(v), 1) == 0
    return v.value


@pytest.mark.parametrize("h,w", [(1, 16), (8, 16), (33, 256), (70, 512), (45, 784), (100, 1040), (5, 2064),
                                 (3, 4096), (21, 2560), (80000, 16)])
@pytest.mark.parametrize("gf_on", [True, False])
def test_tma_staged_path_matches_oracle(h, w, gf_on):
    # rows of 16-byte multiples take the tensor-map (TMA) kernels of fit, residual
    # and decode: 2048-column strips (one or several, the last one partial), CTA
    # row ranges that cross from one strip to the next, tasks longer than 256 rows
    _device_status()
    assert_matches_oracle(make_img(h, w, "scene", seed=h + 3 * w), 80, gf_on)
    assert_matches_oracle(make_img(h, w, "noise", seed=h + 5 * w), 80, gf_on)
    assert _device_status() == 0


def test_host_codec_slots_match_oracle():
    # calls queued back to back on the rotating slots (copies of one call
    # overlapping the next one's coding) leave each call's layers intact
    h, w = 96, 144
    hc = codec.HostCodec(h, w, DEV)
    nslots = len(hc.slots)
    calls = [(make_img(h, w, "scene", seed=10 + i), [50, 75, 90, 60, 85][i]) for i in range(nslots + 2)]
    hosts = [torch.from_numpy(img.view(np.int32).reshape(-1).copy()).pin_memory() for img, _ in calls]
    for host, (_, q) in zip(hosts, calls):
        hc.roundtrip(host, q)
    torch.cuda.synchronize()
    for i in range(len(calls) - nslots, len(calls)):
        img, q = calls[i]
        sl = hc.slots[i % nslots]
        o = O.encode(img, q)
        assert np.array_equal(sl["h_out"].numpy().view(np.uint32).reshape(h, w), img)
        assert np.array_equal(sl["h_r3"].numpy().reshape(3, h, w), o["r3"])
        assert np.array_equal(sl["h_s3"].numpy().reshape(3, h, w), o["s3"])
