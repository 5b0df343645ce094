"""Seeded synthetic Radiance (RGBE) HDR images.

This module only *makes inputs*.  It holds none of the codec's arithmetic
(no tone mapping, no DCT, no regression, no residuals); both the CPU oracle
and the CUDA path receive the packed RGBE words produced here.

Scene model (the stand-in for the paper's 1920x1080 HDR-Eye / DML-HDR
photographs of Sec. IV, which are not available here):

* luminance ``L = 10 ** (lo + (hi - lo) * u)`` where ``u`` in [0, 1] is a
  min-max normalised 2-D fractional Brownian motion field made by spectral
  synthesis (white Gaussian noise, amplitude ``|k| ** -(H + 1)``, H = 0.7);
* per-image colour gains ``g_c ~ U(0.6, 1.4)`` so ``f_c = L * g_c``;
* optional sharp-edged rectangles (luminance times ``10 ** U(-2, 2)``),
  Gaussian specular highlights (peak 1e5) and a smooth sky band.

The floats are written in the Radiance file format (Sec. II-A, Fig. 1):
three 8-bit mantissas sharing one 8-bit exponent, packed little-endian as
``R | G << 8 | B << 16 | E << 24``.  The packing follows Ward's frexp
convention (exponent = frexp exponent + 128, mantissa = floor(f * 2^(136-E)))
in float64; pixels whose largest channel is below 1e-32 become the all-zero
word.  This is the file writer that produces the codec's input, not a step
of the codec.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Tuple

import numpy as np

HURST = 0.7


@dataclasses.dataclass(frozen=True)
class Workload:
    """A named synthetic workload: image sizes, decades and features."""
    name: str
    sizes: Tuple[Tuple[int, int], ...]   # (height, width) per image
    seeds: Tuple[int, ...]
    lo: Tuple[float, ...]                # log10 of darkest luminance per image
    hi: Tuple[float, ...]                # log10 of brightest luminance per image
    rects: int = 0
    highlights: int = 0
    sky: bool = False
    qualities: Tuple[int, ...] = (90,)

    @property
    def pixels(self) -> int:
        return int(sum(h * w for h, w in self.sizes))


def fbm(h: int, w: int, rng: np.random.Generator, hurst: float = HURST) -> np.ndarray:
    """Min-max normalised 2-D fBm field in [0, 1] (float64, shape (h, w))."""
    noise = rng.standard_normal((h, w))
    spec = np.fft.rfft2(noise)
    ky = np.fft.fftfreq(h)[:, None]
    kx = np.fft.rfftfreq(w)[None, :]
    k = np.sqrt(kx * kx + ky * ky)
    k[0, 0] = 1.0
    amp = k ** (-(hurst + 1.0))
    amp[0, 0] = 0.0
    spec *= amp
    field = np.fft.irfft2(spec, s=(h, w))
    lo, hi = field.min(), field.max()
    if hi <= lo:
        return np.zeros((h, w))
    return (field - lo) / (hi - lo)


def hdr_image(h: int, w: int, seed: int, lo: float, hi: float, rects: int = 0,
              highlights: int = 0, sky: bool = False) -> np.ndarray:
    """Linear-light RGB radiance, float64, shape (h, w, 3)."""
    rng = np.random.default_rng(seed)
    u = fbm(h, w, rng)
    if sky:
        band = max(1, h // 3)
        ys = np.arange(band, dtype=np.float64)
        t = 1.0 - ys / band                       # 1 at the top row, 0 at h/3
        grad = 0.95 - 0.25 * (ys / band)          # smooth vertical sky ramp
        u[:band] = t[:, None] * grad[:, None] + (1.0 - t[:, None]) * u[:band]
    lum = 10.0 ** (lo + (hi - lo) * u)
    for _ in range(rects):
        rh = max(1, int(h * rng.uniform(0.02, 0.20)))
        rw = max(1, int(w * rng.uniform(0.02, 0.20)))
        y0 = int(rng.integers(0, max(1, h - rh + 1)))
        x0 = int(rng.integers(0, max(1, w - rw + 1)))
        lum[y0:y0 + rh, x0:x0 + rw] *= 10.0 ** rng.uniform(-2.0, 2.0)
    for _ in range(highlights):
        sig = rng.uniform(1.0, 8.0)
        cy = rng.uniform(0, h)
        cx = rng.uniform(0, w)
        r = int(np.ceil(4 * sig))
        y0, y1 = max(0, int(cy) - r), min(h, int(cy) + r + 1)
        x0, x1 = max(0, int(cx) - r), min(w, int(cx) + r + 1)
        if y0 >= y1 or x0 >= x1:
            continue
        yy = np.arange(y0, y1)[:, None] + 0.5 - cy
        xx = np.arange(x0, x1)[None, :] + 0.5 - cx
        lum[y0:y1, x0:x1] += 1e5 * np.exp(-(yy * yy + xx * xx) / (2 * sig * sig))
    gains = rng.uniform(0.6, 1.4, size=3)
    return lum[:, :, None] * gains[None, None, :]


def pack_radiance(rgb: np.ndarray) -> np.ndarray:
    """Write float64 RGB (h, w, 3) as packed Radiance words (uint32, (h, w))."""
    rgb = np.asarray(rgb, dtype=np.float64)
    v = rgb.max(axis=-1)
    zero = v < 1e-32
    mant, ex = np.frexp(np.where(zero, 1.0, v))
    E = ex.astype(np.int64) + 128
    if (E[~zero] < 1).any() or (E[~zero] > 255).any():
        raise ValueError("radiance outside the range the 8-bit exponent can hold")
    scale = np.ldexp(1.0, (136 - E))
    M = np.floor(rgb * scale[..., None]).astype(np.int64)
    M[zero] = 0
    E = np.where(zero, 0, E)
    word = (M[..., 0] | (M[..., 1] << 8) | (M[..., 2] << 16) | (E << 24)).astype(np.uint32)
    return word


def make_rgbe(h: int, w: int, seed: int, lo: float, hi: float, **kw) -> np.ndarray:
    return pack_radiance(hdr_image(h, w, seed, lo, hi, **kw))


# --------------------------------------------------------------------------
# The workloads.  Sizes, decades and features follow the five synthetic
# configurations the benchmark is defined on; every image is seeded.
# --------------------------------------------------------------------------

def workload_small() -> Workload:
    """512x384, fBm over 6 decades (1e-2..1e4), base quality 90."""
    return Workload("rgbe-512x384-fbm6", ((384, 512),), (1,), (-2.0,), (4.0,), qualities=(90,))


def workload_2k() -> Workload:
    """2048x1536, fBm over 8 decades + 40 rectangles + 200 highlights, q in {50,75,90}."""
    return Workload("rgbe-2048x1536-fbm8-rects40-spec200", ((1536, 2048),), (2,), (-3.0,), (5.0,),
                    rects=40, highlights=200, qualities=(50, 75, 90))


def workload_8k() -> Workload:
    """7680x4320, fBm over 8 decades with a smooth sky band in the top third.

    lo = -3, hi = 5 with gains in [0.6, 1.4] keeps every exponent in [100, 150].
    """
    return Workload("rgbe-7680x4320-fbm8-sky", ((4320, 7680),), (3,), (-3.0,), (5.0,), sky=True,
                    qualities=(90,))


def workload_batch(n: int = 64, seed: int = 4) -> Workload:
    """64 images, W ~ U{256..4096}, H ~ U{256..2160}, 4-8 decades, rectangles and highlights."""
    rng = np.random.default_rng(seed)
    sizes, seeds, los, his = [], [], [], []
    for i in range(n):
        w = int(rng.integers(256, 4097))
        h = int(rng.integers(256, 2161))
        dec = int(rng.integers(4, 9))
        lo = float(rng.uniform(-3.0, 0.0))
        sizes.append((h, w))
        seeds.append(seed * 1000 + i)
        los.append(lo)
        his.append(lo + dec)
    return Workload(f"rgbe-batch{n}-uneven", tuple(sizes), tuple(seeds), tuple(los), tuple(his),
                    rects=40, highlights=200, qualities=(90,))


def make_workload_images(wl: Workload) -> List[np.ndarray]:
    out = []
    for (h, w), s, lo, hi in zip(wl.sizes, wl.seeds, wl.lo, wl.hi):
        out.append(make_rgbe(h, w, s, lo, hi, rects=wl.rects, highlights=wl.highlights, sky=wl.sky))
    return out


def tiny_rgbe(h: int, w: int, seed: int, e_lo: int = 100, e_hi: int = 160,
              zero_frac: float = 0.0, const_e: Optional[int] = None) -> np.ndarray:
    """Small random RGBE words for edge cases (raw bytes, not from a scene).

    Mantissas are uniform bytes with the largest one forced to >= 128
    (normalised words); exponents uniform in [e_lo, e_hi] or constant.
    A fraction ``zero_frac`` of pixels is the all-zero word.
    """
    rng = np.random.default_rng(seed)
    m = rng.integers(0, 256, size=(h, w, 3), dtype=np.int64)
    top = m.argmax(axis=-1)
    idx = np.indices((h, w))
    m[idx[0], idx[1], top] |= 128
    if const_e is None:
        e = rng.integers(e_lo, e_hi + 1, size=(h, w), dtype=np.int64)
    else:
        e = np.full((h, w), const_e, dtype=np.int64)
    if zero_frac > 0:
        z = rng.random((h, w)) < zero_frac
        m[z] = 0
        e[z] = 0
    return (m[..., 0] | (m[..., 1] << 8) | (m[..., 2] << 16) | (e << 24)).astype(np.uint32)
