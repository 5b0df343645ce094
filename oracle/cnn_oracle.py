"""CPU oracle of the learned mantissa estimator (the integer CNN).

TEST INFRASTRUCTURE ONLY: imported by the tests and the benchmark's CPU legs,
never by the product path.  Plain numpy: int64 for the integer inference,
float64 for the training arithmetic.

The paper's estimator is the simple linear regression (Sec. III-B, Eqs. 8-10);
this network is a learned alternative to it, chosen per image only where its
residuals cost fewer bits, with the same residual / lossless decoding
(Sec. III-C).  Its definition (the READING this project fixes):

Input (4 int8 planes, per pixel):  S_c - 128 (c = R, G, B) and
    clamp(E - 137 - J, -128, 127), the exponent relative to the image's
    tone-mapping key J (Sec. II-B's operator uses the same d = E - 137 - J).
Output: three planes y_c in [0, 255] that correct the regression's estimate
    (Eq. 8): M^_c = clamp(M*_c + y_c - 128, 0, 255).  (READING: the network
    refines the regression rather than replacing it; a network that knows
    only the integer part of the key cannot place the mantissas alone.)
Layers l = 1..4: 3x3 convolution, zero padding, stride 1, channels
    4 -> 16 -> 16 -> 16 -> 3; weights int8 in [-127, 127], bias int32,
    per-output-channel multiplier int32 and per-layer shift.
    acc = bias + sum w * a  (exact integer);
    y   = clamp(floor(((acc) * mult + 2^(shift-1)) / 2^shift), lo, hi)
    with [lo, hi] = [0, 127] for layers 1-3 (ReLU) and [0, 255] for layer 4,
    whose three planes are the corrections y_R, y_G, y_B.

Training (float): the same network with fake quantisation (weights per
output channel to int8 steps, hidden activations to multiples of SCALE_A in
[0, 127 SCALE_A]; straight-through gradients inside the range) and an L1
loss between y and the regression's residual plus 128, (M - M*) + 128.
"""
from __future__ import annotations

import numpy as np

CHANNELS = (4, 16, 16, 16, 3)
SCALE_A = 1.0 / 8.0      # hidden activation step of the fake-quantised network


# ------------------------------------------------------------------ input

def cnn_input(s3: np.ndarray, e: np.ndarray, J: int) -> np.ndarray:
    """int64 [4, h, w]: S - 128 and the key-relative exponent (clamped)."""
    s3 = np.asarray(s3, np.int64)
    d = np.clip(np.asarray(e, np.int64) - 137 - int(J), -128, 127)
    return np.concatenate([s3 - 128, d[None]], axis=0)


# ------------------------------------------------------------------ integer inference

def conv3x3_int(a: np.ndarray, w: np.ndarray) -> np.ndarray:
    """sum over input channels and the 3x3 window, zero padding: int64 [Co, h, w]."""
    a = np.asarray(a, np.int64)
    w = np.asarray(w, np.int64)
    ci, h, wd = a.shape
    co = w.shape[0]
    pad = np.zeros((ci, h + 2, wd + 2), np.int64)
    pad[:, 1:-1, 1:-1] = a
    out = np.zeros((co, h, wd), np.int64)
    for dy in range(3):
        for dx in range(3):
            win = pad[:, dy:dy + h, dx:dx + wd]                       # [ci, h, w]
            out += np.einsum("oc,chw->ohw", w[:, :, dy, dx], win)
    return out


def requant(acc: np.ndarray, mult: np.ndarray, shift: int, lo: int, hi: int) -> np.ndarray:
    """clamp(floor((acc * mult + 2^(shift-1)) / 2^shift), lo, hi), exact int64."""
    acc = np.asarray(acc, np.int64)
    m = np.asarray(mult, np.int64).reshape(-1, 1, 1)
    y = (acc * m + (1 << (shift - 1))) >> shift
    return np.clip(y, lo, hi)


def infer(s3: np.ndarray, e: np.ndarray, J: int, net: dict) -> np.ndarray:
    """Output planes y (uint8 [3, h, w]) of the integer network."""
    a = cnn_input(s3, e, J)
    for l in range(4):
        acc = conv3x3_int(a, net["w"][l]) + np.asarray(net["b"][l], np.int64).reshape(-1, 1, 1)
        a = requant(acc, net["m"][l], int(net["sh"][l]), 0, 127 if l < 3 else 255)
    return a.astype(np.uint8)


def refine(mstar3: np.ndarray, y3: np.ndarray) -> np.ndarray:
    """M^ = clamp(M* + y - 128, 0, 255)."""
    return np.clip(np.asarray(mstar3, np.int64) + np.asarray(y3, np.int64) - 128, 0, 255).astype(np.uint8)


def residual(m3: np.ndarray, mhat3: np.ndarray):
    r3 = np.asarray(m3, np.int16) - np.asarray(mhat3, np.int16)
    hist = np.stack([np.bincount(r3[c].reshape(-1) + 255, minlength=511) for c in range(3)]).astype(np.uint32)
    return r3, hist


def random_net(seed: int, w_range: int = 127) -> dict:
    """Seeded random integer network (for parity tests)."""
    rng = np.random.default_rng(seed)
    net = {"w": [], "b": [], "m": [], "sh": []}
    for l in range(4):
        ci, co = CHANNELS[l], CHANNELS[l + 1]
        net["w"].append(rng.integers(-w_range, w_range + 1, size=(co, ci, 3, 3)).astype(np.int8))
        net["b"].append(rng.integers(-20000, 20000, size=co).astype(np.int32))
        net["m"].append(rng.integers(1, 1 << 15, size=co).astype(np.int32))
        net["sh"].append(int(rng.integers(18, 24)))
    return net


# ------------------------------------------------------------------ float training (float64)

def fq_weight(w: np.ndarray) -> np.ndarray:
    """Per-output-channel int8 steps: s = max|w| / 127, w_q = round(w / s) s."""
    co = w.shape[0]
    s = np.abs(w.reshape(co, -1)).max(axis=1) / 127.0
    s = np.where(s > 0, s, 1.0).reshape(-1, 1, 1, 1)
    return np.round(w / s) * s


def fq_act(z: np.ndarray):
    """Hidden activation: clamp(round(z / SCALE_A), 0, 127) SCALE_A, and the
    straight-through mask (1 where 0 < z / SCALE_A < 127.5)."""
    q = z / SCALE_A
    a = np.clip(np.round(q), 0, 127) * SCALE_A
    mask = ((q > 0) & (q < 127.5)).astype(z.dtype)
    return a, mask


def conv3x3_f(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """x [B, Ci, H, W], w [Co, Ci, 3, 3] -> [B, Co, H, W], zero padding."""
    B, ci, h, wd = x.shape
    pad = np.zeros((B, ci, h + 2, wd + 2), x.dtype)
    pad[:, :, 1:-1, 1:-1] = x
    out = np.zeros((B, w.shape[0], h, wd), x.dtype) + b.reshape(1, -1, 1, 1)
    for dy in range(3):
        for dx in range(3):
            out += np.einsum("oc,bchw->bohw", w[:, :, dy, dx], pad[:, :, dy:dy + h, dx:dx + wd])
    return out


def conv3x3_f_back(x: np.ndarray, w: np.ndarray, g: np.ndarray):
    """Gradients of conv3x3_f for upstream g: (dx, dw, db)."""
    B, ci, h, wd = x.shape
    pad = np.zeros((B, ci, h + 2, wd + 2), x.dtype)
    pad[:, :, 1:-1, 1:-1] = x
    dpad = np.zeros_like(pad)
    dw = np.zeros_like(w)
    for dy in range(3):
        for dx in range(3):
            dw[:, :, dy, dx] = np.einsum("bohw,bchw->oc", g, pad[:, :, dy:dy + h, dx:dx + wd])
            dpad[:, :, dy:dy + h, dx:dx + wd] += np.einsum("oc,bohw->bchw", w[:, :, dy, dx], g)
    return dpad[:, :, 1:-1, 1:-1], dw, g.sum(axis=(0, 2, 3))


def unflatten(theta: np.ndarray):
    """Flat parameter vector -> [(w, b)] per layer (layout: w_l then b_l, l = 1..4)."""
    out, o = [], 0
    for l in range(4):
        ci, co = CHANNELS[l], CHANNELS[l + 1]
        w = theta[o:o + co * ci * 9].reshape(co, ci, 3, 3)
        o += co * ci * 9
        b = theta[o:o + co]
        o += co
        out.append((w, b))
    return out


def n_params() -> int:
    return sum(CHANNELS[l + 1] * CHANNELS[l] * 9 + CHANNELS[l + 1] for l in range(4))


def forward_train(x: np.ndarray, theta: np.ndarray, quant: bool = True):
    """Float forward pass; returns (output [B, 3, H, W], cache for backward_train)."""
    layers = unflatten(np.asarray(theta, np.float64))
    a = np.asarray(x, np.float64)
    cache = []
    for l, (w, b) in enumerate(layers):
        wq = fq_weight(w) if quant else w
        z = conv3x3_f(a, wq, b)
        if l < 3:
            if quant:
                an, mask = fq_act(z)
            else:
                an, mask = np.maximum(z, 0.0), (z > 0).astype(z.dtype)
        else:
            an, mask = z, np.ones_like(z)
        cache.append((a, wq, mask))
        a = an
    return a, cache


def backward_train(dout: np.ndarray, cache) -> np.ndarray:
    """Gradient of the loss w.r.t. the flat parameters (straight-through
    through the weight and activation quantisers)."""
    g = np.asarray(dout, np.float64)
    grads = [None] * 4
    for l in range(3, -1, -1):
        a, wq, mask = cache[l]
        g = g * mask
        dx, dw, db = conv3x3_f_back(a, wq, g)
        grads[l] = (dw, db)
        g = dx
    return np.concatenate([np.concatenate([dw.reshape(-1), db]) for dw, db in grads])


def loss_l1(out: np.ndarray, target: np.ndarray):
    """Mean absolute error and its gradient (sign / count; 0 at ties)."""
    d = np.asarray(out, np.float64) - np.asarray(target, np.float64)
    return float(np.abs(d).mean()), np.sign(d) / d.size


def adam_step(theta, grad, m, v, step: int, lr: float, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (bias-corrected), returns (theta, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
