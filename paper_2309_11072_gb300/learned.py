"""Learned mantissa estimator: packing, GPU training loop, per-image pick.

The network and its integer arithmetic are defined in include/slrme.h
(cnn_*); this module marshals arguments, runs the training loop whose every
step is a library kernel (crop gather, forward, loss, backward, Adam), turns
the trained float weights into the integer network, and picks, image by
image, the estimator whose residuals cost fewer bits (the regression of
Eq. 8 stays the fallback and the yardstick).
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
from typing import Dict, List, Optional, Sequence

import numpy as np
import torch

from . import native
from .metrics import entropy_bits

CHANNELS = (4, 16, 16, 16, 3)
SCALE_A = 1.0 / 8.0
N_PARAMS = 5667
NET_BYTES = 6044
_W_OFF = (0, 576, 576 + 2304, 576 + 2 * 2304)          # int8 weights of layers 1..4
_I32_OFF = 5616                                         # b1, b2, b3, b4, m1, ..., m4, shift[4], reserved

_vp = ctypes.c_void_p
_SIGS = {
    "cnn_infer": [_vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int32, _vp, _vp, _vp],
    "cnn_residual_encode": [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int32, _vp, _vp, ctypes.c_int, _vp,
                            _vp, _vp],
    "cnn_residual_decode": [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int32, _vp, _vp, ctypes.c_int, _vp,
                            _vp],
    "cnn_train_forward": [_vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp],
    "cnn_train_backward": [_vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp],
    "cnn_loss_l1": [_vp, _vp, ctypes.c_int64, _vp, _vp, _vp, _vp],
    "cnn_adam_step": [_vp, _vp, _vp, _vp, ctypes.c_int, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                      ctypes.c_float, ctypes.c_int, _vp],
    "cnn_gather_crops": [_vp, _vp, _vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp],
}


def _lib():
    L = native.lib()
    if not getattr(L, "_cnn_sigs", False):
        for name, args in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.cnn_train_workspace_bytes.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.cnn_train_workspace_bytes.restype = ctypes.c_size_t
        L._cnn_sigs = True
    return L


def _call(name, *args):
    rc = getattr(_lib(), name)(*args)
    if rc != 0:
        raise native.SlrmeError(name, rc, native.last_error())


def _ptr(t):
    return None if t is None else native._ptr(t)


def _stream(stream=None):
    return (stream or torch.cuda.current_stream()).cuda_stream


# ------------------------------------------------------------------ integer network

def pack_net(net: dict) -> np.ndarray:
    """Integer network (w: 4 int8 arrays [co][ci][3][3], b, m: int32 [co], sh: 4 ints)
    -> the bytes of slrme_cnn_net."""
    raw = np.zeros(NET_BYTES, np.uint8)
    for l in range(4):
        w = np.ascontiguousarray(net["w"][l], np.int8).reshape(-1)
        raw[_W_OFF[l]:_W_OFF[l] + w.size] = w.view(np.uint8)
    i32 = np.zeros((NET_BYTES - _I32_OFF) // 4, np.int32)
    o = 0
    for key in ("b", "m"):
        for l in range(4):
            v = np.asarray(net[key][l], np.int32)
            i32[o:o + v.size] = v
            o += v.size
    i32[o:o + 4] = np.asarray(net["sh"], np.int32)
    raw[_I32_OFF:] = i32.view(np.uint8)
    return raw


def export_int_net(theta: np.ndarray) -> dict:
    """Trained float parameters (fake-quantised training) -> the integer network.

    Layer l has input scale s_in (1 for the raw int8 input, SCALE_A after),
    weight scale s_w = max|w| / 127 per output channel and output scale s_out
    (SCALE_A for hidden layers, 1 for the mantissa output).  Then w_int =
    round(w / s_w), bias = round(b / (s_w s_in)) and m / 2^shift ~ s_w s_in / s_out.
    """
    theta = np.asarray(theta, np.float64)
    net = {"w": [], "b": [], "m": [], "sh": []}
    o = 0
    for l in range(4):
        ci, co = CHANNELS[l], CHANNELS[l + 1]
        w = theta[o:o + co * ci * 9].reshape(co, ci, 3, 3)
        o += co * ci * 9
        b = theta[o:o + co]
        o += co
        s_w = np.abs(w.reshape(co, -1)).max(axis=1) / 127.0
        s_w = np.where(s_w > 0, s_w, 1.0)
        s_in = 1.0 if l == 0 else SCALE_A
        s_out = SCALE_A if l < 3 else 1.0
        ratio = s_w * s_in / s_out
        sh = int(min(30, math.floor(math.log2((1 << 23) / ratio.max()))))
        net["w"].append(np.clip(np.rint(w / s_w.reshape(-1, 1, 1, 1)), -127, 127).astype(np.int8))
        net["b"].append(np.rint(b / (s_w * s_in)).astype(np.int32))
        net["m"].append(np.maximum(1, np.rint(ratio * (1 << sh))).astype(np.int32))
        net["sh"].append(sh)
    return net


def load_net(path: str) -> dict:
    """Integer network saved by learned_eval (--weights)."""
    z = np.load(path)
    return {"w": [z[f"w{l}"] for l in range(4)], "b": [z[f"b{l}"] for l in range(4)],
            "m": [z[f"m{l}"] for l in range(4)], "sh": [int(v) for v in z["sh"]]}


def default_weights() -> str:
    import os
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "cnn_refine_q90.npz")


def upload_net(net: dict, device="cuda") -> torch.Tensor:
    return torch.from_numpy(pack_net(net).view(np.int32).copy()).to(device)


# ------------------------------------------------------------------ inference entry points

def cnn_infer(s3, e, h, w, J, net_dev, mhat3, stream=None):
    _call("cnn_infer", _ptr(s3), _ptr(e), h, w, int(J), _ptr(net_dev), _ptr(mhat3), _stream(stream))


def cnn_residual_encode(s3, m3, e, h, w, J, net_dev, params, gf_on, r3, hist=None, stream=None):
    _call("cnn_residual_encode", _ptr(s3), _ptr(m3), _ptr(e), h, w, int(J), _ptr(net_dev), _ptr(params),
          int(gf_on), _ptr(r3), _ptr(hist), _stream(stream))


def cnn_residual_decode(s3, e, r3, h, w, J, net_dev, params, gf_on, out, stream=None):
    _call("cnn_residual_decode", _ptr(s3), _ptr(e), _ptr(r3), h, w, int(J), _ptr(net_dev), _ptr(params),
          int(gf_on), _ptr(out), _stream(stream))


# ------------------------------------------------------------------ training

class Trainer:
    """Float32 training state and buffers for batches of B crops of H x W."""

    def __init__(self, B: int, H: int, W: int, seed: int = 0, quant: bool = True, lr: float = 2e-3,
                 device="cuda"):
        self.B, self.H, self.W, self.quant, self.lr = B, H, W, int(bool(quant)), lr
        d = torch.device(device)
        rng = np.random.default_rng(seed)
        theta = np.zeros(N_PARAMS, np.float32)
        o = 0
        for l in range(4):
            ci, co = CHANNELS[l], CHANNELS[l + 1]
            fan_in = ci * 9
            scale = math.sqrt(2.0 / fan_in) if l < 3 else math.sqrt(1.0 / fan_in)
            if l == 0:
                scale /= 64.0     # raw int8 inputs span +-128: keep first activations inside [0, 127/8]
            theta[o:o + co * ci * 9] = rng.normal(0, scale, co * ci * 9)
            o += co * ci * 9
            theta[o:o + co] = 1.0 if l < 3 else 128.0        # hidden units start active; output near mid-range
            o += co
        self.theta = torch.from_numpy(theta).to(d)
        self.m = torch.zeros(N_PARAMS, dtype=torch.float32, device=d)
        self.v = torch.zeros(N_PARAMS, dtype=torch.float32, device=d)
        self.grad = torch.zeros(N_PARAMS, dtype=torch.float32, device=d)
        self.ws = torch.zeros(int(_lib().cnn_train_workspace_bytes(B, H, W)) // 4, dtype=torch.float32, device=d)
        n = B * H * W
        self.x = torch.zeros(B * 4 * H * W, dtype=torch.float32, device=d)
        self.t = torch.zeros(B * 3 * H * W, dtype=torch.float32, device=d)
        self.out = torch.zeros(B * 3 * H * W, dtype=torch.float32, device=d)
        self.dout = torch.zeros(B * 3 * H * W, dtype=torch.float32, device=d)
        self.loss = torch.zeros(1, dtype=torch.float32, device=d)
        self.loss_ws = torch.zeros((3 * n + 255) // 256 + 1, dtype=torch.float32, device=d)
        self.step_no = 0

    def forward(self, x=None, stream=None):
        x = self.x if x is None else x
        _call("cnn_train_forward", _ptr(self.theta), _ptr(x), self.B, self.H, self.W, self.quant, _ptr(self.ws),
              _ptr(self.out), _stream(stream))
        return self.out

    def backward(self, dout=None, x=None, stream=None):
        x = self.x if x is None else x
        dout = self.dout if dout is None else dout
        _call("cnn_train_backward", _ptr(x), _ptr(dout), self.B, self.H, self.W, self.quant, _ptr(self.ws),
              _ptr(self.grad), _stream(stream))
        return self.grad

    def loss_l1(self, stream=None):
        _call("cnn_loss_l1", _ptr(self.out), _ptr(self.t), self.out.numel(), _ptr(self.dout), _ptr(self.loss),
              _ptr(self.loss_ws), _stream(stream))
        return self.loss

    def adam(self, stream=None):
        self.step_no += 1
        _call("cnn_adam_step", _ptr(self.theta), _ptr(self.grad), _ptr(self.m), _ptr(self.v), N_PARAMS,
              float(self.lr), 0.9, 0.999, 1e-8, self.step_no, _stream(stream))

    def step(self, crops_dev, s3, e, r3, stream=None):
        """One training step on the crops (int64 [B, 6] on the device) of coded
        images: decoded SDRI s3, exponents e and the regression's residuals r3."""
        _call("cnn_gather_crops", _ptr(s3), _ptr(e), _ptr(r3), _ptr(crops_dev), self.B, self.H, self.W,
              _ptr(self.x), _ptr(self.t), _stream(stream))
        self.forward(stream=stream)
        self.loss_l1(stream=stream)
        self.backward(stream=stream)
        self.adam(stream=stream)

    def state(self) -> dict:
        return dict(theta=self.theta.cpu().numpy().copy(), m=self.m.cpu().numpy().copy(),
                    v=self.v.cpu().numpy().copy(), step=self.step_no)

    def load_state(self, st: dict) -> None:
        self.theta.copy_(torch.from_numpy(np.asarray(st["theta"], np.float32)))
        self.m.copy_(torch.from_numpy(np.asarray(st["m"], np.float32)))
        self.v.copy_(torch.from_numpy(np.asarray(st["v"], np.float32)))
        self.step_no = int(st["step"])


def crop_table(bc, keys: Sequence[int], B: int, H: int, W: int, rng: np.random.Generator) -> np.ndarray:
    """B random crops of H x W from the images of a BatchCodec (int64 [B, 6])."""
    rows = []
    n = bc.n
    while len(rows) < B:
        i = int(rng.integers(0, n))
        h, w = bc.size(i)
        if h < H or w < W:
            continue
        # the crop table's third entry is the row pitch of the image's planes
        rows.append((bc.offset(i), h, bc.pitch(i), int(rng.integers(0, h - H + 1)), int(rng.integers(0, w - W + 1)),
                     int(keys[i])))
    return np.asarray(rows, np.int64)


def train(bc, keys: Sequence[int], steps: int, B: int = 32, H: int = 64, W: int = 64, seed: int = 0,
          lr: float = 2e-3, log_every: int = 0, history: Optional[list] = None) -> Trainer:
    """Train on crops of the coded images held by a BatchCodec (encode first).
    Every `log_every` steps the L1 loss is appended to `history` (if given)."""
    tr = Trainer(B, H, W, seed=seed, lr=lr, device=bc.device)
    rng = np.random.default_rng(seed + 1)
    crops = torch.zeros((B, 6), dtype=torch.int64, device=bc.device)
    for k in range(steps):
        crops.copy_(torch.from_numpy(crop_table(bc, keys, B, H, W, rng)))
        tr.step(crops, bc.s3, bc.e, bc.r3)
        if log_every and (k == 0 or (k + 1) % log_every == 0):
            loss = float(tr.loss.item())
            if history is not None:
                history.append((k + 1, loss))
    return tr


# ------------------------------------------------------------------ per-image pick

@dataclasses.dataclass
class Pick:
    bits_slr: float
    bits_cnn: float
    use_cnn: bool

    @property
    def bits(self) -> float:
        return min(self.bits_slr, self.bits_cnn)


def rate(hist3: np.ndarray, side_bits: float, n_px: int) -> float:
    """Bits per pixel of three residual planes (order-0 entropy) plus side information."""
    return sum(entropy_bits(h) for h in hist3) + side_bits / float(n_px)


def pick_image(hist_slr: np.ndarray, n_used: int, hist_cnn: np.ndarray, n_px: int) -> Pick:
    """The 1-bit per-image choice: the network only where its residuals cost
    fewer bits than the regression's.  Both carry the regression's parameters
    (the network refines that estimate); the network's residuals also carry
    the key J; the flag costs one bit either way."""
    side = 256 + 3 * 64 * n_used + 1
    b_slr = rate(hist_slr, side, n_px)
    b_cnn = rate(hist_cnn, side + 32, n_px)
    return Pick(b_slr, b_cnn, b_cnn < b_slr)
