"""Python API of the coder: device buffers, encoder and decoder passes.

The encoder (Fig. 2, bottom) is rgbe_split -> sdri_base_roundtrip ->
slr_fit -> residual_encode; the decoder is residual_decode.  Every step runs
in the CUDA library through ``native``; torch only provides device memory
and streams.  Buffers are allocated once per image size and reused.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np
import torch

from . import native
from .metrics import enhancement_bits_per_pixel


@dataclasses.dataclass
class Layers:
    """What the encoder transmits (device tensors, views of Codec buffers).

    s3      decoded base-layer SDRI S, uint8 [3, h, w] (the base layer's content)
    e       exponent plane E, uint8 [h, w]
    r3      residual planes R = M - M*, int16 [3, h, w]
    params  SLRME parameters (slrme_params bytes as int32 [1796])
    hist    residual histograms, int32 [3, 511] (uint32 counts)
    """
    s3: torch.Tensor
    e: torch.Tensor
    r3: torch.Tensor
    params: torch.Tensor
    hist: torch.Tensor


def params_to_numpy(params: torch.Tensor) -> dict:
    """Parse a slrme_params buffer (host or device) into numpy arrays."""
    raw = params.detach().cpu().numpy().view(np.uint8)
    f = raw[:6144].view(np.float32)
    n = raw[6144:6144 + 1024].view(np.int32)
    n_used = int(raw[7168:7172].view(np.int32)[0])
    return dict(a=f[:768].reshape(3, 256).copy(), b=f[768:].reshape(3, 256).copy(), n=n.copy(), n_used=n_used)


def params_from_numpy(a: np.ndarray, b: np.ndarray, n: Optional[np.ndarray] = None) -> np.ndarray:
    """Build slrme_params bytes (as int32 [1796]) on the host."""
    raw = np.zeros(native.PARAMS_BYTES, np.uint8)
    raw[:3072] = np.ascontiguousarray(a, np.float32).reshape(-1).view(np.uint8)
    raw[3072:6144] = np.ascontiguousarray(b, np.float32).reshape(-1).view(np.uint8)
    nn = np.zeros(256, np.int32) if n is None else np.ascontiguousarray(n, np.int32)
    raw[6144:7168] = nn.view(np.uint8)
    raw[7168:7172] = np.array([int((nn > 0).sum())], np.int32).view(np.uint8)
    return raw.view(np.int32)


class Codec:
    """Encoder/decoder for images of one size on one CUDA device."""

    def __init__(self, h: int, w: int, device: str | torch.device = "cuda", gf_on: bool = True,
                 keep_sdr: bool = False):
        self.h, self.w = int(h), int(w)
        self.gf_on = int(bool(gf_on))
        dev = torch.device(device)
        if dev.type == "cuda" and dev.index is None:
            dev = torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        n = self.h * self.w
        d = self.device
        self.m3 = torch.empty(3 * n, dtype=torch.uint8, device=d)
        self.e = torch.empty(n, dtype=torch.uint8, device=d)
        self.stats = torch.zeros(2, dtype=torch.int64, device=d)
        self.s3 = torch.empty(3 * n, dtype=torch.uint8, device=d)
        self.sdr3 = torch.empty(3 * n, dtype=torch.uint8, device=d) if keep_sdr else None
        self.sums = torch.zeros(native.slr_fit_workspace_bytes() // 8, dtype=torch.int64, device=d)
        self.params = torch.zeros(native.PARAMS_BYTES // 4, dtype=torch.int32, device=d)
        self.r3 = torch.empty(3 * n, dtype=torch.int16, device=d)
        self.hist = torch.zeros(3 * native.SLRME_NRES, dtype=torch.int32, device=d)
        self.out = torch.empty(n, dtype=torch.int32, device=d)

    # ------------------------------------------------------------ encoder
    def encode(self, rgbe: torch.Tensor, quality: int, stream=None, hist: bool = True) -> Layers:
        """Encode packed RGBE words (int32 or uint32 view, h*w, on the device)."""
        h, w = self.h, self.w
        if rgbe.numel() != h * w or rgbe.device != self.device:
            raise ValueError("rgbe must hold h*w words on the codec's device")
        native.rgbe_split(rgbe, h, w, self.m3, self.e, self.stats, stream)
        native.sdri_base_roundtrip(self.m3, self.e, h, w, self.stats, quality, self.s3, self.sdr3, stream)
        native.slr_fit(self.s3, self.m3, self.e, h, w, self.gf_on, self.sums, self.params, stream)
        native.residual_encode(self.s3, self.m3, self.e, h, w, self.gf_on, self.params, self.r3,
                               self.hist if hist else None, stream)
        return self.layers()

    def layers(self) -> Layers:
        h, w = self.h, self.w
        return Layers(self.s3.view(3, h, w), self.e.view(h, w), self.r3.view(3, h, w), self.params,
                      self.hist.view(3, native.SLRME_NRES))

    # ------------------------------------------------------------ decoder
    def decode(self, s3: torch.Tensor, e: torch.Tensor, r3: torch.Tensor, params: torch.Tensor,
               out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        out = self.out if out is None else out
        native.residual_decode(s3, e, r3, self.h, self.w, self.gf_on, params, out, stream)
        return out

    # ------------------------------------------------------------ checks
    def check(self) -> None:
        """Waits for the device and raises if a kernel's bounded wait gave up
        since the last check (the library's status word); encode and decode
        are asynchronous, so their outputs are trustworthy after this."""
        native.check_device_status("Codec")

    # ------------------------------------------------------------ rate
    def bits_per_pixel(self) -> float:
        """Enhancement-layer rate: H0 of the residual planes + side information."""
        self.check()
        hist = self.hist.view(3, native.SLRME_NRES).cpu().numpy().view(np.uint32)
        n_used = params_to_numpy(self.params)["n_used"]
        return enhancement_bits_per_pixel(hist, n_used, self.h * self.w)


class HostCodec:
    """End-to-end use from host memory: pinned host RGBE in, host layers out.

    Each call copies the words host -> device, encodes and decodes on the
    device, and copies the enhancement layer (R, E, parameters, histograms),
    the base layer S and the decoded words back to pinned host buffers.
    Device codecs on separate streams take the calls in turn (slots), so the
    copies of one call overlap the coding of the next; within a call the
    encoder's outputs go back on a second stream while the decoder runs.
    Host buffers are per slot.
    """

    def __init__(self, h: int, w: int, device: str | torch.device = "cuda", gf_on: bool = True, slots: int = 3):
        self.slots = []
        n = h * w
        for _ in range(slots):
            c = Codec(h, w, device, gf_on)
            self.slots.append(dict(
                codec=c, stream=torch.cuda.Stream(device=c.device), out_stream=torch.cuda.Stream(device=c.device),
                done=None,
                d_rgbe=torch.empty(n, dtype=torch.int32, device=c.device),
                h_s3=torch.empty(3 * n, dtype=torch.uint8).pin_memory(),
                h_e=torch.empty(n, dtype=torch.uint8).pin_memory(),
                h_r3=torch.empty(3 * n, dtype=torch.int16).pin_memory(),
                h_params=torch.empty(native.PARAMS_BYTES // 4, dtype=torch.int32).pin_memory(),
                h_hist=torch.empty(3 * native.SLRME_NRES, dtype=torch.int32).pin_memory(),
                h_out=torch.empty(n, dtype=torch.int32).pin_memory()))
        self.turn = 0

    @property
    def h_out(self) -> torch.Tensor:
        return self.slots[(self.turn - 1) % len(self.slots)]["h_out"]

    def h2d_bytes(self) -> int:
        return self.slots[0]["d_rgbe"].numel() * 4

    def d2h_bytes(self) -> int:
        sl = self.slots[0]
        return sum(sl[k].numel() * sl[k].element_size() for k in ("h_s3", "h_e", "h_r3", "h_params", "h_hist", "h_out"))

    def roundtrip(self, rgbe_host: torch.Tensor, quality: int) -> None:
        """Enqueue one call on the next slot's streams (asynchronous).  The
        slot's previous call is complete before its buffers are reused: the
        coding stream waits for the slot's last copy back."""
        sl = self.slots[self.turn % len(self.slots)]
        self.turn += 1
        c, s, so = sl["codec"], sl["stream"], sl["out_stream"]
        if sl["done"] is not None:
            s.wait_event(sl["done"])
        with torch.cuda.stream(s):
            sl["d_rgbe"].copy_(rgbe_host, non_blocking=True)
            L = c.encode(sl["d_rgbe"], quality, stream=s)
            encoded = torch.cuda.Event()
            encoded.record(s)
            out = c.decode(L.s3, L.e, L.r3, L.params, stream=s)
            decoded = torch.cuda.Event()
            decoded.record(s)
        with torch.cuda.stream(so):
            so.wait_event(encoded)
            sl["h_s3"].copy_(c.s3, non_blocking=True)
            sl["h_e"].copy_(c.e, non_blocking=True)
            sl["h_r3"].copy_(c.r3, non_blocking=True)
            sl["h_params"].copy_(c.params, non_blocking=True)
            sl["h_hist"].copy_(c.hist, non_blocking=True)
            so.wait_event(decoded)
            sl["h_out"].copy_(out, non_blocking=True)
            done = torch.cuda.Event()
            done.record(so)
        sl["done"] = done

    def streams(self):
        return [st for sl in self.slots for st in (sl["stream"], sl["out_stream"])]

    def wait(self) -> None:
        """Waits for every call enqueued so far (its host buffers are then
        filled) and raises if a kernel's bounded wait gave up."""
        for st in self.streams():
            st.synchronize()
        native.check_device_status("HostCodec")
