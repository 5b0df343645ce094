"""Batch form: many images of uneven sizes through the slrme_batch_* C ABI.

ctypes mirrors of the plan structs plus a small owner class that allocates the
torch device buffers, lays the images out as the plan says, and calls the
library (encode, decode, autotune, CUDA-graph build and launch).  All coding
work runs in the library's persistent stage kernels.
"""
from __future__ import annotations

import ctypes
from typing import List, Sequence, Tuple

import numpy as np
import torch

from . import native
from .codec import params_to_numpy


class BatchImage(ctypes.Structure):
    _fields_ = [("h", ctypes.c_int32), ("w", ctypes.c_int32), ("quality", ctypes.c_int32),
                ("gf_on", ctypes.c_int32), ("px_offset", ctypes.c_int64), ("pitch", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class BatchTiles(ctypes.Structure):
    _fields_ = [("split_ctas_per_sm", ctypes.c_int32), ("base_ctas_per_sm", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class BatchPlan(ctypes.Structure):
    _fields_ = [("n_images", ctypes.c_int32), ("total_px", ctypes.c_int64),
                ("images", ctypes.POINTER(BatchImage)), ("workspace", ctypes.c_void_p),
                ("tiles", BatchTiles), ("split_chunks", ctypes.c_int64), ("base_tasks", ctypes.c_int64),
                ("tile_rows", ctypes.c_int64), ("graph", ctypes.c_void_p)]


class BatchBuffers(ctypes.Structure):
    _fields_ = [("rgbe", ctypes.c_void_p), ("m3", ctypes.c_void_p), ("e", ctypes.c_void_p), ("s3", ctypes.c_void_p),
                ("r3", ctypes.c_void_p), ("params", ctypes.c_void_p), ("hist", ctypes.c_void_p),
                ("rgbe_out", ctypes.c_void_p)]


_vp = ctypes.c_void_p
_BATCH_SIGS = {
    "slrme_batch_plan_init": [_vp, _vp, ctypes.c_int, _vp, _vp],
    "slrme_batch_set_tiles": [_vp, _vp, _vp],
    "slrme_batch_encode": [_vp, _vp, _vp],
    "slrme_batch_decode": [_vp, _vp, _vp],
    "slrme_batch_autotune": [_vp, _vp, ctypes.c_int, _vp],
    "slrme_batch_graph_build": [_vp, _vp, _vp],
    "slrme_batch_graph_launch": [_vp, _vp],
    "slrme_batch_graph_destroy": [_vp],
    "slrme_batch_lum_stats": [_vp, _vp, _vp],
}


def _lib():
    L = native.lib()
    if not getattr(L, "_batch_sigs", False):
        for name, args in _BATCH_SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.slrme_batch_workspace_bytes.argtypes = [ctypes.c_int]
        L.slrme_batch_workspace_bytes.restype = ctypes.c_size_t
        L._batch_sigs = True
    return L


def _call(name, *args):
    rc = getattr(_lib(), name)(*args)
    if rc != 0:
        raise native.SlrmeError(name, rc, native.last_error())


class BatchCodec:
    """Owns a plan, its workspace and the batch planes for a list of image sizes."""

    def __init__(self, sizes: Sequence[Tuple[int, int]], qualities: Sequence[int], gf_on=True,
                 device: str = "cuda"):
        """gf_on: one restoration flag for every image, or one per image."""
        n = len(sizes)
        if n < 1 or len(qualities) != n:
            raise ValueError("need one quality per image")
        gfs = [bool(gf_on)] * n if isinstance(gf_on, (bool, int)) else [bool(g) for g in gf_on]
        if len(gfs) != n:
            raise ValueError("need one restoration flag per image")
        self.device = torch.device(device)
        self.images = (BatchImage * n)()
        for i, ((h, w), q, g) in enumerate(zip(sizes, qualities, gfs)):
            self.images[i] = BatchImage(int(h), int(w), int(q), int(g), 0, 0, 0)
        self.ws = torch.zeros(int(_lib().slrme_batch_workspace_bytes(n)), dtype=torch.uint8, device=self.device)
        self.plan = BatchPlan()
        _call("slrme_batch_plan_init", ctypes.addressof(self.plan), ctypes.addressof(self.images), n,
              self.ws.data_ptr(), torch.cuda.current_stream(self.device).cuda_stream)
        P = int(self.plan.total_px)
        d = self.device
        self.rgbe = torch.zeros(P, dtype=torch.int32, device=d)
        self.m3 = torch.zeros(3 * P, dtype=torch.uint8, device=d)
        self.e = torch.zeros(P, dtype=torch.uint8, device=d)
        self.s3 = torch.zeros(3 * P, dtype=torch.uint8, device=d)
        self.r3 = torch.zeros(3 * P, dtype=torch.int16, device=d)
        self.params = torch.zeros(n * native.PARAMS_BYTES // 4, dtype=torch.int32, device=d)
        self.hist = torch.zeros(n * 3 * native.SLRME_NRES, dtype=torch.int32, device=d)
        self.out = torch.zeros(P, dtype=torch.int32, device=d)
        self.bufs = BatchBuffers(self.rgbe.data_ptr(), self.m3.data_ptr(), self.e.data_ptr(), self.s3.data_ptr(),
                                 self.r3.data_ptr(), self.params.data_ptr(), self.hist.data_ptr(), self.out.data_ptr())
        self.n = n

    # ------------------------------------------------------------ layout helpers
    def offset(self, i: int) -> int:
        return int(self.images[i].px_offset)

    def size(self, i: int) -> Tuple[int, int]:
        return int(self.images[i].h), int(self.images[i].w)

    def pitch(self, i: int) -> int:
        """Row pitch (elements) of every plane of image i."""
        return int(self.images[i].pitch)

    def load(self, imgs: List[np.ndarray]) -> None:
        """Copy host RGBE images (uint32 [h, w]) into the batch word plane
        (rows at the image's pitch, padding words zero)."""
        host = np.zeros(int(self.plan.total_px), dtype=np.uint32)
        for i, img in enumerate(imgs):
            h, w = self.size(i)
            assert img.shape == (h, w)
            o, p = self.offset(i), self.pitch(i)
            host[o:o + h * p].reshape(h, p)[:, :w] = img
        self.rgbe.copy_(torch.from_numpy(host.view(np.int32)))

    def _plane3(self, t: torch.Tensor, i: int) -> torch.Tensor:
        h, w = self.size(i)
        o, p = 3 * self.offset(i), self.pitch(i)
        return t[o:o + 3 * h * p].view(3, h, p)[:, :, :w]

    def _plane1(self, t: torch.Tensor, i: int) -> torch.Tensor:
        h, w = self.size(i)
        o, p = self.offset(i), self.pitch(i)
        return t[o:o + h * p].view(h, p)[:, :w]

    def image_layers(self, i: int) -> dict:
        """Views of image i's planes ([3, h, w] / [h, w], row stride = pitch)."""
        return dict(m3=self._plane3(self.m3, i), e=self._plane1(self.e, i), s3=self._plane3(self.s3, i),
                    r3=self._plane3(self.r3, i), out=self._plane1(self.out, i),
                    params=self.params[i * native.PARAMS_BYTES // 4:(i + 1) * native.PARAMS_BYTES // 4],
                    hist=self.hist[i * 3 * native.SLRME_NRES:(i + 1) * 3 * native.SLRME_NRES].view(3, -1))

    def dense_layers(self, i: int) -> dict:
        """image_layers with every plane copied to a dense tensor (rows of w
        elements), the layout the single-image entry points take."""
        return {k: (v.contiguous() if k in ("m3", "e", "s3", "r3", "out") else v)
                for k, v in self.image_layers(i).items()}

    def image_params(self, i: int) -> dict:
        native.check_device_status("BatchCodec")
        return params_to_numpy(self.image_layers(i)["params"])

    # ------------------------------------------------------------ calls
    def _stream(self, stream=None) -> int:
        return (stream or torch.cuda.current_stream(self.device)).cuda_stream

    def encode(self, stream=None) -> None:
        _call("slrme_batch_encode", ctypes.addressof(self.plan), ctypes.addressof(self.bufs), self._stream(stream))

    def decode(self, stream=None) -> None:
        _call("slrme_batch_decode", ctypes.addressof(self.plan), ctypes.addressof(self.bufs), self._stream(stream))

    def set_tiles(self, **kw) -> None:
        t = BatchTiles(**{**self.plan.tiles.as_dict(), **kw})
        _call("slrme_batch_set_tiles", ctypes.addressof(self.plan), ctypes.addressof(t), self._stream())

    def autotune(self, reps: int = 3) -> dict:
        _call("slrme_batch_autotune", ctypes.addressof(self.plan), ctypes.addressof(self.bufs), int(reps),
              self._stream())
        return self.plan.tiles.as_dict()

    def graph_build(self, stream: torch.cuda.Stream) -> None:
        _call("slrme_batch_graph_build", ctypes.addressof(self.plan), ctypes.addressof(self.bufs), stream.cuda_stream)

    def graph_launch(self, stream=None) -> None:
        _call("slrme_batch_graph_launch", ctypes.addressof(self.plan), self._stream(stream))

    def lum_stats(self) -> np.ndarray:
        """Per-image log-average statistics of the last encode (int64 [n, 2])."""
        native.check_device_status("BatchCodec")
        out = np.zeros((self.n, 2), np.int64)
        _call("slrme_batch_lum_stats", ctypes.addressof(self.plan), out.ctypes.data, self._stream())
        return out

    def keys(self) -> list:
        """Tone-mapping key J of every image (from the last encode)."""
        return [native.rgbe_key_scale(st)[0] for st in self.lum_stats()]

    def close(self) -> None:
        if self.plan.graph:
            _call("slrme_batch_graph_destroy", ctypes.addressof(self.plan))

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
