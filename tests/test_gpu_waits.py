"""The bounded waits of the TMA-staged kernels, tested without any fault:
a wait that nothing completes gives up after its bound, reports through the
device status word, and leaves the CUDA context usable; a wait that is
completed leaves the word alone."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2309_11072_gb300 import codec, native, synth

pytestmark = pytest.mark.gpu


def test_wait_that_nothing_completes_gives_up_and_reports():
    native.lib()
    native.device_status(clear=True)
    native.wait_probe(1000, arrive=False)
    torch.cuda.synchronize()
    assert native.device_status(clear=True) == 1
    # the context still works: a small encode / decode after the timeout
    h, w = 33, 64
    img = synth.make_rgbe(h, w, seed=5, lo=-2.0, hi=4.0)
    c = codec.Codec(h, w, "cuda")
    L = c.encode(torch.from_numpy(img.view(np.int32).reshape(-1).copy()).cuda(), 75)
    out = c.decode(L.s3, L.e, L.r3, L.params)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint32).reshape(h, w), img)
    assert np.array_equal(L.r3.cpu().numpy().reshape(3, h, w), O.encode(img, 75)["r3"])
    assert native.device_status(clear=True) == 0


def test_completed_wait_leaves_status_clear():
    native.lib()
    native.device_status(clear=True)
    native.wait_probe(1000, arrive=True)
    torch.cuda.synchronize()
    assert native.device_status(clear=True) == 0


def test_wait_probe_rejects_bad_bounds():
    L = native.lib()
    assert L.slrme_wait_probe(0, 0, None) == -1
    assert L.slrme_wait_probe(1 << 21, 0, None) == -1
    assert L.slrme_wait_probe(10, 2, None) == -1


def test_python_api_raises_on_a_wait_that_gave_up():
    """The Python API's checks (Codec.check, used by bits_per_pixel; the
    batch form's parameter and statistic reads) read the status word after
    waiting for the device: a wait that gave up raises, and the word is
    cleared so the next check passes."""
    native.lib()
    native.device_status(clear=True)
    h, w = 16, 32
    c = codec.Codec(h, w, "cuda")
    c.check()
    native.wait_probe(1000, arrive=False)
    with pytest.raises(native.SlrmeError) as err:
        c.check()
    assert err.value.code == native.DEVICE_STATUS_ERROR
    c.check()
    native.wait_probe(1000, arrive=False)
    img = synth.make_rgbe(h, w, seed=6, lo=-2.0, hi=4.0)
    c.encode(torch.from_numpy(img.view(np.int32).reshape(-1).copy()).cuda(), 75)
    with pytest.raises(native.SlrmeError):
        c.bits_per_pixel()
    assert c.bits_per_pixel() > 0
