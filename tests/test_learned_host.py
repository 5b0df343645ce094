"""Host logic of the learned estimator (no GPU): the packed network layout,
the float -> integer export and the per-image pick."""
import numpy as np

from oracle import cnn_oracle as C
from paper_2309_11072_gb300 import learned as Lr


def test_packed_layout_offsets():
    net = C.random_net(1)
    raw = Lr.pack_net(net)
    assert raw.size == Lr.NET_BYTES == 6044
    assert np.array_equal(raw[:576].view(np.int8).reshape(16, 4, 3, 3), net["w"][0])
    assert np.array_equal(raw[576 + 2 * 2304:5616].view(np.int8).reshape(3, 16, 3, 3), net["w"][3])
    i32 = raw[5616:].view(np.int32)
    assert np.array_equal(i32[:16], net["b"][0]) and np.array_equal(i32[48:51], net["b"][3])
    assert np.array_equal(i32[51:67], net["m"][0]) and np.array_equal(i32[99:102], net["m"][3])
    assert i32[102:106].tolist() == list(net["sh"])


def test_export_matches_fake_quantised_float_network():
    rng = np.random.default_rng(2)
    theta = rng.normal(0, 0.05, size=Lr.N_PARAMS)
    o = 0
    for l in range(4):                      # positive biases keep units active
        ci, co = C.CHANNELS[l], C.CHANNELS[l + 1]
        o += co * ci * 9
        theta[o:o + co] = 2.0 if l < 3 else 100.0
        o += co
    net = Lr.export_int_net(theta)
    for l in range(4):
        assert net["w"][l].dtype == np.int8 and np.abs(net["w"][l].astype(int)).max() <= 127
        assert (net["m"][l] > 0).all() and net["m"][l].max() < (1 << 24) and 1 <= net["sh"][l] <= 30
    s3 = rng.integers(0, 256, size=(3, 10, 12))
    e = rng.integers(120, 150, size=(10, 12))
    x = C.cnn_input(s3, e, J=0)[None].astype(np.float64)
    ref, _ = C.forward_train(x, theta, quant=True)
    got = C.infer(s3, e, 0, net).astype(np.float64)
    # integer requantisation vs float rounding: within a few grey levels
    assert np.abs(got - np.clip(np.rint(ref[0]), 0, 255)).mean() < 1.0


def test_pick_prefers_the_cheaper_residuals():
    n = 10000
    wide = np.zeros((3, 511), np.uint32)
    narrow = np.zeros((3, 511), np.uint32)
    for c in range(3):
        wide[c, 255 - 20:255 + 20] = n // 40
        narrow[c, 255 - 2:255 + 2] = n // 4
    p = Lr.pick_image(wide, 10, narrow, n)
    assert p.use_cnn and p.bits == p.bits_cnn < p.bits_slr
    q = Lr.pick_image(narrow, 10, wide, n)
    assert not q.use_cnn and q.bits == q.bits_slr
