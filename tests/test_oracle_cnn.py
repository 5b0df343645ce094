"""Pins for the CNN oracle: scipy correlation, exact integer rounding,
closed-form networks, finite differences, and torch's Adam."""
from fractions import Fraction

import numpy as np
import pytest
from scipy.signal import correlate2d

from oracle import cnn_oracle as C


def test_int_conv_against_scipy():
    rng = np.random.default_rng(1)
    a = rng.integers(-128, 128, size=(4, 9, 11))
    w = rng.integers(-127, 128, size=(5, 4, 3, 3))
    out = C.conv3x3_int(a, w)
    for o in range(5):
        ref = sum(correlate2d(a[c], w[o, c], mode="same", boundary="fill", fillvalue=0) for c in range(4))
        assert np.array_equal(out[o], ref)


def test_requant_is_round_half_up_of_the_exact_ratio():
    rng = np.random.default_rng(2)
    acc = rng.integers(-3_000_000, 3_000_000, size=(3, 4, 5))
    acc[0, 0, :3] = [0, -1, 1]
    m = rng.integers(1, 1 << 15, size=3)
    for sh in (1, 7, 20, 24):
        y = C.requant(acc, m, sh, -(1 << 40), 1 << 40)
        for idx in np.ndindex(acc.shape):
            exact = Fraction(int(acc[idx]) * int(m[idx[0]]), 1 << sh) + Fraction(1, 2)
            assert y[idx] == exact.__floor__()
    assert C.requant(np.array([[[10 ** 6]]]), np.array([1 << 10]), 10, 0, 127)[0, 0, 0] == 127
    assert C.requant(np.array([[[-5]]]), np.array([3]), 2, 0, 127)[0, 0, 0] == 0


def test_constant_network_outputs_its_biases():
    net = C.random_net(3)
    for l in range(4):
        net["w"][l][:] = 0
        net["m"][l][:] = 1 << 10
        net["sh"][l] = 10
    net["b"][3][:] = [7, 300, -4]
    s3 = np.random.default_rng(4).integers(0, 256, size=(3, 6, 7))
    e = np.full((6, 7), 130)
    out = C.infer(s3, e, 2, net)
    assert (out[0] == 7).all() and (out[1] == 255).all() and (out[2] == 0).all()


def test_delta_network_reproduces_the_red_plane():
    # layer 1 keeps S_R - 128 + 128 (bias) in channel 0; layers 2-4 copy channel 0
    net = C.random_net(5)
    for l in range(4):
        net["w"][l][:] = 0
        net["w"][l][0, 0, 1, 1] = 1
        net["b"][l][:] = 0
        net["m"][l][:] = 1 << 20
        net["sh"][l] = 20
    net["b"][0][0] = 128 - 1          # S_R - 1 stays in [0, 127] for S_R in [1, 128]
    s3 = np.random.default_rng(6).integers(1, 129, size=(3, 8, 9))
    out = C.infer(s3, np.full((8, 9), 140), 0, net)
    assert np.array_equal(out[0], s3[0] - 1)


def test_hidden_activations_saturate_at_127():
    # every hidden layer's bias alone would give 200 and -50: the ReLU clamp
    # keeps 127 and 0; the last layer sums one 3x3 window of channel 0 with
    # weight 1 and bias 0: 9 x 127 inside the image (over 255 after the / 4:
    # the output clamp), fewer on the zero-padded border
    net = C.random_net(7)
    for l in range(4):
        net["w"][l][:] = 0
        net["m"][l][:] = 1 << 12
        net["sh"][l] = 12
        net["b"][l][:] = 200
        if l < 3:
            net["b"][l][1::2] = -50
    net["w"][3][:, 0] = 1
    net["b"][3][:] = 0
    net["m"][3][:] = 1 << 10                 # the sum / 4, rounded half up
    s3 = np.random.default_rng(8).integers(0, 256, size=(3, 5, 6))
    out = C.infer(s3, np.full((5, 6), 133), 1, net).astype(int)
    cover = np.full((5, 6), 9)
    cover[[0, -1], :] -= 3
    cover[:, [0, -1]] -= 3
    cover[[0, 0, -1, -1], [0, -1, 0, -1]] = 4
    assert np.array_equal(out, np.stack([np.minimum((cover * 127 + 2) // 4, 255)] * 3))


def test_input_planes():
    s3 = np.array([[[0, 255]], [[128, 1]], [[7, 9]]])
    e = np.array([[0, 250]])
    x = C.cnn_input(s3, e, J=-3)
    assert x[:3].tolist() == [[[-128, 127]], [[0, -127]], [[-121, -119]]]
    assert x[3].tolist() == [[-128, 116]]


def _fd_check(f, theta, grad, idxs, eps=1e-6):
    for i in idxs:
        t1 = theta.copy()
        t1[i] += eps
        t2 = theta.copy()
        t2[i] -= eps
        num = (f(t1) - f(t2)) / (2 * eps)
        assert abs(num - grad[i]) <= 1e-6 + 1e-5 * abs(num), (i, num, grad[i])


def test_backward_against_finite_differences():
    rng = np.random.default_rng(7)
    theta = rng.normal(0, 0.2, size=C.n_params())
    x = rng.normal(0, 1, size=(2, 4, 6, 5))
    target = rng.normal(0, 1, size=(2, 3, 6, 5))

    def f(t):
        out, _ = C.forward_train(x, t, quant=False)
        return 0.5 * float(((out - target) ** 2).sum())

    out, cache = C.forward_train(x, theta, quant=False)
    grad = C.backward_train(out - target, cache)
    idxs = list(rng.choice(C.n_params(), size=40, replace=False)) + [0, C.n_params() - 1]
    _fd_check(f, theta, grad, idxs)


def test_l1_loss_gradient():
    rng = np.random.default_rng(8)
    out = rng.normal(size=(2, 3, 4, 4))
    tgt = rng.normal(size=(2, 3, 4, 4))
    loss, g = C.loss_l1(out, tgt)
    assert abs(loss - np.abs(out - tgt).mean()) < 1e-12
    eps = 1e-7
    for idx in [(0, 0, 0, 0), (1, 2, 3, 1)]:
        o1 = out.copy()
        o1[idx] += eps
        assert abs((C.loss_l1(o1, tgt)[0] - loss) / eps - g[idx]) < 1e-6


def test_adam_against_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(9)
    theta = rng.normal(size=50)
    p = torch.tensor(theta.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([p], lr=1e-2)
    m = np.zeros(50)
    v = np.zeros(50)
    for step in range(1, 6):
        g = rng.normal(size=50)
        opt.zero_grad()
        p.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        theta, m, v = C.adam_step(theta, g, m, v, step, lr=1e-2)
        assert np.allclose(theta, p.detach().numpy(), rtol=1e-12, atol=1e-12)


def test_fake_quantisers():
    rng = np.random.default_rng(10)
    w = rng.normal(size=(4, 3, 3, 3))
    wq = C.fq_weight(w)
    s = np.abs(w.reshape(4, -1)).max(axis=1) / 127
    k = wq.reshape(4, -1) / s[:, None]
    assert np.allclose(k, np.round(k)) and (np.abs(k) <= 127 + 1e-9).all()
    z = np.array([-1.0, 0.0, 0.06, 0.07, 3.0, 15.875, 16.0, 100.0]) * 1.0
    a, mask = C.fq_act(z)
    assert a.tolist() == [0.0, 0.0, 0.0, 0.125, 3.0, 15.875, 15.875, 15.875]
    assert mask.tolist() == [0, 0, 1, 1, 1, 1, 0, 0]


def test_neutral_correction_keeps_the_regression_estimate():
    # a network whose output is 128 everywhere leaves M* unchanged
    from oracle import oracle as O
    net = C.random_net(7)
    for l in range(4):
        net["w"][l][:] = 0
        net["m"][l][:] = 1 << 10
        net["sh"][l] = 10
    net["b"][3][:] = 128
    rng = np.random.default_rng(8)
    s3 = rng.integers(0, 256, size=(3, 6, 9)).astype(np.uint8)
    e = rng.integers(120, 140, size=(6, 9)).astype(np.uint8)
    a = rng.uniform(-0.1, 0.1, (3, 256)).astype(np.float32)
    b = rng.uniform(0, 255, (3, 256)).astype(np.float32)
    ms = O.predict(O.gf(s3), e, a, b)
    assert np.array_equal(C.refine(ms, C.infer(s3, e, 0, net)), ms)
    assert C.refine(np.array([[[250, 3]]]), np.array([[[200, 10]]])).tolist() == [[[255, 0]]]
