"""Pins of the FP64 network oracle (CPU): the library convolution against
plain loops, autograd against central finite differences, the loss in
closed form."""
import numpy as np
import torch

from oracle import net_oracle as no


def test_conv_matches_loops_with_dilation():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 3, 7, 9))
    W = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    for d in (1, 2, 4):
        ref = no.conv_loops(x, W, b, d)
        out = torch.nn.functional.conv2d(torch.tensor(x), torch.tensor(W), torch.tensor(b),
                                         padding=d, dilation=d).numpy()
        np.testing.assert_allclose(out, ref, atol=1e-12)


def test_master_layout_round_trip():
    rng = np.random.default_rng(1)
    w = rng.normal(size=no.weight_count())
    layers = no.unpack(w)
    W0 = layers[0][0].numpy()  # (32, 2, 3, 3)
    # master W[co][ky*3+kx][ci]
    co, ci, ky, kx = 5, 1, 2, 0
    assert W0[co, ci, ky, kx] == w[(co * 9 + ky * 3 + kx) * 2 + ci]
    assert layers[0][1].numpy()[co] == w[32 * 9 * 2 + co]


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(2)
    w = rng.normal(0, 0.3, size=no.weight_count())
    L = rng.uniform(0, 255, size=(1, 6, 7))
    R = rng.uniform(0, 255, size=(1, 6, 7))
    label = rng.normal(0, 2, size=(1, 6, 7))
    label[0, 2, 3] = np.nan
    loss, g = no.loss_and_grad(L, R, label, w)
    idx = rng.choice(w.size, size=25, replace=False)
    idx = np.concatenate([idx, [w.size - 1, w.size - 2]])  # last bias and a last-layer weight
    h = 1e-6
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (no.loss_and_grad(L, R, label, wp)[0] - no.loss_and_grad(L, R, label, wm)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])


def test_loss_closed_form_with_constant_output():
    """All weights zero but the last bias b: the output is b everywhere, so the
    loss is mean(huber(b - label)) and d loss / d b = mean(huber'(b - label))."""
    w = np.zeros(no.weight_count())
    b = 0.7
    w[-1] = b
    label = np.array([[[0.0, 0.5, 3.0], [np.nan, -2.0, 0.7]]])
    L = np.zeros((1, 2, 3))
    loss, g = no.loss_and_grad(L, L, label, w)
    e = b - label[np.isfinite(label)]
    hub = np.where(np.abs(e) <= 1, 0.5 * e * e, np.abs(e) - 0.5)
    np.testing.assert_allclose(loss, hub.sum() / 6, rtol=1e-14)
    dh = np.where(np.abs(e) <= 1, e, np.sign(e))
    np.testing.assert_allclose(g[-1], dh.sum() / 6, rtol=1e-14)
