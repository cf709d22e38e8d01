"""Pins for the oracle's warm-start CNN (four 3x3 convolutions, not in the paper):
closed-form networks and finite differences of every layer's weights and of the input."""
import numpy as np


def test_param_count(orc):
    assert orc.cnn_param_count() == 19105


def test_relu_identity_network(orc):
    # one channel passes its input through three centre taps: net(x) = relu(x)
    p = np.zeros(orc.cnn_param_count())
    for ws, bs, cin, cout in orc.cnn_layer_slices():
        w = np.zeros((cout, cin, 3, 3))
        w[0, 0, 1, 1] = 1.0
        p[ws] = w.ravel()
    x = np.random.default_rng(1).standard_normal((2, 7, 9))
    assert np.allclose(orc.cnn_forward(x, p), np.maximum(x, 0.0), atol=1e-15)


def test_shift_and_bias(orc):
    # a right-shift tap in the last layer, biases elsewhere, zero padding at the border
    p = np.zeros(orc.cnn_param_count())
    layers = orc.cnn_layer_slices()
    for l, (ws, bs, cin, cout) in enumerate(layers):
        w = np.zeros((cout, cin, 3, 3))
        w[0, 0, 1, 1 if l < 3 else 0] = 1.0  # last layer reads x - 1
        p[ws] = w.ravel()
    p[layers[3][1]] = 0.25
    x = np.abs(np.random.default_rng(2).standard_normal((5, 6))) + 0.1
    ref = np.full_like(x, 0.25)
    ref[:, 1:] += x[:, :-1]
    assert np.allclose(orc.cnn_forward(x, p), ref, atol=1e-14)


def test_gradients_match_finite_differences(orc):
    rng = np.random.default_rng(3)
    n = orc.cnn_param_count()
    p = np.zeros(n)
    for ws, bs, cin, cout in orc.cnn_layer_slices():
        p[ws] = rng.normal(0, np.sqrt(2.0 / (9 * cin)), ws.stop - ws.start)
        p[bs] = rng.normal(0, 0.05, bs.stop - bs.start)
    x = rng.standard_normal((2, 6, 7))
    gout = rng.standard_normal(x.shape)
    gp, gx = orc.cnn_backward(x, p, gout)
    L = lambda pp, xx: float(np.sum(gout * orc.cnn_forward(xx, pp)))
    h = 1e-6
    for ws, bs, cin, cout in orc.cnn_layer_slices():
        for idx in list(rng.integers(ws.start, ws.stop, 6)) + [bs.start, bs.stop - 1]:
            e = np.zeros(n)
            e[idx] = h
            fd = (L(p + e, x) - L(p - e, x)) / (2 * h)
            assert abs(gp[idx] - fd) <= 1e-6 * max(1.0, abs(fd)), idx
    for idx in [(0, 0, 0), (1, 3, 4), (0, 5, 6), (1, 2, 0)]:
        e = np.zeros_like(x)
        e[idx] = h
        fd = (L(p, x + e) - L(p, x - e)) / (2 * h)
        assert abs(gx[idx] - fd) <= 1e-6 * max(1.0, abs(fd)), idx
