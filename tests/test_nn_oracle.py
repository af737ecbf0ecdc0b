"""Pins of the FP64 reference network (oracle/nn_oracle.py) against things
other than itself: scipy's correlation for the convolution, adjoint
identities for pooling and upsampling, and central finite differences of the
loss for every layer's gradient."""
import numpy as np
import pytest

from oracle import nn_oracle as O


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def test_conv3x3_is_scipy_correlation_with_zero_padding():
    scipy_signal = pytest.importorskip("scipy.signal")
    r = rng(1)
    B, H, W, ci, co = 2, 7, 9, 3, 4
    x = r.standard_normal((B, H, W, ci))
    wt = r.standard_normal((co, 9 * ci))
    bias = r.standard_normal(co)
    y = O.conv(x, wt, bias, 9)
    for b in range(B):
        for o in range(co):
            ref = np.full((H, W), bias[o])
            for c in range(ci):
                k = np.array([[wt[o, (3 * ky + kx) * ci + c] for kx in range(3)] for ky in range(3)])
                ref += scipy_signal.correlate2d(x[b, :, :, c], k, mode="same", boundary="fill")
            assert np.allclose(y[b, :, :, o], ref, rtol=1e-12, atol=1e-12)


def test_conv1x1_is_a_channel_matrix_product():
    r = rng(2)
    x = r.standard_normal((1, 3, 5, 6))
    wt = r.standard_normal((4, 6))
    y = O.conv(x, wt, None, 1)
    assert np.allclose(y[0, 2, 3], wt @ x[0, 2, 3])


@pytest.mark.parametrize("taps", [9, 1])
def test_conv_backward_matches_finite_differences(taps):
    r = rng(3)
    x = r.standard_normal((2, 5, 6, 3))
    wt = r.standard_normal((4, taps * 3))
    bias = r.standard_normal(4)
    G = r.standard_normal((2, 5, 6, 4))
    f = lambda x_, w_, b_: float((O.conv(x_, w_, b_, taps) * G).sum())
    dx, dw, db = O.conv_bwd(x, wt, taps, G)
    h = 1e-6
    for idx in [(0, 0, 0, 0), (1, 4, 5, 2), (0, 2, 3, 1)]:
        e = np.zeros_like(x); e[idx] = h
        assert abs((f(x + e, wt, bias) - f(x - e, wt, bias)) / (2 * h) - dx[idx]) < 1e-6
    for idx in [(0, 0), (3, taps * 3 - 1), (2, taps * 3 // 2)]:
        e = np.zeros_like(wt); e[idx] = h
        assert abs((f(x, wt + e, bias) - f(x, wt - e, bias)) / (2 * h) - dw[idx]) < 1e-6
    e = np.zeros(4); e[1] = h
    assert abs((f(x, wt, bias + e) - f(x, wt, bias - e)) / (2 * h) - db[1]) < 1e-6


def test_pool_and_upsample_adjoints():
    r = rng(4)
    x = r.standard_normal((2, 8, 6, 3))
    y = r.standard_normal((2, 4, 3, 3))
    assert np.isclose((O.pool(x) * y).sum(), (x * O.pool_bwd(y)).sum())
    assert np.isclose((O.up(y) * x).sum(), (y * O.up_bwd(x)).sum())
    assert np.allclose(O.pool(O.up(y)), y)
    assert np.allclose(O.pool(np.full((1, 4, 4, 2), 3.5)), 3.5)


def test_network_gradient_matches_finite_differences():
    """Every layer's weight and bias gradient of the loss against central
    differences on a small network (4 levels, 8 x 16 input)."""
    r = rng(5)
    ch, cin, head = [4, 6, 8, 10], 5, 4
    p = O.init_params(cin, ch, head, seed=6)
    for k in p:
        if k.endswith(".b"):
            p[k] = 0.1 * r.standard_normal(p[k].shape)
    x = r.standard_normal((2, 8, 16, cin))
    target = r.standard_normal((2, 8, 16, 3))
    loss, g, pred = O.loss_and_grad(p, x, target, ch)
    assert np.isclose(loss, ((pred - target) ** 2).mean())
    h = 1e-6
    for name, ci, co, taps in O.layer_shapes(cin, ch, head):
        for key in (name + ".w", name + ".b"):
            flat = p[key].reshape(-1)
            for j in rng(sum(key.encode())).choice(flat.size, size=min(3, flat.size), replace=False):
                old = flat[j]
                flat[j] = old + h
                lp = O.loss_and_grad(p, x, target, ch)[0]
                flat[j] = old - h
                lm = O.loss_and_grad(p, x, target, ch)[0]
                flat[j] = old
                fd = (lp - lm) / (2 * h)
                an = g[key].reshape(-1)[j]
                assert abs(fd - an) <= 1e-6 + 1e-5 * abs(fd), (key, j, fd, an)
