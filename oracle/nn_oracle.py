"""FP64 reference of the learned fast-forward's network (test infrastructure).

Only tests, the smoke check and the benchmark's CPU baseline use this module;
the CUDA path shares no code with it.  Plain numpy in float64, written from
the definitions:

  * convolution (3 x 3, zero padding 1, or 1 x 1), channels last:
        y[b, i, j, o] = bias[o] + sum_{ky, kx, c} w[o, (3 ky + kx) ci + c] x[b, i + ky - 1, j + kx - 1, c];
  * ReLU, 2 x 2 average pooling, nearest 2x upsampling, channel concatenation;
  * the encoder-decoder: per level two 3 x 3 convolutions with ReLU, pooling
    between levels, on the way up nearest upsampling, concatenation with the
    level's encoder output and two 3 x 3 convolutions with ReLU, then a 1 x 1
    head; the prediction is the input's first three channels plus the head's
    first three;
  * the loss: mean squared error of the prediction over positions and those
    three channels.

The backward pass is written out layer by layer (the adjoint of each
operation); tests pin it to central finite differences of the loss and the
convolution to scipy's correlate.
"""
from __future__ import annotations

import numpy as np


def conv(x, wt, bias, taps):
    """x [B, H, W, ci], wt [co, taps * ci], bias [co] -> [B, H, W, co] (float64)."""
    B, H, W, ci = x.shape
    co = wt.shape[0]
    y = np.zeros((B, H, W, co))
    if taps == 1:
        y += np.einsum("bhwc,oc->bhwo", x, wt)
    else:
        xp = np.zeros((B, H + 2, W + 2, ci))
        xp[:, 1:-1, 1:-1] = x
        for ky in range(3):
            for kx in range(3):
                tap = 3 * ky + kx
                y += np.einsum("bhwc,oc->bhwo", xp[:, ky:ky + H, kx:kx + W], wt[:, tap * ci:(tap + 1) * ci])
    if bias is not None:
        y += bias
    return y


def conv_bwd(x, wt, taps, dz):
    """Adjoint of conv at x: (dx, dwt, dbias) for the output gradient dz."""
    B, H, W, ci = x.shape
    dbias = dz.sum(axis=(0, 1, 2))
    if taps == 1:
        return np.einsum("bhwo,oc->bhwc", dz, wt), np.einsum("bhwo,bhwc->oc", dz, x), dbias
    xp = np.zeros((B, H + 2, W + 2, ci))
    xp[:, 1:-1, 1:-1] = x
    dxp = np.zeros_like(xp)
    dwt = np.zeros_like(wt, dtype=np.float64)
    for ky in range(3):
        for kx in range(3):
            tap = 3 * ky + kx
            wk = wt[:, tap * ci:(tap + 1) * ci]
            dxp[:, ky:ky + H, kx:kx + W] += np.einsum("bhwo,oc->bhwc", dz, wk)
            dwt[:, tap * ci:(tap + 1) * ci] = np.einsum("bhwo,bhwc->oc", dz, xp[:, ky:ky + H, kx:kx + W])
    return dxp[:, 1:-1, 1:-1], dwt, dbias


def pool(x):
    B, H, W, C = x.shape
    return x.reshape(B, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def pool_bwd(dy):
    return np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2) / 4.0


def up(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up_bwd(dy):
    B, H, W, C = dy.shape
    return dy.reshape(B, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


def layer_shapes(cin, ch, head):
    """(name, ci, co, taps) of every convolution of the network with input
    channels cin, level channels ch (4 levels) and head channels head."""
    L = len(ch)
    out = []
    for l in range(L):
        out.append(("enc%d_1" % l, cin if l == 0 else ch[l - 1], ch[l], 9))
        out.append(("enc%d_2" % l, ch[l], ch[l], 9))
    for l in range(L - 2, -1, -1):
        out.append(("dec%d_1" % l, ch[l + 1] + ch[l], ch[l], 9))
        out.append(("dec%d_2" % l, ch[l], ch[l], 9))
    out.append(("head", ch[0], head, 1))
    return out


def init_params(cin, ch, head, seed=0):
    """Seeded He-normal weights, zero biases (float64)."""
    r = np.random.Generator(np.random.PCG64(seed))
    p = {}
    for name, ci, co, taps in layer_shapes(cin, ch, head):
        p[name + ".w"] = r.standard_normal((co, taps * ci)) * np.sqrt(2.0 / (taps * ci))
        p[name + ".b"] = np.zeros(co)
    return p


def forward(p, x, ch, ncomp=3):
    """Head output d [B, H, W, head] and the cache of activations."""
    L = len(ch)
    relu = lambda a: np.maximum(a, 0.0)
    cache = {"x": x}
    h = x
    for l in range(L):
        if l > 0:
            h = pool(cache["skip%d" % (l - 1)])
            cache["in%d" % l] = h
        a = relu(conv(h, p["enc%d_1.w" % l], p["enc%d_1.b" % l], 9))
        s = relu(conv(a, p["enc%d_2.w" % l], p["enc%d_2.b" % l], 9))
        cache["ea%d" % l], cache["skip%d" % l] = a, s
    d = cache["skip%d" % (L - 1)]
    for l in range(L - 2, -1, -1):
        c = np.concatenate([up(d), cache["skip%d" % l]], axis=3)
        a = relu(conv(c, p["dec%d_1.w" % l], p["dec%d_1.b" % l], 9))
        d = relu(conv(a, p["dec%d_2.w" % l], p["dec%d_2.b" % l], 9))
        cache["dc%d" % l], cache["da%d" % l], cache["dd%d" % l] = c, a, d
    out = conv(d, p["head.w"], p["head.b"], 1)
    return out, cache


def loss_and_grad(p, x, target, ch, ncomp=3):
    """MSE of pred = x[..., :ncomp] + d[..., :ncomp] against target, and the
    gradient of the loss with respect to every parameter."""
    L = len(ch)
    d, cache = forward(p, x, ch, ncomp)
    pred = x[..., :ncomp] + d[..., :ncomp]
    r = pred - target
    n = r.size
    loss = float((r * r).sum() / n)
    g = {}
    dd = np.zeros_like(d)
    dd[..., :ncomp] = 2.0 * r / n
    dh, g["head.w"], g["head.b"] = conv_bwd(cache["dd0"], p["head.w"], 1, dd)
    dskip = {}
    cur = dh                                            # gradient wrt d of the current decoder level
    for l in range(L - 1):
        dz2 = cur * (cache["dd%d" % l] > 0)
        da, g["dec%d_2.w" % l], g["dec%d_2.b" % l] = conv_bwd(cache["da%d" % l], p["dec%d_2.w" % l], 9, dz2)
        dz1 = da * (cache["da%d" % l] > 0)
        dc, g["dec%d_1.w" % l], g["dec%d_1.b" % l] = conv_bwd(cache["dc%d" % l], p["dec%d_1.w" % l], 9, dz1)
        cu = ch[l + 1]
        dskip[l] = dc[..., cu:]
        cur = up_bwd(dc[..., :cu])                      # gradient wrt d of level l + 1
    dskip[L - 1] = cur
    for l in range(L - 1, -1, -1):
        dz2 = dskip[l] * (cache["skip%d" % l] > 0)
        da, g["enc%d_2.w" % l], g["enc%d_2.b" % l] = conv_bwd(cache["ea%d" % l], p["enc%d_2.w" % l], 9, dz2)
        dz1 = da * (cache["ea%d" % l] > 0)
        h = cache["x"] if l == 0 else cache["in%d" % l]
        dx, g["enc%d_1.w" % l], g["enc%d_1.b" % l] = conv_bwd(h, p["enc%d_1.w" % l], 9, dz1)
        if l > 0:
            dskip[l - 1] = dskip[l - 1] + pool_bwd(dx)
    return loss, g, pred
