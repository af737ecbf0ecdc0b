"""The learned fast-forward's network on the GPU: ctypes binding of
``include/lbm_nn.h`` and a U-Net-style encoder-decoder assembled from those
kernels (forward, backward, Adam).

PyTorch only provides device memory here (tensors as buffers, zeroing);
every operation of the network runs in the library's kernels, and loading
fails loudly when the library is missing.

Network: 4 levels with channels ``ch`` (32, 64, 128, 256 by default); per
level two 3 x 3 convolutions with ReLU, 2 x 2 average pooling between
levels; on the way up nearest 2x upsampling, concatenation with the level's
encoder output, two 3 x 3 convolutions with ReLU; a 1 x 1 head whose first
three channels are added to the input's first three (phi, u, v): the network
predicts the change of the coarse fields over K solver steps.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import lbm as _lbm

LBM_NN_OK, LBM_NN_ERR_ARG, LBM_NN_ERR_CUDA = 0, -1, -2
NN_EXPORTS = ["lbm_nn_last_error", "lbm_nn_conv_fwd", "lbm_nn_set_conv_path", "lbm_nn_conv_status", "lbm_nn_conv_wgrad", "lbm_nn_flip_weights", "lbm_nn_relu_bwd",
              "lbm_nn_pool", "lbm_nn_pool_bwd", "lbm_nn_upsample", "lbm_nn_upsample_bwd", "lbm_nn_mse", "lbm_nn_adam",
              "lbm_nn_to_bf16", "lbm_nn_add", "lbm_nn_coarsen", "lbm_nn_refine", "lbm_nn_sharpen", "lbm_nn_mass_project",
              "lbm_nn_interface_stats", "lbm_nn_jet_length"]

_lib = None


class NNError(RuntimeError):
    pass


def load():
    global _lib
    if _lib is not None:
        return _lib
    lib = _lbm.load()
    vp, i32, i64, f32, fp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_void_p
    sig = {
        "lbm_nn_conv_fwd": [vp, i32, i32, i32, vp, fp, i32, vp, i32, i32, fp, i32, i32, i32, i32, i32, vp],
        "lbm_nn_conv_wgrad": [vp, i32, i32, i32, vp, i32, i32, fp, fp, i32, i32, i32, vp],
        "lbm_nn_set_conv_path": [i32],
        "lbm_nn_conv_status": [ctypes.POINTER(ctypes.c_int32)],
        "lbm_nn_flip_weights": [vp, i32, i32, i32, vp, vp],
        "lbm_nn_relu_bwd": [vp, i32, i32, vp, i32, i32, vp, i32, i32, i64, vp],
        "lbm_nn_pool": [vp, i32, i32, vp, i32, i32, i32, i32, i32, i32, vp],
        "lbm_nn_pool_bwd": [vp, i32, vp, i32, i32, i32, i32, i32, i32, vp],
        "lbm_nn_upsample": [vp, i32, vp, i32, i32, i32, i32, i32, i32, vp],
        "lbm_nn_upsample_bwd": [vp, i32, i32, vp, i32, i32, i32, i32, i32, vp],
        "lbm_nn_mse": [fp, i32, vp, i32, fp, i32, i64, fp, vp, i32, fp, vp],
        "lbm_nn_adam": [fp, fp, fp, fp, vp, i64, f32, f32, f32, f32, i32, vp],
        "lbm_nn_to_bf16": [fp, vp, i64, vp],
        "lbm_nn_add": [vp, i32, i32, vp, i32, i32, i32, i64, vp],
        "lbm_nn_coarsen": [fp, fp, fp, i32, i32, i32, f32, f32, vp, i32, fp, vp],
        "lbm_nn_refine": [fp, i32, i32, i32, f32, f32, fp, fp, fp, vp],
        "lbm_nn_sharpen": [fp, i64, ctypes.c_float, vp],
        "lbm_nn_mass_project": [fp, i64, ctypes.c_double, fp, vp],
        "lbm_nn_interface_stats": [fp, fp, i32, i32, fp, vp],
        "lbm_nn_jet_length": [fp, fp, i32, i32, i32, i32, fp, vp],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.lbm_nn_last_error.argtypes = []
    lib.lbm_nn_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def set_conv_path(path: int):
    """0: tcgen05 tensor-memory convolutions; 1: warp-level mma.sync; 2 (default):
    tcgen05 for calls of at least 4 GFLOP, else mma.sync."""
    lib = load()
    if lib.lbm_nn_set_conv_path(int(path)) != 0:
        raise NNError(lib.lbm_nn_last_error().decode())


def conv_timed_out() -> bool:
    """True if a bounded wait of the tcgen05 kernels gave up since the last call."""
    lib = load()
    t = ctypes.c_int32()
    if lib.lbm_nn_conv_status(ctypes.byref(t)) != 0:
        raise NNError(lib.lbm_nn_last_error().decode())
    return bool(t.value)


def _s(stream):
    return ctypes.c_void_p(0 if stream is None else int(stream.cuda_stream))


def call(name, *args):
    lib = load()
    code = getattr(lib, name)(*args)
    if code != LBM_NN_OK:
        raise NNError("%s failed (%d): %s" % (name, code, lib.lbm_nn_last_error().decode()))


def layer_shapes(cin, ch, head):
    """(name, ci, co, taps) of every convolution, in parameter order."""
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


class UNet:
    """Parameters (float32 master copy, bfloat16 copy, flipped bfloat16
    copy, Adam moments and gradients) live in flat device buffers with one
    view per layer; activations are allocated per batch shape."""

    def __init__(self, cin=8, ch=(32, 64, 128, 256), head=8, ncomp=3, device="cuda", stream=None):
        import torch
        assert cin % 8 == 0 and head % 8 == 0 and all(c % 8 == 0 for c in ch)
        self.torch = torch
        self.cin, self.ch, self.head, self.ncomp = cin, list(ch), head, ncomp
        self.L = len(ch)
        self.stream = stream
        self.layers = layer_shapes(cin, self.ch, head)
        nw = sum(co * taps * ci for _, ci, co, taps in self.layers)
        nb = sum(co for _, ci, co, taps in self.layers)
        n = nw + nb
        f32 = dict(dtype=torch.float32, device=device)
        self.w = torch.zeros(n, **f32)
        self.g = torch.zeros(n, **f32)
        self.m = torch.zeros(n, **f32)
        self.v = torch.zeros(n, **f32)
        self.wb = torch.zeros(n, dtype=torch.bfloat16, device=device)
        self.wf = torch.zeros(nw, dtype=torch.bfloat16, device=device)
        self.view = {}
        o = 0
        for name, ci, co, taps in self.layers:
            k = co * taps * ci
            self.view[name] = dict(ci=ci, co=co, taps=taps, w=self.w[o:o + k], g=self.g[o:o + k],
                                   wb=self.wb[o:o + k], wf=self.wf[o:o + k])
            o += k
        for name, ci, co, taps in self.layers:
            self.view[name].update(b=self.w[o:o + co], gb=self.g[o:o + co])
            o += co
        self.t = 0
        self._acts = {}

    # ------------------------------------------------------------ parameters
    def set_params(self, params: dict):
        """Load float64/float32 host arrays {name.w: [co, taps ci], name.b: [co]}."""
        torch = self.torch
        for name, *_ in self.layers:
            self.view[name]["w"].copy_(torch.from_numpy(np.ascontiguousarray(params[name + ".w"], np.float32).reshape(-1)))
            self.view[name]["b"].copy_(torch.from_numpy(np.ascontiguousarray(params[name + ".b"], np.float32)))
        self.sync_copies()

    def init_he(self, seed=0):
        """Seeded He-normal weights (std sqrt(2 / fan-in)), zero biases."""
        r = np.random.Generator(np.random.PCG64(seed))
        p = {}
        for name, ci, co, taps in self.layers:
            p[name + ".w"] = r.standard_normal((co, taps * ci)) * np.sqrt(2.0 / (taps * ci))
            p[name + ".b"] = np.zeros(co)
        self.set_params(p)

    def get_params(self) -> dict:
        out = {}
        for name, ci, co, taps in self.layers:
            out[name + ".w"] = self.view[name]["w"].cpu().numpy().reshape(co, taps * ci)
            out[name + ".b"] = self.view[name]["b"].cpu().numpy().copy()
        return out

    def get_grads(self) -> dict:
        out = {}
        for name, ci, co, taps in self.layers:
            out[name + ".w"] = self.view[name]["g"].cpu().numpy().reshape(co, taps * ci)
            out[name + ".b"] = self.view[name]["gb"].cpu().numpy().copy()
        return out

    def sync_copies(self):
        """bf16 weights from the f32 master copy and the flipped copies."""
        call("lbm_nn_to_bf16", _p(self.w), _p(self.wb), self.w.numel(), _s(self.stream))
        self._flip()

    def _flip(self):
        for name, ci, co, taps in self.layers:
            v = self.view[name]
            call("lbm_nn_flip_weights", _p(v["wb"]), ci, co, taps, _p(v["wf"]), _s(self.stream))

    # ------------------------------------------------------------ activations
    def _alloc(self, B, H, W):
        key = (B, H, W)
        if key in self._acts:
            return self._acts[key]
        torch = self.torch
        bf = dict(dtype=torch.bfloat16, device=self.w.device)
        A = {}
        for l in range(self.L):
            m = B * (H >> l) * (W >> l)
            c = self.ch[l]
            if l > 0:
                A["in%d" % l] = torch.zeros(m, self.ch[l - 1], **bf)
            A["ea%d" % l] = torch.zeros(m, c, **bf)
            A["skip%d" % l] = torch.zeros(m, c, **bf)
            A["dskip%d" % l] = torch.zeros(m, c, **bf)
            A["dz%d" % l] = torch.zeros(m, max(c, self.ch[min(l + 1, self.L - 1)] + c), **bf)
            A["dt%d" % l] = torch.zeros(m, max(c, self.ch[min(l + 1, self.L - 1)] + c), **bf)
            if l < self.L - 1:
                cc = self.ch[l + 1] + c
                A["dc%d" % l] = torch.zeros(m, cc, **bf)
                A["da%d" % l] = torch.zeros(m, c, **bf)
                A["dd%d" % l] = torch.zeros(m, c, **bf)
                A["ddc%d" % l] = torch.zeros(m, cc, **bf)
                A["gd%d" % l] = torch.zeros(m, c, **bf)
        m0 = B * H * W
        A["head"] = torch.zeros(m0, self.head, dtype=torch.float32, device=self.w.device)
        A["dhead"] = torch.zeros(m0, self.head, **bf)
        A["pred"] = torch.zeros(m0, self.ncomp, dtype=torch.float32, device=self.w.device)
        A["loss"] = torch.zeros(1, dtype=torch.float32, device=self.w.device)
        self._acts[key] = A
        return A

    def _conv(self, name, x, xs, y, ys, yo, relu, B, H, W, yf=None, yfs=0):
        v = self.view[name]
        call("lbm_nn_conv_fwd", _p(x), xs, v["ci"], v["taps"], _p(v["wb"]), _p(v["b"]), v["co"], _p(y), ys, yo,
             _p(yf), yfs, 1 if relu else 0, B, H, W, _s(self.stream))

    def _conv_bwd_data(self, name, dz, dzs, dx, dxs, dxo, B, H, W):
        v = self.view[name]
        call("lbm_nn_conv_fwd", _p(dz), dzs, v["co"], v["taps"], _p(v["wf"]), None, v["ci"], _p(dx), dxs, dxo,
             None, 0, 0, B, H, W, _s(self.stream))

    def _wgrad(self, name, x, xs, dz, dzs, B, H, W):
        v = self.view[name]
        call("lbm_nn_conv_wgrad", _p(x), xs, v["ci"], v["taps"], _p(dz), dzs, v["co"], _p(v["g"]), _p(v["gb"]),
             B, H, W, _s(self.stream))

    # ------------------------------------------------------------ passes
    def forward(self, x, B, H, W, target=None):
        """x: bf16 [B H W, cin] (channels last); returns the activations dict
        (pred f32 [B H W, ncomp], loss when a target f32 [B H W, ncomp] is given)."""
        A = self._alloc(B, H, W)
        L, ch = self.L, self.ch
        for l in range(L):
            Hl, Wl = H >> l, W >> l
            if l == 0:
                src, cs = x, self.cin
            else:
                call("lbm_nn_pool", _p(A["skip%d" % (l - 1)]), ch[l - 1], 0, _p(A["in%d" % l]), ch[l - 1], 0,
                     ch[l - 1], B, Hl * 2, Wl * 2, _s(self.stream))
                src, cs = A["in%d" % l], ch[l - 1]
            self._conv("enc%d_1" % l, src, cs, A["ea%d" % l], ch[l], 0, True, B, Hl, Wl)
            self._conv("enc%d_2" % l, A["ea%d" % l], ch[l], A["skip%d" % l], ch[l], 0, True, B, Hl, Wl)
        d, dc_ = A["skip%d" % (L - 1)], ch[L - 1]
        for l in range(L - 2, -1, -1):
            Hl, Wl = H >> l, W >> l
            cc = ch[l + 1] + ch[l]
            c = A["dc%d" % l]
            call("lbm_nn_upsample", _p(d), dc_, _p(c), cc, 0, ch[l + 1], B, Hl, Wl, _s(self.stream))
            self._copy_channels(A["skip%d" % l], ch[l], c, cc, ch[l + 1], ch[l], B * Hl * Wl)
            self._conv("dec%d_1" % l, c, cc, A["da%d" % l], ch[l], 0, True, B, Hl, Wl)
            self._conv("dec%d_2" % l, A["da%d" % l], ch[l], A["dd%d" % l], ch[l], 0, True, B, Hl, Wl)
            d, dc_ = A["dd%d" % l], ch[l]
        self._conv("head", A["dd0"], ch[0], None, 0, 0, False, B, H, W, yf=A["head"], yfs=self.head)
        m0 = B * H * W
        if target is not None:
            A["loss"].zero_()
        A["dhead"].zero_()
        call("lbm_nn_mse", _p(A["head"]), self.head, _p(x), self.cin, _p(target), self.ncomp, m0, _p(A["pred"]),
             _p(A["dhead"]) if target is not None else None, self.head,
             _p(A["loss"]) if target is not None else None, _s(self.stream))
        return A

    def _copy_channels(self, src, ss, dst, ds, do, c, m):
        # channel slice copy (through the add kernel onto a zeroed slice)
        dst.view(m, ds)[:, do:do + c].zero_()
        call("lbm_nn_add", _p(src), ss, 0, _p(dst), ds, do, c, m, _s(self.stream))

    def backward(self, x, B, H, W, zero_grad=True):
        """Gradients of the loss of the last forward with a target, added to
        the f32 gradient buffer (zeroed first unless zero_grad is False, which
        accumulates over several samples)."""
        A = self._alloc(B, H, W)
        L, ch = self.L, self.ch
        if zero_grad:
            self.g.zero_()
        s = _s(self.stream)
        # head (1 x 1, no activation): dhead is the gradient of its output
        self._wgrad("head", A["dd0"], ch[0], A["dhead"], self.head, B, H, W)
        g_d = A["gd0"]                                      # gradient wrt the decoder output of level 0
        self._conv_bwd_data("head", A["dhead"], self.head, g_d, ch[0], 0, B, H, W)
        for l in range(L - 1):
            Hl, Wl = H >> l, W >> l
            m = B * Hl * Wl
            cc = ch[l + 1] + ch[l]
            dz, dt = A["dz%d" % l], A["dt%d" % l]
            call("lbm_nn_relu_bwd", _p(g_d), ch[l], 0, _p(A["dd%d" % l]), ch[l], 0, _p(dz), ch[l], ch[l], m, s)
            self._wgrad("dec%d_2" % l, A["da%d" % l], ch[l], dz, ch[l], B, Hl, Wl)
            self._conv_bwd_data("dec%d_2" % l, dz, ch[l], dt, ch[l], 0, B, Hl, Wl)
            call("lbm_nn_relu_bwd", _p(dt), ch[l], 0, _p(A["da%d" % l]), ch[l], 0, _p(dz), ch[l], ch[l], m, s)
            self._wgrad("dec%d_1" % l, A["dc%d" % l], cc, dz, ch[l], B, Hl, Wl)
            ddc = A["ddc%d" % l]
            self._conv_bwd_data("dec%d_1" % l, dz, ch[l], ddc, cc, 0, B, Hl, Wl)
            # the skip half goes to the encoder's output gradient, the upsampled
            # half back through the upsampling to the level below's output
            self._slice_to(ddc, cc, ch[l + 1], A["dskip%d" % l], ch[l], ch[l], m)
            nxt = A["gd%d" % (l + 1)] if l + 1 < L - 1 else A["dskip%d" % (L - 1)]
            call("lbm_nn_upsample_bwd", _p(ddc), cc, 0, _p(nxt), ch[l + 1], ch[l + 1], B, Hl, Wl, s)
            g_d = nxt
        for l in range(L - 1, -1, -1):
            Hl, Wl = H >> l, W >> l
            m = B * Hl * Wl
            dz, dt = A["dz%d" % l], A["dt%d" % l]
            call("lbm_nn_relu_bwd", _p(A["dskip%d" % l]), ch[l], 0, _p(A["skip%d" % l]), ch[l], 0, _p(dz), ch[l],
                 ch[l], m, s)
            self._wgrad("enc%d_2" % l, A["ea%d" % l], ch[l], dz, ch[l], B, Hl, Wl)
            self._conv_bwd_data("enc%d_2" % l, dz, ch[l], dt, ch[l], 0, B, Hl, Wl)
            call("lbm_nn_relu_bwd", _p(dt), ch[l], 0, _p(A["ea%d" % l]), ch[l], 0, _p(dz), ch[l], ch[l], m, s)
            src, cs = (x, self.cin) if l == 0 else (A["in%d" % l], ch[l - 1])
            self._wgrad("enc%d_1" % l, src, cs, dz, ch[l], B, Hl, Wl)
            if l > 0:
                self._conv_bwd_data("enc%d_1" % l, dz, ch[l], dt, ch[l - 1], 0, B, Hl, Wl)
                call("lbm_nn_pool_bwd", _p(dt), ch[l - 1], _p(A["dskip%d" % (l - 1)]), ch[l - 1], 0, ch[l - 1], B,
                     Hl * 2, Wl * 2, s)

    def _slice_to(self, src, ss, so, dst, ds, c, m):
        dst.zero_()
        call("lbm_nn_add", _p(src), ss, so, _p(dst), ds, 0, c, m, _s(self.stream))

    def adam_step(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.t += 1
        call("lbm_nn_adam", _p(self.w), _p(self.m), _p(self.v), _p(self.g), _p(self.wb), self.w.numel(), lr, beta1,
             beta2, eps, self.t, _s(self.stream))
        self._flip()
