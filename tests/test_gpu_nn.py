"""The learned fast-forward's kernels (include/lbm_nn.h) against the FP64
reference network (oracle/nn_oracle.py).

Inputs are rounded to bfloat16 on the host and the reference computes in
float64 on exactly those values, so the only differences are the kernels'
float32 accumulation (relative ~1e-6 per layer) and, where a kernel stores
bfloat16, that rounding (2^-9 relative per value).  Single kernels are held
to 1e-5 (float32 outputs) and 4e-3 (bfloat16 outputs).  Through the whole
network (19 layers, bfloat16 activations and gradients) the output agrees to
a few 1e-3; the gradients of the deepest layers agree to a few per cent,
because a pre-activation within the rounding of zero takes the other side of
its ReLU mask on the GPU: the bound is 1e-1 relative L2 per parameter tensor
with a cosine similarity of at least 0.99 (a missing or misrouted gradient
term shows up as errors of order one).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_12205_gb300 import build, nn
    build.build()
    nn.load()
    from oracle import nn_oracle
    return torch, nn, nn_oracle


def bf16_round(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)


def to_dev(torch, a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(dtype).cuda().contiguous()


def rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30)


@pytest.mark.parametrize("path", [0, 1])
@pytest.mark.parametrize("taps,ci,co,B,H,W", [(9, 8, 16, 2, 12, 20), (9, 32, 72, 2, 12, 20), (1, 32, 8, 2, 12, 20),
                                             (9, 16, 130, 2, 12, 20), (9, 128, 256, 1, 8, 24), (9, 64, 128, 3, 16, 16)])
def test_conv_forward_backward_and_weight_gradient(env, report, taps, ci, co, B, H, W, path):
    """Both contractions (path 0: tcgen05 with the accumulator in tensor
    memory; path 1: warp-level mma.sync).  480 positions are ragged against
    64- and 128-row tiles; 192 positions with K = 1152 and 256 channels take
    the split-K path; 130 channels leave a partial channel tile."""
    torch, nn, O = env
    nn.set_conv_path(path)
    r = np.random.Generator(np.random.PCG64(10 + taps + ci + co))
    x = bf16_round(r.standard_normal((B, H, W, ci)))
    wt = bf16_round(r.standard_normal((co, taps * ci)) / np.sqrt(taps * ci))
    bias = r.standard_normal(co).astype(np.float32).astype(np.float64)
    dz = bf16_round(r.standard_normal((B, H, W, co)))
    ref = O.conv(x, wt, bias, taps)
    rdx, rdw, rdb = O.conv_bwd(x, wt, taps, dz)
    xd, wd, dzd = to_dev(torch, x, torch.bfloat16), to_dev(torch, wt, torch.bfloat16), to_dev(torch, dz, torch.bfloat16)
    bd = to_dev(torch, bias, torch.float32)
    M = B * H * W
    y = torch.zeros(M, co + 8, dtype=torch.bfloat16, device="cuda")       # written at channel offset 8
    yf = torch.zeros(M, co, dtype=torch.float32, device="cuda")
    nn.call("lbm_nn_conv_fwd", nn._p(xd), ci, ci, taps, nn._p(wd), nn._p(bd), co, nn._p(y), co + 8, 8, nn._p(yf), co,
            0, B, H, W, None)
    wf = torch.zeros(ci * taps * co, dtype=torch.bfloat16, device="cuda")
    nn.call("lbm_nn_flip_weights", nn._p(wd), ci, co, taps, nn._p(wf), None)
    dx = torch.zeros(M, ci, dtype=torch.float32, device="cuda")
    if co % 8 == 0:
        nn.call("lbm_nn_conv_fwd", nn._p(dzd), co, co, taps, nn._p(wf), None, ci, None, 0, 0, nn._p(dx), ci, 0, B, H, W,
                None)
        dw = torch.zeros(co * taps * ci, dtype=torch.float32, device="cuda")
        db = torch.zeros(co, dtype=torch.float32, device="cuda")
        nn.call("lbm_nn_conv_wgrad", nn._p(xd), ci, ci, taps, nn._p(dzd), co, co, nn._p(dw), nn._p(db), B, H, W, None)
    torch.cuda.synchronize()
    e_yf = rel(yf.cpu().numpy(), ref.reshape(M, co))
    e_y = rel(y.float().cpu().numpy()[:, 8:], ref.reshape(M, co))
    assert e_yf < 1e-5
    assert e_y < 4e-3
    assert np.all(y.float().cpu().numpy()[:, :8] == 0)           # channels below the offset untouched
    vals = dict(fwd_f32=e_yf, fwd_bf16=e_y)
    if co % 8 == 0:
        e_dx = rel(dx.cpu().numpy(), rdx.reshape(M, ci))
        e_dw = rel(dw.cpu().numpy().reshape(co, taps * ci), rdw)
        e_db = rel(db.cpu().numpy(), rdb)
        vals.update(bwd_data=e_dx, wgrad=e_dw, bgrad=e_db)
        assert e_dx < 1e-5 and e_dw < 1e-5 and e_db < 1e-5
    report("nn_conv_t%d_ci%d_co%d_path%d" % (taps, ci, co, path), **vals)
    assert not nn.conv_timed_out()
    nn.set_conv_path(2)


def test_pool_upsample_relu_kernels(env):
    torch, nn, O = env
    r = np.random.Generator(np.random.PCG64(21))
    B, H, W, c = 2, 8, 12, 16
    x = bf16_round(r.standard_normal((B, H, W, c)))
    xd = to_dev(torch, x, torch.bfloat16)
    y = torch.zeros(B * H * W // 4, c, dtype=torch.bfloat16, device="cuda")
    nn.call("lbm_nn_pool", nn._p(xd), c, 0, nn._p(y), c, 0, c, B, H, W, None)
    up = torch.zeros(B * H * W, c, dtype=torch.bfloat16, device="cuda")
    nn.call("lbm_nn_upsample", nn._p(y), c, nn._p(up), c, 0, c, B, H, W, None)
    ub = torch.zeros(B * H * W // 4, c, dtype=torch.bfloat16, device="cuda")
    nn.call("lbm_nn_upsample_bwd", nn._p(xd), c, 0, nn._p(ub), c, c, B, H, W, None)
    pb = torch.zeros(B * H * W, c, dtype=torch.bfloat16, device="cuda")
    nn.call("lbm_nn_pool_bwd", nn._p(y), c, nn._p(pb), c, 0, c, B, H, W, None)
    dz = torch.zeros(B * H * W, c, dtype=torch.bfloat16, device="cuda")
    nn.call("lbm_nn_relu_bwd", nn._p(xd), c, 0, nn._p(xd), c, 0, nn._p(dz), c, c, B * H * W, None)
    torch.cuda.synchronize()
    yp = O.pool(x)
    assert rel(y.float().cpu().numpy(), yp.reshape(-1, c)) < 4e-3
    yq = y.float().cpu().numpy().reshape(B, H // 2, W // 2, c)
    assert np.array_equal(up.float().cpu().numpy(), O.up(yq).reshape(-1, c))
    assert rel(ub.float().cpu().numpy(), O.up_bwd(x).reshape(-1, c)) < 4e-3
    assert rel(pb.float().cpu().numpy(), O.pool_bwd(yq).reshape(-1, c)) < 4e-3
    assert np.array_equal(dz.float().cpu().numpy(), np.where(x > 0, x, 0).reshape(-1, c))


def test_network_loss_and_gradients_against_the_oracle(env, report):
    torch, nn, O = env
    ch, cin, head = [8, 16, 24, 32], 8, 8
    B, H, W = 2, 16, 32
    r = np.random.Generator(np.random.PCG64(31))
    p = O.init_params(cin, ch, head, seed=32)
    for k in list(p):
        p[k] = bf16_round(p[k]) if k.endswith(".w") else 0.05 * r.standard_normal(p[k].shape)
        p[k] = p[k].astype(np.float32).astype(np.float64)
    x = bf16_round(r.standard_normal((B, H, W, cin)))
    target = r.standard_normal((B, H, W, 3)).astype(np.float32).astype(np.float64)
    loss, g, pred = O.loss_and_grad(p, x, target, ch)
    net = nn.UNet(cin=cin, ch=ch, head=head)
    net.set_params(p)
    xd = to_dev(torch, x.reshape(-1, cin), torch.bfloat16)
    td = to_dev(torch, target.reshape(-1, 3), torch.float32)
    A = net.forward(xd, B, H, W, target=td)
    net.backward(xd, B, H, W)
    torch.cuda.synchronize()
    gl = float(A["loss"].item())
    e_pred = rel(A["pred"].cpu().numpy(), pred.reshape(-1, 3))
    gg = net.get_grads()
    worst, worst_cos = 0.0, 1.0
    for k in g:
        e = rel(gg[k], g[k])
        a, b = gg[k].reshape(-1).astype(np.float64), g[k].reshape(-1)
        cos = float(a @ b / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-30))
        worst, worst_cos = max(worst, e), min(worst_cos, cos)
        report("nn_grad_" + k, rel_l2=e, cos=cos)
    report("nn_network", loss_rel=abs(gl / loss - 1), pred_rel=e_pred, worst_grad=worst, worst_cos=worst_cos)
    assert abs(gl / loss - 1) < 1e-2
    assert e_pred < 1e-2
    assert worst < 1e-1 and worst_cos > 0.99


def test_adam_steps_reduce_the_loss(env):
    torch, nn, O = env
    ch, cin, head = [8, 16, 24, 32], 8, 8
    B, H, W = 2, 16, 32
    r = np.random.Generator(np.random.PCG64(41))
    net = nn.UNet(cin=cin, ch=ch, head=head)
    net.set_params(O.init_params(cin, ch, head, seed=42))
    x = r.standard_normal((B * H * W, cin)).astype(np.float32)
    xd = to_dev(torch, x, torch.bfloat16)
    td = to_dev(torch, x[:, :3] + 0.3 * np.sin(np.arange(B * H * W))[:, None], torch.float32)
    losses = []
    for _ in range(30):
        A = net.forward(xd, B, H, W, target=td)
        losses.append(float(A["loss"].item()))
        net.backward(xd, B, H, W)
        net.adam_step(lr=3e-3)
    assert losses[-1] < 0.5 * losses[0]


def test_training_step_is_reproducible(env):
    """Two identical training steps give bit-identical weights: the weight
    and bias gradients are reduced in a fixed order, not with atomics."""
    torch, nn, O = env
    ch, cin, head = [8, 16, 24, 32], 8, 8
    B, H, W = 2, 32, 64
    r = np.random.Generator(np.random.PCG64(51))
    x = r.standard_normal((B * H * W, cin)).astype(np.float32)
    xd = to_dev(torch, x, torch.bfloat16)
    td = to_dev(torch, np.sin(x[:, :3]), torch.float32)
    out = []
    for _ in range(2):
        net = nn.UNet(cin=cin, ch=ch, head=head)
        net.set_params(O.init_params(cin, ch, head, seed=52))
        for _ in range(3):
            net.forward(xd, B, H, W, target=td)
            net.backward(xd, B, H, W)
            net.adam_step(lr=1e-3)
        torch.cuda.synchronize()
        out.append(net.get_params())
    for k in out[0]:
        assert np.array_equal(out[0][k], out[1][k]), k
