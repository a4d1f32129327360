"""Device denoiser (through the C ABI) against the FP64 oracle.

The device rounds convolution weights and the operands entering each
tensor-core contraction to BF16 and accumulates in FP32.  The oracle is given
the same BF16-rounded weights and runs with the same operand rounding, so
the ReLU masks -- decisions taken on rounded values -- are taken in the
device's precision on both sides.

Single operations (convolution, its data and weight gradients, pooling,
upsampling) then agree to FP32-against-FP64 accumulation: relative 1e-5.

A composed network does not: every rounding point turns a relative
difference e of its input into one-ulp flips of about e / 2^-8 of the
rounded values, so the difference grows like sqrt(e 2^-8) per layer towards
the bfloat16 resolution (measured on a two-level net: 3e-7 at the pooled
input, 9e-5 two convolutions later, 8e-4 at the output).  Bounds for whole
networks: relative 1e-2 for outputs, loss and the full gradient vector,
3e-2 for each parameter tensor.
"""
import numpy as np
import pytest

from oracle import unet

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_1380_gb300 import build
    build.build()
    return torch


def flat(params, levels, base):
    return np.concatenate([np.concatenate([params[n + ".W"].ravel(), params[n + ".b"].ravel()])
                           for n, *_ in unet.layer_specs(levels, base)])


def unflat(vec, levels, base):
    out, o = {}, 0
    for name, co, ci, k in unet.layer_specs(levels, base):
        nw = co * k * k * ci
        out[name + ".W"] = vec[o:o + nw].reshape(co, k, k, ci)
        out[name + ".b"] = vec[o + nw:o + nw + co]
        o += nw + co
    assert o == vec.size
    return out


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-30))


@pytest.mark.parametrize("levels,base,B,H,W", [(1, 64, 1, 12, 8), (1, 32, 2, 16, 16), (2, 64, 2, 16, 16),
                                               (2, 32, 3, 8, 24), (3, 32, 2, 16, 16)])
def test_unet_forward_backward_parity(torch_cuda, levels, base, B, H, W):
    torch = torch_cuda
    from paper_1009_1380_gb300 import cpct
    rng = np.random.default_rng(100 + levels)
    p = unet.init_params(levels, base, rng)
    for k in p:
        if k.endswith(".b"):
            p[k] = 0.05 * rng.standard_normal(p[k].shape)
    vec = flat(p, levels, base).astype(np.float32)
    # the oracle sees what the device computes with: BF16 3x3 weights, FP32 rest
    po = unflat(vec.astype(np.float64), levels, base)
    for name, co, ci, k in unet.layer_specs(levels, base):
        if k == 3:
            po[name + ".W"] = unet.bf16_round(po[name + ".W"])
    x = rng.standard_normal((B, H, W)).astype(np.float32)
    t = (x + 0.3 * rng.standard_normal((B, H, W))).astype(np.float32)
    net = cpct.UNet(levels, base, B, H, W)
    net.set_params(vec)
    assert np.array_equal(net.get_params(), vec)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    out = net.forward(xd).cpu().numpy()
    loss = net.backward(xd, td)
    g = net.get_grads()
    q = unet.bf16_round
    out_o, _ = unet.forward(po, x.astype(np.float64), levels, base, q)
    loss_o, grads_o, _ = unet.backward(po, x.astype(np.float64), t.astype(np.float64), levels, base, q)
    # compare the network's correction (out - x), the part the layers compute
    e_out = _rel(out - x, out_o - x)
    print("out", e_out, "loss", loss, loss_o)
    assert e_out < 1e-2
    assert abs(loss - loss_o) <= 1e-2 * loss_o
    gd = unflat(g.astype(np.float64), levels, base)
    assert _rel(g, flat(grads_o, levels, base)) < 1e-2
    worst = 0.0
    for name, *_ in unet.layer_specs(levels, base):
        for part in (".W", ".b"):
            e = _rel(gd[name + part], grads_o[name + part])
            worst = max(worst, e)
            assert e < 3e-2, (name + part, e)
    print("worst gradient rel", worst)


def test_unet_training_reduces_loss(torch_cuda):
    torch = torch_cuda
    from paper_1009_1380_gb300 import cpct
    rng = np.random.default_rng(7)
    levels, base, B, H, W = 3, 32, 4, 32, 32
    vec = flat(unet.init_params(levels, base, rng), levels, base).astype(np.float32)
    vec[-1] = 0.0
    net = cpct.UNet(levels, base, B, H, W)
    net.set_params(vec)
    t = rng.standard_normal((B, H, W)).astype(np.float32)
    x = (t + 0.5 * rng.standard_normal((B, H, W))).astype(np.float32)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    l0 = net.backward(xd, td)
    # the reported norm is the 2-norm of the gradients of the last backward
    g = net.get_grads()
    nrm = net.adam_step(1e-3, return_norm=True)
    assert abs(nrm - np.linalg.norm(g.astype(np.float64))) <= 1e-5 * nrm
    for _ in range(30):
        net.backward(xd, td)
        net.adam_step(1e-3, max_grad_norm=0.5 * nrm)
    l1 = net.backward(xd, td)
    print("loss", l0, "->", l1)
    assert l1 < 0.5 * l0


def _nhwc(a):
    return np.ascontiguousarray(np.transpose(a, (0, 2, 3, 1)))


def _nchw(a):
    return np.transpose(a, (0, 3, 1, 2))


@pytest.mark.parametrize("C1,C2,Cout,H,W", [(32, 0, 32, 9, 13), (64, 0, 128, 8, 8), (32, 32, 32, 16, 16),
                                            (64, 64, 64, 8, 8), (32, 0, 64, 16, 32)])
def test_conv_op_parity(torch_cuda, C1, C2, Cout, H, W):
    """One convolution (and its data gradient) against the oracle with the
    same bfloat16 operand rounding: FP32 against FP64 accumulation."""
    torch = torch_cuda
    from paper_1009_1380_gb300 import cpct
    rng = np.random.default_rng(C1 + 7 * C2 + Cout)
    B = 2
    a = rng.standard_normal((B, C1, H, W))
    b = rng.standard_normal((B, C2, H, W)) if C2 else None
    Wt = rng.standard_normal((Cout, 3, 3, C1 + C2)) * np.sqrt(2.0 / (9 * (C1 + C2)))
    bias = 0.1 * rng.standard_normal(Cout)
    hw = np.concatenate([Wt.ravel(), bias]).astype(np.float32)
    q = unet.bf16_round
    Wq = q(Wt.astype(np.float32))
    x = np.concatenate([a, b], axis=1) if C2 else a
    x32 = x.astype(np.float32)
    ad = torch.from_numpy(_nhwc(x32[:, :C1])).cuda()
    bd = torch.from_numpy(_nhwc(x32[:, C1:])).cuda() if C2 else None
    y = cpct.unet_debug_op(0, ad, bd, (B, H, W, Cout), w=hw, C1=C1, C2=C2, Cout=Cout).cpu().numpy()
    # the forward pass's kernel (BF16 input copies) computes the same values
    y7 = cpct.unet_debug_op(7, ad, bd, (B, H, W, Cout), w=hw, C1=C1, C2=C2, Cout=Cout).cpu().numpy()
    assert np.array_equal(y, y7)
    # ... and so does the tensor-memory kernel, up to FP32 accumulation order
    y8 = cpct.unet_debug_op(8, ad, bd, (B, H, W, Cout), w=hw, C1=C1, C2=C2, Cout=Cout).cpu().numpy()
    assert np.max(np.abs(y8 - y)) <= 1e-5 * np.max(np.abs(y))
    yo = unet.relu(unet.conv(q(x32.astype(np.float64)), Wq, bias.astype(np.float32).astype(np.float64)))
    e = _rel(_nchw(y), yo)
    print("conv", e)
    assert e < 1e-5
    # data gradient with the ReLU mask of the output
    gy = rng.standard_normal((B, Cout, H, W)).astype(np.float32)
    gd = cpct.unet_debug_op(5, torch.from_numpy(_nhwc(gy)).cuda(), torch.from_numpy(_nhwc(yo.astype(np.float32))).cuda(),
                            (B, H, W, C1 + C2), w=hw, C1=C1, C2=C2, Cout=Cout).cpu().numpy()
    gx, _, _ = unet.conv_backward(x32.astype(np.float64), Wq, q(gy.astype(np.float64) * (yo > 0)))
    e = _rel(_nchw(gd), gx)
    print("dgrad", e)
    assert e < 1e-5
    if C2 == 0:
        # the tensor-memory kernel on the BF16 copy of the masked gradient
        g11 = cpct.unet_debug_op(11, torch.from_numpy(_nhwc(gy)).cuda(),
                                 torch.from_numpy(_nhwc(yo.astype(np.float32))).cuda(), (B, H, W, C1), w=hw, C1=C1,
                                 C2=0, Cout=Cout).cpu().numpy()
        e = _rel(_nchw(g11), gx)
        print("dgrad tcgen05", e)
        assert e < 1e-5
        assert np.max(np.abs(g11 - gd)) <= 1e-5 * np.max(np.abs(gd))


@pytest.mark.parametrize("C1,C2,Cout,B,H,W", [
    (32, 0, 32, 3, 21, 19),      # 1197 pixels: 9 full M tiles and a ragged tail
    (32, 32, 64, 2, 16, 24),     # concatenated inputs
    (128, 0, 128, 1, 30, 17),    # 64-channel chunks
    (64, 64, 64, 2, 16, 33),     # 64-channel chunks from both inputs
    (256, 0, 256, 2, 12, 11),    # N tile of 256 tensor-memory columns
    (128, 128, 512, 1, 10, 13),  # two N tiles, 8 channel chunks per tap
    # images that tile into 128-pixel TMA boxes (Wb x Hb)
    (32, 0, 32, 2, 6, 128),      # 128 x 1
    (32, 32, 64, 1, 8, 256),     # two boxes per row, concatenated inputs
    (64, 64, 64, 2, 16, 64),     # 64 x 2, 64-channel chunks from both inputs
    (128, 0, 128, 1, 32, 32),    # 32 x 4
    (256, 0, 256, 2, 16, 16),    # 16 x 8
    (128, 128, 512, 1, 8, 16),   # two N tiles of 256
])
def test_conv_tc_parity(torch_cuda, C1, C2, Cout, B, H, W):
    """The tensor-memory (tcgen05) forward convolution against the oracle
    with the same bfloat16 operand rounding (FP32 against FP64 accumulation),
    at shapes spanning several 128-pixel tiles, a ragged tail and every N tile
    width; with the operand tiles loaded by TMA where the image tiles into
    128-pixel boxes (op 8) and by cp.async gathers (op 9)."""
    torch = torch_cuda
    from paper_1009_1380_gb300 import cpct
    rng = np.random.default_rng(1000 + C1 + 3 * C2 + Cout + H)
    a = rng.standard_normal((B, C1, H, W))
    b = rng.standard_normal((B, C2, H, W)) if C2 else None
    Wt = rng.standard_normal((Cout, 3, 3, C1 + C2)) * np.sqrt(2.0 / (9 * (C1 + C2)))
    bias = 0.1 * rng.standard_normal(Cout)
    hw = np.concatenate([Wt.ravel(), bias]).astype(np.float32)
    q = unet.bf16_round
    x32 = (np.concatenate([a, b], axis=1) if C2 else a).astype(np.float32)
    ad = torch.from_numpy(_nhwc(x32[:, :C1])).cuda()
    bd = torch.from_numpy(_nhwc(x32[:, C1:])).cuda() if C2 else None
    yo = unet.relu(unet.conv(q(x32.astype(np.float64)), q(Wt.astype(np.float32)),
                             bias.astype(np.float32).astype(np.float64)))
    tol = 1e-5 * np.max(np.abs(yo))
    for op in (8, 9):
        y = cpct.unet_debug_op(op, ad, bd, (B, H, W, Cout), w=hw, C1=C1, C2=C2, Cout=Cout).cpu().numpy()
        e = _rel(_nchw(y), yo)
        print("tcgen05 conv op", op, e)
        assert e < 1e-5
        # element-wise: FP32 accumulation of 9 (C1 + C2) products
        assert np.max(np.abs(_nchw(y) - yo)) <= tol


@pytest.mark.parametrize("Cout,B,H,W", [(32, 2, 9, 13), (64, 1, 32, 32), (8, 3, 5, 7)])
def test_first_conv_op_parity(torch_cuda, Cout, B, H, W):
    """The network's first layer (one input channel, direct kernel) against
    the oracle with the same bfloat16 operand rounding."""
    torch = torch_cuda
    from paper_1009_1380_gb300 import cpct
    rng = np.random.default_rng(500 + Cout + H)
    x = rng.standard_normal((B, H, W)).astype(np.float32)
    Wt = rng.standard_normal((Cout, 3, 3, 1)) * np.sqrt(2.0 / 9)
    bias = 0.1 * rng.standard_normal(Cout)
    hw = np.concatenate([Wt.ravel(), bias]).astype(np.float32)
    y = cpct.unet_debug_op(10, torch.from_numpy(x).cuda(), None, (B, H, W, Cout), w=hw, C1=1, C2=0,
                           Cout=Cout).cpu().numpy()
    q = unet.bf16_round
    yo = unet.relu(unet.conv(q(x.astype(np.float64))[:, None], q(Wt.astype(np.float32)),
                             bias.astype(np.float32).astype(np.float64)))
    assert np.max(np.abs(_nchw(y) - yo)) <= 1e-6 * np.max(np.abs(yo))


@pytest.mark.parametrize("C1,Cout,H,W", [(32, 32, 9, 13), (64, 128, 8, 8), (128, 64, 4, 4), (32, 64, 40, 24)])
def test_wgrad_op_parity(torch_cuda, C1, Cout, H, W):
    torch = torch_cuda
    from paper_1009_1380_gb300 import cpct
    rng = np.random.default_rng(C1 * 3 + Cout)
    B = 2
    x = rng.standard_normal((B, C1, H, W)).astype(np.float32)
    gy = rng.standard_normal((B, Cout, H, W)).astype(np.float32)
    y = cpct.unet_debug_op(6, torch.from_numpy(_nhwc(x)).cuda(), torch.from_numpy(_nhwc(gy)).cuda(),
                           (Cout * 9 * C1 + Cout,), C1=C1, Cout=Cout).cpu().numpy()
    q = unet.bf16_round
    W0 = np.zeros((Cout, 3, 3, C1))
    _, gW, gb = unet.conv_backward(q(x.astype(np.float64)), W0, q(gy.astype(np.float64)))
    gb = gy.astype(np.float64).sum(axis=(0, 2, 3))
    e_w = _rel(y[:Cout * 9 * C1], gW.ravel())
    e_b = _rel(y[Cout * 9 * C1:], gb)
    print("wgrad", e_w, "bias", e_b)
    assert e_w < 1e-5 and e_b < 1e-5
    # the kernel that reads BF16 copies of both operands (32 x 32 warp tiles)
    y12 = cpct.unet_debug_op(12, torch.from_numpy(_nhwc(x)).cuda(), torch.from_numpy(_nhwc(gy)).cuda(),
                             (Cout * 9 * C1 + Cout,), C1=C1, Cout=Cout).cpu().numpy()
    e_w = _rel(y12[:Cout * 9 * C1], gW.ravel())
    print("wgrad bf16", e_w)
    assert e_w < 1e-5
    assert np.array_equal(y12[Cout * 9 * C1:], y[Cout * 9 * C1:])


def test_pool_upsample_ops(torch_cuda):
    torch = torch_cuda
    from paper_1009_1380_gb300 import cpct
    rng = np.random.default_rng(21)
    B, C, H, W = 2, 32, 8, 12
    x = rng.standard_normal((B, C, H, W)).astype(np.float32)
    xs = rng.standard_normal((B, C, H // 2, W // 2)).astype(np.float32)
    dev = lambda t: torch.from_numpy(_nhwc(t)).cuda()
    y = cpct.unet_debug_op(1, dev(x), None, (B, H // 2, W // 2, C)).cpu().numpy()
    np.testing.assert_allclose(_nchw(y), unet.avgpool2(x.astype(np.float64)), rtol=1e-6, atol=1e-6)
    y = cpct.unet_debug_op(2, dev(xs), None, (B, H, W, C)).cpu().numpy()
    np.testing.assert_array_equal(_nchw(y), unet.upsample2(xs))
    y = cpct.unet_debug_op(3, dev(xs), dev(x), (B, H, W, C)).cpu().numpy()
    np.testing.assert_allclose(_nchw(y), unet.avgpool2_backward(xs.astype(np.float64)) + x, rtol=1e-6, atol=1e-6)
    y = cpct.unet_debug_op(4, dev(x), None, (B, H // 2, W // 2, C)).cpu().numpy()
    np.testing.assert_allclose(_nchw(y), unet.upsample2_backward(x.astype(np.float64)), rtol=1e-6, atol=1e-6)
