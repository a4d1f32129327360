"""Pins of the FP64 denoiser oracle against things other than itself.

* the 3x3 convolution equals scipy's 2D cross-correlation (zero fill) summed
  over input channels, plus the bias;
* average pooling and nearest upsampling: exact adjoint pairs with the
  hand-written backward steps, and the mean / replication on constants;
* the hand-written backward pass equals central finite differences of the
  forward pass (relative 1e-6) for every parameter tensor and the input;
* the residual form: with a zero head the network is the identity;
* the bfloat16 operand rounding equals torch's CPU float32 -> bfloat16
  conversion (round to nearest even), and leaves representable operands
  unchanged.
"""
import numpy as np
import pytest
from scipy import signal

from oracle import unet


def test_conv_matches_scipy_correlate():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, 3, 9, 11))
    W = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = unet.conv(x, W, b)
    for bb in range(2):
        for co in range(4):
            ref = b[co] + sum(signal.correlate2d(x[bb, ci], W[co, :, :, ci], mode="same", boundary="fill")
                              for ci in range(3))
            np.testing.assert_allclose(y[bb, co], ref, rtol=1e-12, atol=1e-12)
    # 1x1 convolution is a per-pixel matrix product
    W1 = rng.standard_normal((2, 1, 1, 3))
    y1 = unet.conv(x, W1, np.zeros(2))
    np.testing.assert_allclose(y1, np.einsum("oc,bchw->bohw", W1[:, 0, 0], x), rtol=1e-12)


def test_pool_upsample_adjoint_pairs():
    rng = np.random.default_rng(4)
    x = rng.standard_normal((2, 3, 8, 6))
    y = rng.standard_normal((2, 3, 4, 3))
    assert np.isclose(np.sum(unet.avgpool2(x) * y), np.sum(x * unet.avgpool2_backward(y)), rtol=1e-13)
    assert np.isclose(np.sum(unet.upsample2(y) * x), np.sum(y * unet.upsample2_backward(x)), rtol=1e-13)
    c = np.full((1, 1, 4, 4), 2.5)
    assert np.allclose(unet.avgpool2(c), 2.5) and np.allclose(unet.upsample2(c[:, :, :2, :2]), 2.5)
    z = np.arange(16.0).reshape(1, 1, 4, 4)
    assert unet.avgpool2(z)[0, 0, 0, 0] == (0 + 1 + 4 + 5) / 4


def test_zero_head_is_identity():
    rng = np.random.default_rng(5)
    p = unet.init_params(3, 2, rng)
    p["head.W"][:] = 0.0
    x = rng.standard_normal((2, 8, 8))
    out, _ = unet.forward(p, x, 3, 2)
    np.testing.assert_array_equal(out, x)


def _flat(params, levels, base):
    return np.concatenate([np.concatenate([params[n + ".W"].ravel(), params[n + ".b"]])
                           for n, *_ in unet.layer_specs(levels, base)])


@pytest.mark.parametrize("levels,base", [(1, 3), (3, 2)])
def test_backward_matches_finite_differences(levels, base):
    rng = np.random.default_rng(6 + levels)
    p = unet.init_params(levels, base, rng)
    for k in p:
        if k.endswith(".b"):
            p[k] = 0.1 * rng.standard_normal(p[k].shape)
    x = rng.standard_normal((2, 8, 8))
    t = rng.standard_normal((2, 8, 8))
    L0, grads, gx = unet.backward(p, x, t, levels, base)

    def L(pp, xx):
        out, _ = unet.forward(pp, xx, levels, base)
        return unet.loss(out, t)

    h = 1e-6
    for name, co, ci, k in unet.layer_specs(levels, base):
        for part in (".W", ".b"):
            key = name + part
            arr = p[key]
            flat_idx = rng.choice(arr.size, size=min(arr.size, 12), replace=False)
            fd = np.empty(len(flat_idx))
            for i, fi in enumerate(flat_idx):
                orig = arr.flat[fi]
                arr.flat[fi] = orig + h
                lp = L(p, x)
                arr.flat[fi] = orig - h
                lm = L(p, x)
                arr.flat[fi] = orig
                fd[i] = (lp - lm) / (2 * h)
            an = grads[key].ravel()[flat_idx]
            err = np.linalg.norm(an - fd) / max(np.linalg.norm(fd), 1e-12)
            assert err < 1e-6, (key, err)
    # input gradient
    idx = rng.choice(x.size, size=16, replace=False)
    fd = []
    for fi in idx:
        xp, xm = x.copy(), x.copy()
        xp.flat[fi] += h
        xm.flat[fi] -= h
        fd.append((L(p, xp) - L(p, xm)) / (2 * h))
    fd = np.array(fd)
    assert np.linalg.norm(gx.ravel()[idx] - fd) / np.linalg.norm(fd) < 1e-6


def test_planted_mistake_is_caught():
    """A dropped ReLU mask in the backward pass (planted in a copy of the
    oracle's step) fails the finite-difference comparison."""
    rng = np.random.default_rng(9)
    x = rng.standard_normal((1, 3, 6, 6))
    W = rng.standard_normal((2, 3, 3, 3))
    b = rng.standard_normal(2)
    gy = rng.standard_normal((1, 2, 6, 6))

    def f(xx):
        return np.sum(unet.relu(unet.conv(xx, W, b)) * gy)

    z = unet.conv(x, W, b)
    good, _, _ = unet.conv_backward(x, W, gy * (z > 0))
    bad, _, _ = unet.conv_backward(x, W, gy)
    h = 1e-6
    fd = np.empty(x.size)
    for i in range(x.size):
        xp, xm = x.copy(), x.copy()
        xp.flat[i] += h
        xm.flat[i] -= h
        fd[i] = (f(xp) - f(xm)) / (2 * h)
    assert np.linalg.norm(good.ravel() - fd) / np.linalg.norm(fd) < 1e-6
    assert np.linalg.norm(bad.ravel() - fd) / np.linalg.norm(fd) > 1e-2


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(11)
    a = np.concatenate([rng.standard_normal(10000) * 10.0 ** rng.integers(-20, 20, 10000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.01171875, -3.5e-40, 65504.0]]).astype(np.float32)
    ref = torch.from_numpy(a).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(unet.bf16_round(a), ref)


def test_rounded_mode_is_the_exact_mode_on_representable_values():
    """With operands already bfloat16-representable and a one-level net, the
    rounded forward equals the exact forward on its first contraction."""
    rng = np.random.default_rng(12)
    p = unet.init_params(1, 2, rng)
    for k in p:
        p[k] = unet.bf16_round(p[k])
    x = unet.bf16_round(rng.standard_normal((1, 6, 6)))
    z_exact = unet.conv(x[:, None], p["enc0.a.W"], p["enc0.a.b"])
    out_q, (tape, _) = unet.forward(p, x, 1, 2, q=unet.bf16_round)
    np.testing.assert_array_equal(tape[0][2], unet.relu(z_exact))
