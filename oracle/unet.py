"""FP64 reference of the learned warm start's convolutional denoiser.

Test infrastructure only (like the rest of ``oracle/``): the product path
never imports it.

The paper has no learned component; the denoiser is an extension that maps
a filtered back-projection of the data to a starting point for SPGL1 (the
solver of the paper's L1 problem, section "Introduction").  Its definition
is fixed here, and the device kernels implement the same function:

* U-Net with ``levels`` resolution levels and ``base`` channels at level 0
  (channels c_l = base * 2**l).  Images are single-channel, H and W
  divisible by 2**(levels-1).
* Encoder, level l = 0..L-1: h = relu(conv_b(relu(conv_a(x)))), with conv_a
  taking the level's input channels (1 at level 0, c_{l-1} above) to c_l and
  conv_b c_l -> c_l; skip_l = h; below the last level x = avgpool2x2(h).
* Decoder, level l = L-2..0: u = relu(conv_up(upsample2x_nearest(h))) with
  conv_up c_{l+1} -> c_l; h = relu(conv_b(relu(conv_a([skip_l, u])))) with
  conv_a 2 c_l -> c_l (skip channels first) and conv_b c_l -> c_l.
* Head: out = x_in + (1x1 conv c_0 -> 1)(h)  (the net predicts a correction
  of its input).
* All 3x3 convolutions are cross-correlations with zero padding 1 and a bias:
  y[co, p, q] = b[co] + sum_{ci, dy, dx} W[co, dy, dx, ci] x[ci, p+dy-1, q+dx-1].
* Loss: L = sum (out - target)^2 / (2 P) over the P = batch * H * W pixels.

Parameters are a dict name -> array; ``layer_specs`` lists the layers in a
fixed order with their shapes (W as (Cout, 3, 3, Cin), b as (Cout,)).

The backward pass is written out by hand (the adjoint of every step), and is
checked in the tests against central finite differences of the forward pass,
and the convolution against scipy's 2D correlation.

Operand rounding (``q``): the device rounds the operands of every 3x3
contraction to bfloat16 (the activations entering a convolution, the
masked output gradient entering the data and weight gradients, and the
weights) and accumulates in floating point.  ``forward`` / ``backward`` take
an optional rounding function q applied at exactly those points (the
caller rounds the weights); with q = None the network is computed exactly.
The ReLU masks are decisions taken on rounded values, so comparisons with
the device use q = bf16_round, to take them in the device's precision.
"""
from __future__ import annotations

import numpy as np


def channels(levels: int, base: int):
    return [base * (2 ** l) for l in range(levels)]


def layer_specs(levels: int, base: int):
    """[(name, cout, cin, k)] in the fixed parameter order."""
    c = channels(levels, base)
    specs = []
    for l in range(levels):
        cin = 1 if l == 0 else c[l - 1]
        specs.append((f"enc{l}.a", c[l], cin, 3))
        specs.append((f"enc{l}.b", c[l], c[l], 3))
    for l in range(levels - 2, -1, -1):
        specs.append((f"dec{l}.up", c[l], c[l + 1], 3))
        specs.append((f"dec{l}.a", c[l], 2 * c[l], 3))
        specs.append((f"dec{l}.b", c[l], c[l], 3))
    specs.append(("head", 1, c[0], 1))
    return specs


def init_params(levels: int, base: int, rng: np.random.Generator):
    """He-normal weights, zero biases (FP64)."""
    p = {}
    for name, co, ci, k in layer_specs(levels, base):
        std = np.sqrt(2.0 / (ci * k * k))
        p[name + ".W"] = rng.standard_normal((co, k, k, ci)) * std
        p[name + ".b"] = np.zeros(co)
    return p


# ---------------------------------------------------------------------------
# primitive ops (batch, channel, row, column) and their adjoints
# ---------------------------------------------------------------------------
def conv(x: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Cross-correlation with zero padding (k-1)/2: x (B, Ci, H, W) -> (B, Co, H, W)."""
    B, Ci, H, Wd = x.shape
    Co, k, _, _ = W.shape
    r = (k - 1) // 2
    xp = np.pad(x, ((0, 0), (0, 0), (r, r), (r, r)))
    y = np.zeros((B, Co, H, Wd))
    for dy in range(k):
        for dx in range(k):
            patch = xp[:, :, dy:dy + H, dx:dx + Wd]              # (B, Ci, H, W)
            # sum over ci of W[co, dy, dx, ci] patch[b, ci]  -> (Co, B, H, W)
            y += np.tensordot(W[:, dy, dx, :], patch, axes=([1], [1])).transpose(1, 0, 2, 3)
    return y + b[None, :, None, None]


def conv_backward(x: np.ndarray, W: np.ndarray, gy: np.ndarray):
    """Adjoint of conv in x and in (W, b): returns (gx, gW, gb)."""
    B, Ci, H, Wd = x.shape
    Co, k, _, _ = W.shape
    r = (k - 1) // 2
    xp = np.pad(x, ((0, 0), (0, 0), (r, r), (r, r)))
    gxp = np.zeros_like(xp)
    gW = np.zeros_like(W)
    for dy in range(k):
        for dx in range(k):
            patch = xp[:, :, dy:dy + H, dx:dx + Wd]
            # sum over b, p, q of gy[b, co] patch[b, ci]; sum over co of W[co, ci] gy[b, co]
            gW[:, dy, dx, :] = np.tensordot(gy, patch, axes=([0, 2, 3], [0, 2, 3]))
            gxp[:, :, dy:dy + H, dx:dx + Wd] += np.tensordot(W[:, dy, dx, :], gy, axes=([0], [1])).transpose(1, 0, 2, 3)
    gx = gxp[:, :, r:r + H, r:r + Wd]
    gb = gy.sum(axis=(0, 2, 3))
    return gx, gW, gb


def avgpool2(x):
    B, C, H, W = x.shape
    return x.reshape(B, C, H // 2, 2, W // 2, 2).mean(axis=(3, 5))


def avgpool2_backward(gy):
    return np.repeat(np.repeat(gy, 2, axis=2), 2, axis=3) / 4.0


def upsample2(x):
    return np.repeat(np.repeat(x, 2, axis=2), 2, axis=3)


def upsample2_backward(gy):
    B, C, H, W = gy.shape
    return gy.reshape(B, C, H // 2, 2, W // 2, 2).sum(axis=(3, 5))


def relu(x):
    return np.maximum(x, 0.0)


def bf16_round(a):
    """Round to the nearest bfloat16 value (ties to even), via float32."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


# ---------------------------------------------------------------------------
# network
# ---------------------------------------------------------------------------
def forward(params, x_in: np.ndarray, levels: int, base: int, q=None):
    """x_in (B, H, W) -> (out (B, H, W), tape for backward)."""
    tape = []
    x = x_in[:, None, :, :].astype(np.float64)
    qf = q if q is not None else (lambda a: a)

    def cr(name, inp):
        z = conv(qf(inp), params[name + ".W"], params[name + ".b"])
        y = relu(z)
        tape.append((name, inp, y))
        return y

    skips = []
    h = x
    for l in range(levels):
        h = cr(f"enc{l}.a", h)
        h = cr(f"enc{l}.b", h)
        skips.append(h)
        if l < levels - 1:
            h = avgpool2(h)
    for l in range(levels - 2, -1, -1):
        u = cr(f"dec{l}.up", upsample2(h))
        h = cr(f"dec{l}.a", np.concatenate([skips[l], u], axis=1))
        h = cr(f"dec{l}.b", h)
    head = conv(h, params["head.W"], params["head.b"])
    out = x[:, 0] + head[:, 0]
    return out, (tape, h)


def loss(out: np.ndarray, target: np.ndarray) -> float:
    return float(np.sum((out - target) ** 2) / (2.0 * out.size))


def backward(params, x_in: np.ndarray, target: np.ndarray, levels: int, base: int, q=None):
    """Loss and its gradient with respect to every parameter (dict) and to x_in."""
    out, (tape, h_last) = forward(params, x_in, levels, base, q)
    qf = q if q is not None else (lambda a: a)
    P = out.size
    g_out = (out - target) / P                                   # dL/d out
    grads = {}
    # head and residual
    gx_total = g_out.copy()
    gh, grads["head.W"], grads["head.b"] = conv_backward(h_last, params["head.W"], g_out[:, None])
    rec = {name: (inp, y) for name, inp, y in tape}

    def cr_back(name, gy):
        inp, y = rec[name]
        gz = gy * (y > 0)
        gi, grads[name + ".W"], _ = conv_backward(qf(inp), params[name + ".W"], qf(gz))
        grads[name + ".b"] = gz.sum(axis=(0, 2, 3))
        return gi

    c = channels(levels, base)
    g_skip = [None] * levels
    # decoder adjoint, level 0 upward: g is the gradient of decoder level l's
    # output; it leaves as the gradient of that level's input h, which is
    # decoder level l+1's output (or the bottom encoder output)
    g = gh
    for l in range(0, levels - 1):
        g = cr_back(f"dec{l}.b", g)
        gcat = cr_back(f"dec{l}.a", g)
        g_skip[l] = gcat[:, :c[l]]
        g = upsample2_backward(cr_back(f"dec{l}.up", gcat[:, c[l]:]))
    # g: gradient w.r.t. the output of the encoder's last level (bottom)
    for l in range(levels - 1, -1, -1):
        if l < levels - 1:
            g = avgpool2_backward(g) + g_skip[l]
        g = cr_back(f"enc{l}.b", g)
        g = cr_back(f"enc{l}.a", g)
    gx_total = gx_total + g[:, 0]
    return loss(out, target), grads, gx_total
