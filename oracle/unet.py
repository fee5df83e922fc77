"""FP64 CPU reference of the learned preconditioner's network (TEST INFRASTRUCTURE ONLY).

Only the tests may import this module.  It restates, in plain numpy, the
network that the CUDA library trains and evaluates, so that the library's
forward pass and its gradients can be checked against an independent
implementation; the finite-difference tests pin this reference itself.

Network (L levels, C channels, inputs (sigma_t, sigma_s, b) scaled):
  encoder level l = 0 .. L-1 at resolution n / 2^l:
      a_l = relu(conv3(x_l)),  e_l = relu(conv3(a_l)),
      x_0 = input (3 channels), x_l = avgpool2(e_{l-1})
  decoder level l = L-2 .. 0:
      c_l = concat(upsample2(d_{l+1}), e_l)        (d_{L-1} = e_{L-1})
      b_l = relu(conv3(c_l)),  d_l = relu(conv3(b_l))
  output o = conv1(d_0)   (1 x 1 convolution to one channel, no relu)
conv3 is a 3 x 3 convolution with zero padding 1 and a bias; avgpool2 the
2 x 2 mean; upsample2 the nearest-neighbour copy.  Loss = mean((o - t)^2).

With bf16=True the forward pass is the one the BF16 inference kernels
compute: every weight, and the input of every 3 x 3 convolution, rounded to
the nearest BF16 value (ties to even) before an exact product; biases and
everything between the convolutions stay unrounded.

Parameters are a flat list [w, bias] per convolution in the order
E0.1, E0.2, E1.1, E1.2, ..., D(L-2).1, D(L-2).2, ..., D0.1, D0.2, head;
weights have shape [Cout, Cin, k, k].
"""
from __future__ import annotations

import numpy as np


def layer_shapes(levels: int, channels: int, cin: int = 3):
    shapes = []
    for l in range(levels):
        shapes.append((channels, cin if l == 0 else channels, 3))
        shapes.append((channels, channels, 3))
    for l in range(levels - 2, -1, -1):
        shapes.append((channels, 2 * channels, 3))
        shapes.append((channels, channels, 3))
    shapes.append((1, channels, 1))
    return shapes


def init_params(levels: int, channels: int, seed: int = 0):
    rng = np.random.default_rng(seed)
    params = []
    for co, ci, k in layer_shapes(levels, channels):
        std = np.sqrt(2.0 / (ci * k * k))
        params.append(rng.standard_normal((co, ci, k, k)) * std)
        params.append(np.zeros(co))
    return params


def round_bf16(x):
    """Nearest BF16 value of each FP32 value of x, ties to even: the high 16
    bits of the FP32 pattern after adding 0x7fff plus the lowest kept bit
    (finite values)."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def conv(x, w, b):
    """x [B, Ci, H, W], w [Co, Ci, k, k] (k = 1 or 3, zero padding k // 2)."""
    k = w.shape[2]
    p = k // 2
    B, Ci, H, W = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (p, p), (p, p)))
    out = np.zeros((B, w.shape[0], H, W))
    for dy in range(k):
        for dx in range(k):
            patch = xp[:, :, dy:dy + H, dx:dx + W]            # [B, Ci, H, W]
            out += np.einsum("bchw,oc->bohw", patch, w[:, :, dy, dx])
    return out + b[None, :, None, None]


def conv_backward(x, w, gout):
    """Gradients (dx, dw, db) of conv(x, w, b) given d out = gout."""
    k = w.shape[2]
    p = k // 2
    B, Ci, H, W = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (p, p), (p, p)))
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for dy in range(k):
        for dx in range(k):
            patch = xp[:, :, dy:dy + H, dx:dx + W]
            dw[:, :, dy, dx] = np.einsum("bohw,bchw->oc", gout, patch)
            dxp[:, :, dy:dy + H, dx:dx + W] += np.einsum("bohw,oc->bchw", gout, w[:, :, dy, dx])
    db = gout.sum(axis=(0, 2, 3))
    return dxp[:, :, p:p + H, p:p + W], dw, db


def avgpool2(x):
    B, C, H, W = x.shape
    return x.reshape(B, C, H // 2, 2, W // 2, 2).mean(axis=(3, 5))


def avgpool2_backward(g):
    return np.repeat(np.repeat(g, 2, axis=2), 2, axis=3) / 4.0


def upsample2(x):
    return np.repeat(np.repeat(x, 2, axis=2), 2, axis=3)


def upsample2_backward(g):
    B, C, H, W = g.shape
    return g.reshape(B, C, H // 2, 2, W // 2, 2).sum(axis=(3, 5))


def forward(params, x, levels: int, bf16: bool = False):
    """Returns (o, cache)."""
    if bf16:
        def conv(x, w, b):  # noqa: F811  (the BF16 inference arithmetic)
            if w.shape[2] == 3:
                x = round_bf16(x)
            return globals()["conv"](x, round_bf16(w), b)
    else:
        conv = globals()["conv"]
    cache = {"x": x}
    idx = 0
    xl = x
    enc = []
    for l in range(levels):
        w, b = params[2 * idx], params[2 * idx + 1]
        z1 = conv(xl, w, b)
        a = np.maximum(z1, 0)
        idx += 1
        w, b = params[2 * idx], params[2 * idx + 1]
        z2 = conv(a, w, b)
        e = np.maximum(z2, 0)
        idx += 1
        cache[("enc", l)] = (xl, z1, a, z2)
        enc.append(e)
        if l < levels - 1:
            xl = avgpool2(e)
    d = enc[-1]
    for l in range(levels - 2, -1, -1):
        c = np.concatenate([upsample2(d), enc[l]], axis=1)
        w, b = params[2 * idx], params[2 * idx + 1]
        z1 = conv(c, w, b)
        bb = np.maximum(z1, 0)
        idx += 1
        w, b = params[2 * idx], params[2 * idx + 1]
        z2 = conv(bb, w, b)
        d = np.maximum(z2, 0)
        idx += 1
        cache[("dec", l)] = (c, z1, bb, z2)
    w, b = params[2 * idx], params[2 * idx + 1]
    o = conv(d, w, b)
    cache["d0"] = d
    return o, cache


def loss_and_grads(params, x, t, levels: int):
    """Mean squared error and its gradients with respect to every parameter."""
    o, cache = forward(params, x, levels)
    diff = o - t
    loss = float(np.mean(diff ** 2))
    go = 2.0 * diff / diff.size
    grads = [None] * len(params)
    nconv = len(params) // 2
    gx, gw, gb = conv_backward(cache["d0"], params[2 * (nconv - 1)], go)
    grads[2 * (nconv - 1)], grads[2 * (nconv - 1) + 1] = gw, gb
    gd = gx
    idx = nconv - 1
    genc = [None] * levels
    C = params[0].shape[0]
    for l in range(0, levels - 1):
        c, z1, bb, z2 = cache[("dec", l)]
        idx -= 2
        gz2 = gd * (z2 > 0)
        gbb, gw, gb = conv_backward(bb, params[2 * (idx + 1)], gz2)
        grads[2 * (idx + 1)], grads[2 * (idx + 1) + 1] = gw, gb
        gz1 = gbb * (z1 > 0)
        gc, gw, gb = conv_backward(c, params[2 * idx], gz1)
        grads[2 * idx], grads[2 * idx + 1] = gw, gb
        genc[l] = gc[:, C:]
        gd = upsample2_backward(gc[:, :C])
    # gd is now the gradient of d_{L-1} = e_{L-1}
    genc[levels - 1] = gd
    gprev = None
    for l in range(levels - 1, -1, -1):
        xl, z1, a, z2 = cache[("enc", l)]
        ge = genc[l] if gprev is None else genc[l] + gprev
        gz2 = ge * (z2 > 0)
        ga, gw, gb = conv_backward(a, params[4 * l + 2], gz2)
        grads[4 * l + 2], grads[4 * l + 3] = gw, gb
        gz1 = ga * (z1 > 0)
        gx, gw, gb = conv_backward(xl, params[4 * l], gz1)
        grads[4 * l], grads[4 * l + 1] = gw, gb
        gprev = avgpool2_backward(gx) if l > 0 else None
    return loss, grads, o
