"""FP64 CPU reference of the proposal network (test infrastructure).

The learned candidate proposal is this library's addition, not part of the
paper: a small fully convolutional network that scores, per 4x4 target block,
every one of the W^2 = 1024 DFT candidates of the greedy loop (Sec. IV) and
predicts how many iterations the block needs.  This module restates its
forward pass, loss and gradients in plain numpy FP64 so the CUDA kernels'
gradients can be checked against it; only the test suite uses it.

Network (one training sample = a 16x16 patch of L-pixels, LR rows/cols
[2bi - 8, 2bi + 8) x [2bj - 8, 2bj + 8) around target block (bi, bj)):

* input 5 x 16 x 16: y / 3 and the one-hot opaque-quadrant code (all zero
  where the patch leaves the image);
* conv1 5->32, 3x3, stride 1, pad 1, ReLU      (L-pixel grid)
* conv2 32->32, 3x3, stride 2, pad 1, ReLU     (target-block grid)
* conv3 32->32, 3x3, stride 1, pad 1, ReLU     (target-block grid)
* activations at positions outside the image are zero after every layer, which
  is what zero padding gives when the network runs over the whole image;
* head: the 3x3 block-grid neighbourhood of conv3 at the patch centre (block
  grid index (4, 4)), 288 features in the order c * 9 + (dy + 1) * 3 + (dx + 1),
  times W_h (1026 x 288) plus b_h: 1024 candidate logits, one iteration
  output and one gate;
* weights enter the forward pass rounded to bfloat16 (round to nearest even);
* loss, averaged over samples: mean over candidates of
  w(t) * (softplus(z) - t z), w = pos_weight for t = 1, else 1; plus
  nu_weight * (z_1024 - nu_target)^2; plus, given the sample's mass vector m
  (the plain loop's |gamma delta| per candidate), gate_weight *
  (sigmoid(z_1025) - s)^2 where s is the share of m outside the sample's
  own 64 largest candidate logits (a target: not differentiated).
"""
from __future__ import annotations

import numpy as np

C = 32
N_OUT = 1026
SHAPES = [("conv1.w", (C, 5, 3, 3)), ("conv1.b", (C,)), ("conv2.w", (C, C, 3, 3)), ("conv2.b", (C,)),
          ("conv3.w", (C, C, 3, 3)), ("conv3.b", (C,)), ("head.w", (N_OUT, 9 * C)), ("head.b", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unflatten(flat):
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    return out


def flatten(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def bf16_round(x):
    """Round float32 values to the nearest bfloat16 (ties to even), as float64."""
    x = np.asarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _conv(x, w, b, stride):
    """x: (C_in, H, W); cross-correlation with zero padding 1."""
    ci, H, Wd = x.shape
    co = w.shape[0]
    Ho, Wo = (H - 1) // stride + 1, (Wd - 1) // stride + 1
    xp = np.zeros((ci, H + 2, Wd + 2))
    xp[:, 1:-1, 1:-1] = x
    out = np.zeros((co, Ho, Wo))
    for dy in range(3):
        for dx in range(3):
            patch = xp[:, dy:dy + stride * (Ho - 1) + 1:stride, dx:dx + stride * (Wo - 1) + 1:stride]
            out += np.einsum("oc,chw->ohw", w[:, :, dy, dx], patch)
    return out + b[:, None, None]


def _conv_back(x, w, gout, stride):
    """Gradients of _conv w.r.t. x, w, b."""
    ci, H, Wd = x.shape
    _, Ho, Wo = gout.shape
    xp = np.zeros((ci, H + 2, Wd + 2))
    xp[:, 1:-1, 1:-1] = x
    gxp = np.zeros_like(xp)
    gw = np.zeros_like(w)
    for dy in range(3):
        for dx in range(3):
            sl = (slice(None), slice(dy, dy + stride * (Ho - 1) + 1, stride), slice(dx, dx + stride * (Wo - 1) + 1, stride))
            gw[:, :, dy, dx] = np.einsum("ohw,chw->oc", gout, xp[sl])
            gxp[sl] += np.einsum("oc,ohw->chw", w[:, :, dy, dx], gout)
    return gxp[:, 1:-1, 1:-1], gw, gout.sum(axis=(1, 2))


def valid_masks(origin, lr_shape):
    """Masks of positions inside the image for the L-pixel grid (16x16) and the
    block grid (8x8) of a patch whose (0, 0) is global L-pixel ``origin``."""
    y0, x0 = origin
    lr_h, lr_w = lr_shape
    yy, xx = np.meshgrid(np.arange(16) + y0, np.arange(16) + x0, indexing="ij")
    m1 = (yy >= 0) & (yy < lr_h) & (xx >= 0) & (xx < lr_w)
    by, bx = np.meshgrid(np.arange(8) + y0 // 2, np.arange(8) + x0 // 2, indexing="ij")
    m2 = (by >= 0) & (by < lr_h // 2) & (bx >= 0) & (bx < lr_w // 2)
    return m1.astype(np.float64), m2.astype(np.float64)


def forward(params, x, origin, lr_shape, bf16=True):
    """One sample: returns (z (1025,), cache).  ``bf16=False`` keeps the
    weights in FP64 (used to pin the gradients by finite differences)."""
    p = {k: (bf16_round(v) if (bf16 and k.endswith(".w")) else np.asarray(v, np.float64))
         for k, v in params.items()}
    m1, m2 = valid_masks(origin, lr_shape)
    a1 = np.maximum(_conv(x, p["conv1.w"], p["conv1.b"], 1), 0) * m1
    a2 = np.maximum(_conv(a1, p["conv2.w"], p["conv2.b"], 2), 0) * m2
    a3 = np.maximum(_conv(a2, p["conv3.w"], p["conv3.b"], 1), 0) * m2
    f = a3[:, 3:6, 3:6].reshape(-1)            # c * 9 + (dy+1) * 3 + (dx+1)
    z = p["head.w"] @ f + p["head.b"]
    return z, (p, x, m1, m2, a1, a2, a3, f)


def loss_and_grads(params, xs, origins, lr_shape, targets, nu_targets, masses=None, pos_weight=8.0,
                   nu_weight=0.1, gate_weight=1.0, bf16=True):
    """Mean loss over samples and its gradient w.r.t. every parameter (with
    respect to the bf16-rounded weights, as the GPU computes it)."""
    n = len(xs)
    grads = {k: np.zeros_like(np.asarray(v, np.float64)) for k, v in params.items()}
    total = 0.0
    for i, (x, o, t, nt) in enumerate(zip(xs, origins, targets, nu_targets)):
        z, (p, x, m1, m2, a1, a2, a3, f) = forward(params, x, o, lr_shape, bf16)
        zc, t = z[:1024], np.asarray(t, np.float64)
        w = np.where(t > 0.5, pos_weight, 1.0)
        sp = np.logaddexp(0.0, zc)
        total += np.mean(w * (sp - t * zc)) + nu_weight * (z[1024] - nt) ** 2
        gz = np.zeros(N_OUT)
        gz[:1024] = w * (1.0 / (1.0 + np.exp(-zc)) - t) / 1024.0
        gz[1024] = 2.0 * nu_weight * (z[1024] - nt)
        if masses is not None:
            m = np.asarray(masses[i], np.float64)
            inside = zc >= np.sort(zc)[-64]                    # the 64 largest (ties count as in)
            share = m[~inside].sum() / m.sum() if m.sum() > 0 else 0.0
            sg = 1.0 / (1.0 + np.exp(-z[1025]))
            total += gate_weight * (sg - share) ** 2
            gz[1025] = 2.0 * gate_weight * (sg - share) * sg * (1.0 - sg)
        gz /= n
        grads["head.w"] += np.outer(gz, f)
        grads["head.b"] += gz
        gf = p["head.w"].T @ gz
        g3 = np.zeros_like(a3)
        g3[:, 3:6, 3:6] = gf.reshape(C, 3, 3)
        g3 = g3 * (a3 > 0)
        g2, gw, gb = _conv_back(a2, p["conv3.w"], g3, 1)
        grads["conv3.w"] += gw
        grads["conv3.b"] += gb
        g2 = g2 * (a2 > 0)
        g1, gw, gb = _conv_back(a1, p["conv2.w"], g2, 2)
        grads["conv2.w"] += gw
        grads["conv2.b"] += gb
        g1 = g1 * (a1 > 0)
        _, gw, gb = _conv_back(x, p["conv1.w"], g1, 1)
        grads["conv1.w"] += gw
        grads["conv1.b"] += gb
    return total / n, grads


def patch(y, mask, bi, bj):
    """Input tensor (5, 16, 16) and origin of block (bi, bj)'s patch."""
    lr_h, lr_w = mask.shape
    y0, x0 = 2 * bi - 8, 2 * bj - 8
    x = np.zeros((5, 16, 16))
    for a in range(16):
        for b in range(16):
            P, Q = y0 + a, x0 + b
            if 0 <= P < lr_h and 0 <= Q < lr_w:
                x[0, a, b] = float(np.float32(y[P, Q]) / np.float32(3.0))
                x[1 + int(mask[P, Q]), a, b] = 1.0
    return x, (y0, x0)
