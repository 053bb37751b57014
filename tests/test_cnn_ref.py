"""Pins for the FP64 reference of the proposal network: its analytic
gradients against central finite differences, and the patch/full-image
equivalence its validity masks are meant to give."""
import numpy as np

from oracle import cnn_ref
from paper_2205_02646_gb300 import synth


def _setup(seed=0, n=2):
    rng = np.random.default_rng(seed)
    f = synth.image(48, 48, 16, 2, 77)
    mask = synth.recurrent_mask(24, 24, 4, 3)
    y = synth.measure(f, mask)
    params = {k: rng.normal(0, 0.3, s) for k, s in cnn_ref.SHAPES}
    blocks = [(0, 0), (5, 7), (11, 2)][:n]
    xs, origins = zip(*[cnn_ref.patch(y, mask, bi, bj) for bi, bj in blocks])
    targets = [(rng.random(1024) < 0.08).astype(float) for _ in blocks]
    nus = rng.random(len(blocks))
    masses = [rng.random(1024) * (rng.random(1024) < 0.1) for _ in blocks]
    return params, list(xs), list(origins), mask.shape, targets, nus, masses


def test_gradients_match_finite_differences():
    params, xs, origins, shape, targets, nus, masses = _setup()
    loss, g = cnn_ref.loss_and_grads(params, xs, origins, shape, targets, nus, masses, bf16=False)
    rng = np.random.default_rng(1)
    eps = 1e-6
    for name, shp in cnn_ref.SHAPES:
        for _ in range(6):
            idx = tuple(int(rng.integers(0, s)) for s in shp)
            if name.startswith("head") and _ == 0:
                idx = (1025,) + idx[1:]                      # the gate row
            p1 = {k: v.copy() for k, v in params.items()}
            p2 = {k: v.copy() for k, v in params.items()}
            p1[name][idx] += eps
            p2[name][idx] -= eps
            l1, _ = cnn_ref.loss_and_grads(p1, xs, origins, shape, targets, nus, masses, bf16=False)
            l2, _ = cnn_ref.loss_and_grads(p2, xs, origins, shape, targets, nus, masses, bf16=False)
            num = (l1 - l2) / (2 * eps)
            assert abs(num - g[name][idx]) <= 1e-6 + 1e-5 * abs(num), (name, idx, num, g[name][idx])


def test_patch_equals_full_image_pass():
    """The head features of a block computed on its patch equal those of one
    pass of the same layers over the whole (zero-padded) image."""
    params, xs, origins, shape, targets, nus, _ = _setup(n=3)
    rng = np.random.default_rng(2)
    f = synth.image(48, 48, 16, 2, 77)
    mask = synth.recurrent_mask(24, 24, 4, 3)
    y = synth.measure(f, mask)
    lr_h, lr_w = mask.shape
    x = np.zeros((5, lr_h, lr_w))
    x[0] = (y.astype(np.float32) / np.float32(3.0)).astype(np.float64)
    for c in range(4):
        x[1 + c] = mask == c
    p = {k: (cnn_ref.bf16_round(v) if k.endswith(".w") else v) for k, v in params.items()}
    a1 = np.maximum(cnn_ref._conv(x, p["conv1.w"], p["conv1.b"], 1), 0)
    a2 = np.maximum(cnn_ref._conv(a1, p["conv2.w"], p["conv2.b"], 2), 0)
    a3 = np.maximum(cnn_ref._conv(a2, p["conv3.w"], p["conv3.b"], 1), 0)
    a3p = np.zeros((32, a3.shape[1] + 2, a3.shape[2] + 2))
    a3p[:, 1:-1, 1:-1] = a3
    for bi, bj in [(0, 0), (5, 7), (11, 2), (11, 11), (3, 0)]:
        xp, o = cnn_ref.patch(y, mask, bi, bj)
        z, cache = cnn_ref.forward(params, xp, o, (lr_h, lr_w))
        f_patch = cache[-1]
        f_full = a3p[:, bi:bi + 3, bj:bj + 3].reshape(-1)
        np.testing.assert_allclose(f_patch, f_full, rtol=1e-12, atol=1e-12)
