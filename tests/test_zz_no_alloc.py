"""rljsde_propose_noalloc: the proposal pass for callers that may not
allocate device memory (their device memory belongs to another allocator or
a budget fixed at start-up, or they must not allocate while streaming).  It
runs out of a fixed scratch array inside the library instead of a caller
workspace.  Checked here through the C ABI: it equals rljsde_propose byte for
byte on several images in a row (one near the size limit, whose tiles
several CTAs each walk in turn), its shortlists agree with the FP64
reference network, and an image over the limit is refused."""
import ctypes

import numpy as np
import pytest

from oracle import cnn_ref
from paper_2205_02646_gb300 import synth

pytestmark = pytest.mark.gpu


def _image(lr_h, lr_w, seed):
    f = synth.image(2 * lr_h, 2 * lr_w, 24, 3, 9700 + seed)
    mask = synth.recurrent_mask(lr_h, lr_w, 4, 40 + seed)
    return mask, synth.measure(f, mask).astype(np.float32)


def test_propose_noalloc_matches_propose_on_two_calls():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_02646_gb300 import build, rljsde
    build.build()
    lib = rljsde.load()
    fn = lib.rljsde_propose_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                   ctypes.c_void_p]
    net = rljsde.Net(seed=21)
    params = cnn_ref.unflatten(net.get_params())
    # head weights and biases spread like a trained network's, so the 64th
    # largest logit stands clear of its neighbours by more than the bfloat16
    # rounding of the whole-image activations moves it
    rng = np.random.default_rng(6)
    params["head.w"] = rng.normal(0.0, 0.05, params["head.w"].shape)
    params["head.b"] = rng.normal(-2.0, 1.5, params["head.b"].shape)
    net.set_params(cnn_ref.flatten(params).astype(np.float32))
    params = cnn_ref.unflatten(net.get_params())
    stream = torch.cuda.current_stream()
    # 584 x 584 L-pixels: 85,264 blocks, about 31.2 MiB of the 32 MiB scratch
    for lr_h, lr_w, seed in ((40, 56, 1), (584, 584, 3), (64, 48, 2)):
        mask, y = _image(lr_h, lr_w, seed)
        plan = rljsde.Plan(mask, rljsde.default_params(nu_max=20))
        lr = torch.from_numpy(y).cuda()
        ref = plan.propose(net, lr)
        got = torch.full_like(ref, 0xFF)
        assert fn(plan.handle, net.handle, lr.data_ptr(), lr.stride(0), got.data_ptr(),
                  ctypes.c_void_p(stream.cuda_stream)) == 0
        plan.check()
        assert torch.equal(got, ref)                      # the same kernels on the same inputs
        nbh, nbw = lr_h // 2, lr_w // 2
        gi, gm, gn = rljsde.shortlist_view(got, nbh * nbw)
        # against the FP64 reference network on a few blocks (corners, a middle one)
        for bi, bj in ((0, 0), (nbh - 1, nbw - 1), (0, nbw - 1), (nbh // 2, nbw // 2)):
            x, origin = cnn_ref.patch(y, mask, bi, bj)
            z, _ = cnn_ref.forward(params, x, origin, mask.shape)
            top = set(np.argsort(-z[:1024], kind="stable")[:64].tolist())
            b = bi * nbw + bj
            assert len(top & set(gi[b].tolist())) >= 56   # bfloat16 activations in the whole-image pass
            assert abs(gn[b] - z[1024]) < 0.05 * (1 + abs(z[1024]))
    # an image whose working set exceeds the fixed scratch is refused
    big = np.zeros((600, 600), np.uint8)
    plan = rljsde.Plan(big, rljsde.default_params(nu_max=1))
    lr = torch.zeros((600, 600), device="cuda")
    out = torch.zeros(300 * 300 * rljsde.SHORTLIST_BYTES, dtype=torch.uint8, device="cuda")
    assert fn(plan.handle, net.handle, lr.data_ptr(), 600, out.data_ptr(), ctypes.c_void_p(stream.cuda_stream)) == 2
