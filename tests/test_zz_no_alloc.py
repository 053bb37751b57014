"""rljsde_propose_noalloc: the proposal pass for callers that may not
allocate device memory (their device memory belongs to another allocator or
a budget fixed at start-up, or they must not allocate while streaming).  It
runs out of a fixed scratch array inside the library instead of a caller
workspace.  Checked here through the C ABI against rljsde_propose, on two
different images in a row, and for the size limit."""
import ctypes

import numpy as np
import pytest

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
    stream = torch.cuda.current_stream()
    for lr_h, lr_w, seed in ((40, 56, 1), (64, 48, 2)):
        mask, y = _image(lr_h, lr_w, seed)
        plan = rljsde.Plan(mask, rljsde.default_params(nu_max=20))
        lr = torch.from_numpy(y).cuda()
        ref = plan.propose(net, lr)
        got = torch.full_like(ref, 0xFF)
        assert fn(plan.handle, net.handle, lr.data_ptr(), lr.stride(0), got.data_ptr(),
                  ctypes.c_void_p(stream.cuda_stream)) == 0
        plan.check()
        nb = (lr_h // 2) * (lr_w // 2)
        ri, rm, rn = rljsde.shortlist_view(ref, nb)
        gi, gm, gn = rljsde.shortlist_view(got, nb)
        overlap = np.array([len(set(a.tolist()) & set(b.tolist())) for a, b in zip(ri, gi)])
        assert overlap.min() >= 56                        # tolerance of the whole-image shortlist test
        assert (overlap == 64).mean() >= 0.99
        np.testing.assert_allclose(gm, rm, rtol=1e-2, atol=1e-4)
        assert np.all(np.abs(gn - rn) < 0.05 * (1 + np.abs(rn)))
    # an image whose working set exceeds the fixed scratch is refused
    big = np.zeros((512, 512), np.uint8)
    plan = rljsde.Plan(big, rljsde.default_params(nu_max=1))
    lr = torch.zeros((512, 512), device="cuda")
    out = torch.zeros(256 * 256 * rljsde.SHORTLIST_BYTES, dtype=torch.uint8, device="cuda")
    assert fn(plan.handle, net.handle, lr.data_ptr(), 512, out.data_ptr(), ctypes.c_void_p(stream.cuda_stream)) == 2
