"""Degenerate inputs and size extremes of the GPU path, against the FP64
oracle where it is cheap enough, else against properties that hold for any
size."""
import numpy as np
import pytest

from paper_2205_02646_gb300 import synth
from parity import compare
from test_gpu_parity import TIE, TOL, check, gpu_run, oracle_run, rl  # noqa: F401  (rl: fixture)

pytestmark = pytest.mark.gpu


def test_zero_image_gives_zero_and_dc_selections(rl):
    """y = 0: every score is 0, so the argmax takes index 0 (lowest index)
    with delta 0, on both sides, and the output is exactly 0."""
    mask = synth.recurrent_mask(16, 24, 4, 3)
    y = np.zeros(mask.shape, np.float32)
    g = gpu_run(rl, y, mask, nu_max=20)
    hr, tr = oracle_run(y, mask, nu_max=20)
    assert np.all(g["hr"] == 0.0) and np.all(hr == 0.0)
    assert np.all((g["sel"].astype(np.int64) & 0xFFFF) == 0) and np.all(tr["sel"] == 0)
    assert np.all(g["dc"] == 0.0)


@pytest.mark.parametrize("case", ["constant", "q_zero", "gamma_high", "rho_one"])
def test_degenerate_parameters_vs_oracle(rl, case):
    mask = synth.recurrent_mask(16, 24, 4, 5)
    f = synth.image(32, 48, 16, 2, 77)
    y = synth.measure(f, mask).astype(np.float32)
    kw, okw = {}, {}
    if case == "constant":
        y = np.full(mask.shape, 1.5, np.float32)          # a flat grey image: the DC atom explains it
    elif case == "q_zero":
        kw = okw = dict(q_table=np.zeros(1024))           # every score 0: the DC atom every time
        okw = dict(q_mode=2, q_table=np.zeros(1024))
    elif case == "gamma_high":
        kw = okw = dict(gamma_odc=1.9)
    else:
        kw = okw = dict(rho_decay=1.0)                    # unweighted window
    # a flat image is explained by the DC atom alone: with gamma 0.5 its residual
    # halves every iteration and reaches FP32 rounding after about 24, from
    # where the FP32 selections follow rounding noise (with no effect on the
    # output); compare the iterations before that
    nu = 20 if case == "constant" else 40
    g = gpu_run(rl, y, mask, nu_max=nu, **kw)
    hr, tr = oracle_run(y, mask, nu_max=nu, **okw)
    res = compare(g["hr"], g["sel"], hr, tr["sel"], tr["gap"], np.arange(g["sel"].shape[0]), mask.shape[1] // 2,
                  TOL, TIE, gpu_dc=g["dc"], orc_dc=tr["dc"])
    check(res)
    if case in ("q_zero", "constant"):
        assert np.all((g["sel"].astype(np.int64) & 0xFFFF) == 0)


def test_longest_loop_is_a_prefix_extension(rl):
    """nu_max = 4096 (the largest accepted): the first iterations are those of
    a short run (the loop does not depend on its length), and the output
    stays finite."""
    f, mask, y = synth.workload("rljsde_64x64")
    long = gpu_run(rl, y, mask, nu_max=4096)
    short = gpu_run(rl, y, mask, nu_max=64)
    assert np.array_equal(long["sel"][:, :64], short["sel"])
    assert np.array_equal(long["dc"][:, :64], short["dc"])
    assert np.isfinite(long["hr"]).all()
    with pytest.raises(rl.RljsdeError):
        rl.Plan(mask, rl.default_params(nu_max=4097))


def test_large_image_sampled_blocks(rl):
    """An 8192x8192 HR image (4,194,304 blocks) in one traced launch; the
    oracle recomputes corner, edge and random blocks one by one, and a block
    whose selections depart from the oracle's passes only at a near-tie of
    the oracle's scores at the first differing iteration."""
    import torch
    lr_h = lr_w = 4096
    nu = 60
    mask = synth.recurrent_mask(lr_h, lr_w, 4, 21)
    f = synth.image(2 * lr_h, 2 * lr_w, 64, 8, 4242)
    y = synth.measure(f, mask).astype(np.float32)
    nbh, nbw = lr_h // 2, lr_w // 2
    nb = nbh * nbw
    plan = rl.Plan(mask, rl.default_params(nu_max=nu))
    lr = torch.from_numpy(y).cuda()
    hr = torch.full((2 * lr_h, 2 * lr_w), float("nan"), device="cuda")
    sel = torch.zeros(nb * nu, dtype=torch.int16, device="cuda")
    dc = torch.zeros(nb * nu * 2, device="cuda")
    plan.reconstruct_trace(lr, hr, sel, dc)
    plan.check()
    assert bool(torch.isfinite(hr).all())
    rng = np.random.default_rng(5)
    corners = [0, nbw - 1, (nbh - 1) * nbw, nbh * nbw - 1, 3 * nbw + 2, (nbh - 2) * nbw + nbw - 3]
    blocks = np.unique(np.concatenate([corners, rng.choice(nb, 40, replace=False)])).astype(np.int64)
    bt = torch.from_numpy(blocks).cuda()
    gsel = sel.view(nb, nu)[bt].cpu().numpy()
    gdc = dc.view(nb, nu, 2)[bt].cpu().numpy()
    ohr, tr = oracle_run(y, mask, blocks=blocks, nu_max=nu)
    res = compare(hr.cpu().numpy(), gsel, ohr, tr["sel"], tr["gap"], blocks, nbw, TOL, TIE,
                  gpu_dc=gdc[..., 0] + 1j * gdc[..., 1], orc_dc=tr["dc"])
    check(res)
