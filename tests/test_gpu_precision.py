"""GPU parity on the 8x8-LR mask tile (16 interior and 144 local masks in
all) and at the full 4096x3072 size: the FP32 loop and the all-FP64 loop
against the FP64 oracle, block by block, with every departure of the FP32
selection sequence traced back to a near-tie in the oracle's scores."""
import numpy as np
import pytest

from paper_2205_02646_gb300 import synth
from parity import compare
from test_gpu_parity import TIE, TOL, check, gpu_run, oracle_run, rl  # noqa: F401  (rl: fixture)

pytestmark = pytest.mark.gpu


def test_8x8_tile_every_table_type_vs_oracle(rl):
    """A 256x256 image behind an 8x8-LR tile holds every local mask such a
    tile can produce: 4 x 4 interior phases and, per axis, 4 top- and 4
    bottom-clipped window positions, (4 + 8)^2 = 144 in all.  Every one of
    its 4,096 blocks is compared with the oracle (recurrent FP64 form, pinned
    equal to the direct form), trace and coefficient increments included."""
    f = synth.image(256, 256, 128, 16, 3100)
    mask = synth.recurrent_mask(128, 128, 8, 10)
    y = synth.measure(f, mask).astype(np.float32)
    g = gpu_run(rl, y, mask)
    info = g["plan"].info()
    assert info["n_tables"] == 144 and info["n_interior_tables"] == 16
    import oracle
    hr, tr = oracle.reconstruct(y.astype(np.float64), mask, oracle.Params(nu_max=100), recurrent=True, trace=True)
    blocks = np.arange(64 * 64)
    res = compare(g["hr"], g["sel"], hr, tr["sel"], tr["gap"], blocks, 64, TOL, TIE,
                  gpu_dc=g["dc"], orc_dc=tr["dc"])
    check(res, max_tie_frac=0.01)
    assert np.isfinite(g["hr"]).all()
    print("8x8 tile: matched %d / %d, near-ties %d, max err %.3g"
          % (res["matched"], res["n"], res["near_ties"], res["max_err"]))


def test_full_size_departures_are_near_ties(rl):
    """The 4096x3072 workload with the 8x8-LR tile (786,432 blocks, one
    launch each for the FP32 and the FP64 loop, as the benchmark runs it).
    Sampled blocks -- every border and corner table type, random interior
    blocks, and up to 24 blocks where the FP32 and FP64 outputs differ by
    more than 1e-4 -- are recomputed by the oracle one by one: the FP64 loop
    matches every one of them, and each FP32 departure sits at a near-tie of
    the oracle's scores at the first differing iteration."""
    import torch
    f, mask, y = synth.workload("rljsde_4096x3072")
    lr_h, lr_w = mask.shape
    nbh, nbw = lr_h // 2, lr_w // 2
    nb, nu = nbh * nbw, 100
    lr = torch.from_numpy(y).cuda()
    runs = {}
    for name, prec in (("fp32", 0), ("fp64", 1)):
        plan = rl.Plan(mask, rl.default_params(nu_max=nu, precision=prec))
        hr = torch.full((2 * lr_h, 2 * lr_w), float("nan"), device="cuda")
        sel = torch.zeros(nb * nu, dtype=torch.int16, device="cuda")
        dc = torch.zeros(nb * nu * 2, device="cuda")
        plan.reconstruct_trace(lr, hr, sel, dc)
        plan.check()
        runs[name] = (hr, sel.view(nb, nu), dc.view(nb, nu, 2))
        plan.close()
    d = (runs["fp32"][0] - runs["fp64"][0]).abs().reshape(nbh, 4, nbw, 4).amax(dim=(1, 3)).flatten()
    assert bool(torch.isfinite(runs["fp32"][0]).all())
    departed = torch.nonzero(d > 1e-4).flatten().cpu().numpy()
    assert len(departed) <= 0.005 * nb                  # a small share of near-ties
    rng = np.random.default_rng(7)
    edge_rows = list(range(4)) + list(range(nbh - 4, nbh))
    edge_cols = list(range(4)) + list(range(nbw - 4, nbw))
    border = [bi * nbw + bj for bi in edge_rows for bj in range(4, 8)] + \
             [bi * nbw + bj for bi in range(4, 8) for bj in edge_cols] + \
             [bi * nbw + bj for bi in edge_rows for bj in edge_cols]
    picked = rng.choice(departed, min(24, len(departed)), replace=False) if len(departed) else []
    blocks = np.unique(np.concatenate([border, rng.choice(nb, 64, replace=False), picked]).astype(np.int64))
    ohr, tr = oracle_run(y, mask, blocks=blocks, nu_max=nu)
    bt = torch.from_numpy(blocks).cuda()
    for name, tol, tie in (("fp64", 2e-7, 1e-6), ("fp32", TOL, TIE)):
        hr, sel, dc = runs[name]
        ghr = hr.cpu().numpy()
        gsel = sel[bt].cpu().numpy()
        gdc = dc[bt].cpu().numpy()
        gdc = gdc[..., 0] + 1j * gdc[..., 1]
        res = compare(ghr, gsel, ohr, tr["sel"], tr["gap"], blocks, nbw, tol, tie, gpu_dc=gdc, orc_dc=tr["dc"])
        assert not res["fails"], (name, res["fails"][:5])
        if name == "fp64":
            assert res["near_ties"] == 0
        else:
            assert res["near_ties"] >= len(picked)      # every sampled departure is a near-tie
        print("%s: matched %d / %d, near-ties %d, max err %.3g, departed blocks %d of %d"
              % (name, res["matched"], res["n"], res["near_ties"], res["max_err"], len(departed), nb))
