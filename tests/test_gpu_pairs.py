"""GPU parity of the conjugate-pair update (params.pairs = 1, the frequency
selective variant of the loop) against the oracle's pairs mode, on every
path and layout that offers it."""
import numpy as np
import pytest

import oracle
from paper_2205_02646_gb300 import synth
from parity import compare, mirror
from test_gpu_parity import TIE, TOL, check, gpu_run, oracle_run, rl  # noqa: F401  (rl: fixture)

pytestmark = pytest.mark.gpu


def _parity(g, hr, tr, nbw, tol=TOL, tie=TIE, dc_tol=1e-3, max_tie_frac=0.03):
    res = compare(g["hr"], g["sel"], hr, tr["sel"], tr["gap"], np.arange(g["sel"].shape[0]), nbw, tol, tie,
                  gpu_dc=g["dc"], orc_dc=tr["dc"], dc_tol=dc_tol)
    check(res, max_tie_frac)
    sel = g["sel"].astype(np.int64) & 0xFFFF
    assert np.all(sel <= mirror(sel))                   # one member of each conjugate pair
    assert np.isfinite(g["hr"]).all()
    return res


@pytest.mark.parametrize("index", [0, 1])
def test_pairs_64x64_every_block(rl, index):
    f, mask, y = synth.workload("rljsde_64x64", index=index)
    g = gpu_run(rl, y, mask, pairs=1)
    hr, tr = oracle_run(y, mask, pairs=1)
    res = _parity(g, hr, tr, mask.shape[1] // 2)
    print("pairs 64x64 #%d: matched %d / %d, near-ties %d, max err %.3g"
          % (index, res["matched"], res["n"], res["near_ties"], res["max_err"]))


def test_pairs_fp64_loop(rl):
    f, mask, y = synth.workload("rljsde_64x64", index=2)
    g = gpu_run(rl, y, mask, nu_max=60, pairs=1, precision=1)
    hr, tr = oracle_run(y, mask, nu_max=60, pairs=1)
    _parity(g, hr, tr, mask.shape[1] // 2, tol=2e-7, tie=1e-9, dc_tol=1e-6, max_tie_frac=0.0)


def test_pairs_1024_sampled_blocks(rl):
    f, mask, y = synth.workload("rljsde_1024x1024")
    g = gpu_run(rl, y, mask, pairs=1)
    nbh, nbw = mask.shape[0] // 2, mask.shape[1] // 2
    rng = np.random.default_rng(1)
    edge = [bi * nbw + bj for bi in (0, 1, 2, 3, nbh - 1) for bj in (0, 1, 2, 3, nbw - 1)]
    blocks = np.unique(np.concatenate([edge, rng.choice(nbh * nbw, 64, replace=False)]))
    hr, tr = oracle_run(y, mask, blocks=blocks, pairs=1)
    res = compare(g["hr"], g["sel"][blocks], hr, tr["sel"], tr["gap"], blocks, nbw, TOL, TIE,
                  gpu_dc=g["dc"][blocks], orc_dc=tr["dc"])
    check(res)


@pytest.mark.parametrize("path", [2, 3])
def test_pairs_direct_and_in_kernel_tables(rl, path):
    f = synth.image(48, 64, 24, 3, 5100 + path)
    mask = synth.random_mask(24, 32, 40 + path)
    y = synth.measure(f, mask).astype(np.float32)
    g = gpu_run(rl, y, mask, nu_max=50, pairs=1, path=path)
    assert g["plan"].info()["path"] == path
    hr, tr = oracle_run(y, mask, nu_max=50, pairs=1)
    _parity(g, hr, tr, mask.shape[1] // 2)


@pytest.mark.parametrize("name", ["quarter", "mixed"])
def test_pairs_other_layouts(rl, name):
    f = synth.image(64, 96, 32, 4, 7300)
    mask = synth.aperture_mask(32, 48, 4, 7400, synth.APERTURE_SETS[name])
    y = synth.measure(f, mask, 1).astype(np.float32)
    g = gpu_run(rl, y, mask, nu_max=60, pairs=1, layout=1)
    hr, tr = oracle_run(y, mask, nu_max=60, pairs=1, layout=1)
    _parity(g, hr, tr, mask.shape[1] // 2)


def test_pairs_refused_by_learned_path(rl):
    import torch
    f, mask, y = synth.workload("rljsde_64x64")
    plan = rl.Plan(mask, rl.default_params(pairs=1))
    lr = torch.from_numpy(y).cuda()
    hr = torch.zeros((64, 64), device="cuda")
    sl = torch.zeros(plan.info()["n_blocks"] * rl.SHORTLIST_BYTES, dtype=torch.uint8, device="cuda")
    with pytest.raises(rl.RljsdeError) as e:
        plan.reconstruct_learned(lr, hr, sl, max_missing=1e9)
    assert e.value.status == 8
