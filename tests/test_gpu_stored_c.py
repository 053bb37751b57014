"""GPU parity of the stored Gram-matrix supply (params.c_supply): the paper's
recurrent form of Table I, in which every iteration reads the column
C_{., uv} of Eq. 14 from a matrix stored per local measurement matrix, built
on the device in FP64 and stored FP32.  Checked against the FP64 oracle block
by block (traces and coefficient increments included) on the 8x8-LR tile's
144 local matrices, on the other sensor layouts and with the conjugate-pair
update; against the factored supply at full size; and the frugal choice,
which stores only the much-used table sets and runs the others factored in a
second kernel, block for block against both."""
import numpy as np
import pytest

import oracle
from paper_2205_02646_gb300 import synth
from parity import compare, mirror
from test_gpu_parity import TIE, TOL, check, gpu_run, oracle_run, rl  # noqa: F401  (rl: fixture)

pytestmark = pytest.mark.gpu

TABLE_C_BYTES = 1024 * 1024 * 8 + 8192 + 4096   # scaled columns, row scales, 1 / (s D)


def _every_block(g, hr, tr, nbw, max_tie_frac=0.03):
    res = compare(g["hr"], g["sel"], hr, tr["sel"], tr["gap"], np.arange(g["sel"].shape[0]), nbw, TOL, TIE,
                  gpu_dc=g["dc"], orc_dc=tr["dc"])
    check(res, max_tie_frac)
    assert np.isfinite(g["hr"]).all()
    return res


@pytest.mark.parametrize("index", [0, 1])
def test_stored_c_64x64_every_block(rl, index):
    f, mask, y = synth.workload("rljsde_64x64", index=index)
    g = gpu_run(rl, y, mask, c_supply=1)
    info = g["plan"].info()
    assert info["n_stored_c_tables"] == info["n_tables"]
    assert info["device_c_bytes"] == info["n_tables"] * TABLE_C_BYTES
    hr, tr = oracle_run(y, mask)
    res = _every_block(g, hr, tr, mask.shape[1] // 2)
    print("stored C 64x64 #%d: matched %d / %d, near-ties %d, max err %.3g"
          % (index, res["matched"], res["n"], res["near_ties"], res["max_err"]))


def test_stored_c_8x8_tile_every_table_type(rl):
    """All 144 local matrices of an 8x8-LR tile (16 interior phases, the
    clipped border and corner windows), each with its own stored C."""
    f = synth.image(256, 256, 128, 16, 3100)
    mask = synth.recurrent_mask(128, 128, 8, 10)
    y = synth.measure(f, mask).astype(np.float32)
    g = gpu_run(rl, y, mask, c_supply=1)
    info = g["plan"].info()
    assert info["n_tables"] == 144 and info["n_stored_c_tables"] == 144
    hr, tr = oracle.reconstruct(y.astype(np.float64), mask, oracle.Params(nu_max=100), recurrent=True, trace=True)
    res = _every_block(g, hr, tr, 64, max_tie_frac=0.01)
    print("stored C 8x8 tile: matched %d / %d, near-ties %d, max err %.3g"
          % (res["matched"], res["n"], res["near_ties"], res["max_err"]))


@pytest.mark.parametrize("name", ["quarter", "mixed"])
def test_stored_c_other_layouts(rl, name):
    f = synth.image(64, 96, 32, 4, 7300)
    mask = synth.aperture_mask(32, 48, 4, 7400, synth.APERTURE_SETS[name])
    y = synth.measure(f, mask, 1).astype(np.float32)
    g = gpu_run(rl, y, mask, nu_max=60, layout=1, c_supply=1)
    assert g["plan"].info()["n_stored_c_tables"] > 0
    hr, tr = oracle_run(y, mask, nu_max=60, layout=1)
    _every_block(g, hr, tr, mask.shape[1] // 2)


def test_stored_c_pairs(rl):
    f, mask, y = synth.workload("rljsde_64x64", index=1)
    g = gpu_run(rl, y, mask, pairs=1, c_supply=1)
    hr, tr = oracle_run(y, mask, pairs=1)
    _every_block(g, hr, tr, mask.shape[1] // 2)
    sel = g["sel"].astype(np.int64) & 0xFFFF
    assert np.all(sel <= mirror(sel))


def test_stored_c_agrees_with_factored_supply_at_full_size(rl):
    """The 1024x1024 workload through both supplies in one process: the
    selection sequences agree on all but near-tie blocks, which the oracle
    confirms on a sample that includes every departing block (up to 24)."""
    import torch
    f, mask, y = synth.workload("rljsde_1024x1024")
    lr_h, lr_w = mask.shape
    nbh, nbw = lr_h // 2, lr_w // 2
    nb, nu = nbh * nbw, 100
    lr = torch.from_numpy(y).cuda()
    runs = {}
    for supply in (0, 1, 2, 3):
        plan = rl.Plan(mask, rl.default_params(nu_max=nu, c_supply=supply))
        info = plan.info()
        assert info["n_stored_c_tables"] == {0: 100, 1: 100, 2: 0, 3: 4}[supply]
        assert info["n_launches"] == (2 if supply == 3 else 1)
        hr = torch.full((2 * lr_h, 2 * lr_w), float("nan"), device="cuda")
        sel = torch.zeros(nb * nu, dtype=torch.int16, device="cuda")
        dc = torch.zeros(nb * nu * 2, device="cuda")
        plan.reconstruct_trace(lr, hr, sel, dc)
        plan.check()
        d = dc.view(nb, nu, 2).cpu().numpy()
        runs[supply] = (hr.cpu().numpy(), sel.view(nb, nu).cpu().numpy(), d[..., 0] + 1j * d[..., 1])
        del plan
    # auto stores all 100 table sets here, as 1 does; 3 stores the 4 interior
    # ones (about 15,000 blocks each) and runs the border ones (at most 128
    # blocks each) factored: every block's output equals that of one of the
    # uniform supplies bit for bit
    hb = {s: runs[s][0].reshape(nbh, 4, nbw, 4) for s in runs}
    assert np.array_equal(hb[0], hb[1])
    eq1 = np.all(hb[3] == hb[1], axis=(1, 3))
    eq2 = np.all(hb[3] == hb[2], axis=(1, 3))
    assert np.all(eq1 | eq2)
    assert (eq1 & ~eq2).sum() > nb // 2 and (eq2 & ~eq1).sum() > 0
    same = np.all(runs[1][1] == runs[2][1], axis=1)
    print("stored vs factored: %d of %d blocks with identical selections" % (same.sum(), nb))
    assert same.mean() > 0.99
    # where the sequences agree the outputs differ by FP32 rounding only
    e = np.abs(runs[1][0].astype(np.float64) - runs[2][0]).reshape(nbh, 4, nbw, 4).max(axis=(1, 3)).ravel()
    assert e[same].max() < 1e-4
    rng = np.random.default_rng(5)
    differ = np.nonzero(~same)[0][:24]
    edge = [bi * nbw + bj for bi in (0, 1, nbh - 1) for bj in (0, 1, nbw - 1)]
    blocks = np.unique(np.concatenate([differ, edge, rng.choice(nb, 24, replace=False)])).astype(np.int64)
    hr, tr = oracle_run(y, mask, blocks=blocks)
    g_hr, g_sel, g_dc = runs[1]
    res = compare(g_hr, g_sel[blocks], hr, tr["sel"], tr["gap"], blocks, nbw, TOL, TIE,
                  gpu_dc=g_dc[blocks], orc_dc=tr["dc"])
    assert not res["fails"], res["fails"][:5]
    print("stored C 1024x1024 sample: matched %d / %d, near-ties %d" % (res["matched"], res["n"], res["near_ties"]))


def test_stored_c_refused_where_there_is_no_table_set(rl):
    """Stored C needs host table sets: a random (non-recurrent) mask, whose
    auto path builds tables in the kernel, and 15 apertures, which only the
    direct path holds, are refused; so are the FP64 loop and a frequency
    weight with a zero."""
    rnd = synth.random_mask(256, 256, 3)
    with pytest.raises(rl.RljsdeError) as e:
        rl.Plan(rnd, rl.default_params(c_supply=1))
    assert e.value.status == 8
    many = (np.arange(64 * 64, dtype=np.uint8).reshape(64, 64) % 15 + 1).astype(np.uint8)
    with pytest.raises(rl.RljsdeError) as e:
        rl.Plan(many, rl.default_params(c_supply=1, layout=1))
    assert e.value.status == 8
    f, mask, y = synth.workload("rljsde_64x64")
    with pytest.raises(rl.RljsdeError) as e:
        rl.Plan(mask, rl.default_params(c_supply=1, precision=1))
    assert e.value.status == 8
    # a frequency weight of 0 (the stored loop's state sqrt(q / D) R loses R
    # there): auto keeps the factored loop, stored is refused
    qz = np.ones(1024)
    qz[33] = 0.0
    assert rl.Plan(mask, rl.default_params(q_table=qz)).info()["n_stored_c_tables"] == 0
    with pytest.raises(rl.RljsdeError) as e:
        rl.Plan(mask, rl.default_params(q_table=qz, c_supply=1))
    assert e.value.status == 8
