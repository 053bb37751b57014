"""GPU parity for sensor layouts other than three-quarter sampling (Sec. I:
any periodically repeating layout).  Mask codes are apertures, the set of
transparent sub-pixels of each L-pixel; the CUDA library is compared with
the FP64 oracle block by block, as for three-quarter sampling."""
import numpy as np
import pytest

from paper_2205_02646_gb300 import synth
from parity import compare
from test_gpu_parity import TIE, TOL, check, gpu_run, oracle_run, rl  # noqa: F401  (rl: fixture)

pytestmark = pytest.mark.gpu

APERTURE = 1


def layout_case(name, lr=(32, 48), tile=4, seed=0):
    lr_h, lr_w = lr
    f = synth.image(2 * lr_h, 2 * lr_w, 32, 4, 7000 + seed)
    mask = synth.aperture_mask(lr_h, lr_w, tile, 7100 + seed, synth.APERTURE_SETS[name])
    return mask, synth.measure(f, mask, APERTURE).astype(np.float32)


def test_three_quarter_apertures_match_opaque_codes_bitwise(rl):
    f, mask, y = synth.workload("rljsde_64x64", index=6)
    a = gpu_run(rl, y, mask, nu_max=60)
    b = gpu_run(rl, y, synth.apertures_of(mask), nu_max=60, layout=APERTURE)
    assert np.array_equal(a["sel"], b["sel"])
    assert np.array_equal(a["hr"], b["hr"])
    assert b["plan"].info()["n_apertures"] == 4


@pytest.mark.parametrize("name,seed", [("quarter", 1), ("pairs", 2), ("mixed", 3)])
def test_recurrent_layouts_vs_oracle(rl, name, seed):
    mask, y = layout_case(name, seed=seed)
    g = gpu_run(rl, y, mask, nu_max=60, layout=APERTURE)
    info = g["plan"].info()
    assert info["path"] == 1 and info["n_apertures"] == len(synth.APERTURE_SETS[name])
    hr, tr = oracle_run(y, mask, nu_max=60, layout=APERTURE)
    res = compare(g["hr"], g["sel"], hr, tr["sel"], tr["gap"], np.arange(g["sel"].shape[0]),
                  mask.shape[1] // 2, TOL, TIE, gpu_dc=g["dc"], orc_dc=tr["dc"])
    check(res)
    print("%s: matched %d / %d, near-ties %d, max err %.3g"
          % (name, res["matched"], res["n"], res["near_ties"], res["max_err"]))


@pytest.mark.parametrize("name", ["mixed", "symmetric", "quarter"])
def test_layout_fp64_loop_vs_oracle(rl, name):
    """FP64 loop: the same selections as the oracle, including the exact
    ties of the transpose-symmetric layout (both sides compare binary32
    keys and keep the lowest index)."""
    mask, y = layout_case(name, seed=4)
    g = gpu_run(rl, y, mask, nu_max=60, layout=APERTURE, precision=1)
    hr, tr = oracle_run(y, mask, nu_max=60, layout=APERTURE)
    res = compare(g["hr"], g["sel"], hr, tr["sel"], tr["gap"], np.arange(g["sel"].shape[0]),
                  mask.shape[1] // 2, 2e-7, 1e-9, gpu_dc=g["dc"], orc_dc=tr["dc"], dc_tol=1e-6)
    check(res, max_tie_frac=0.0)


def test_many_apertures_take_the_direct_path(rl):
    mask, y = layout_case("all", lr=(24, 32), seed=5)
    g = gpu_run(rl, y, mask, nu_max=40, layout=APERTURE)
    info = g["plan"].info()
    assert info["path"] == 2 and info["n_apertures"] == len(set(np.unique(mask)) - {0}) > 4
    hr, tr = oracle_run(y, mask, nu_max=40, layout=APERTURE)
    res = compare(g["hr"], g["sel"], hr, tr["sel"], tr["gap"], np.arange(g["sel"].shape[0]),
                  mask.shape[1] // 2, TOL, TIE, gpu_dc=g["dc"], orc_dc=tr["dc"])
    check(res)
    with pytest.raises(rl.RljsdeError) as e:
        rl.Plan(mask, rl.default_params(layout=APERTURE, path=1))
    assert e.value.status == 8                              # RLJSDE_ERR_UNSUPPORTED


@pytest.mark.parametrize("path", [1, 2])
def test_full_aperture_sensor_properties(rl, path):
    """A regular LR sensor (every aperture full): candidates in the Nyquist
    row / column are seen by no measurement and never chosen; the four
    aliases of each frequency tie exactly, so which one wins is rounding's
    choice, but with w = q = gamma = 1 and 256 iterations every alias class
    is taken once and the block's 2x2 box sums reproduce the measurements."""
    rng = np.random.default_rng(8)
    y = rng.uniform(0.0, 4.0, (24, 24)).astype(np.float32)
    mask = np.full((24, 24), 15, np.uint8)
    g = gpu_run(rl, y, mask, nu_max=256, layout=APERTURE, gamma_odc=1.0, rho_decay=1.0, q_mode=1, path=path)
    b = 5 * 12 + 5                                     # window inside the image
    sel = g["sel"][b].astype(np.int64) & 0xFFFF
    k1, k2 = sel // 32, sel % 32
    assert not np.any((k1 == 16) | (k2 == 16))
    assert sorted(((k1 % 16) * 16 + k2 % 16).tolist()) == list(range(256))
    blk = g["hr"][20:24, 20:24].astype(np.float64)
    np.testing.assert_allclose(blk.reshape(2, 2, 2, 2).sum(axis=(1, 3)), y[10:12, 10:12], atol=2e-4)
    allsel = g["sel"].astype(np.int64) & 0xFFFF
    assert not np.any((allsel // 32 == 16) | (allsel % 32 == 16))


def test_layout_errors(rl):
    mask, y = layout_case("quarter", seed=6)

    def status(fn):
        with pytest.raises(rl.RljsdeError) as e:
            fn()
        return e.value.status

    # in-kernel tables take three-quarter apertures only
    assert status(lambda: rl.Plan(mask, rl.default_params(layout=APERTURE, path=3))) == 8
    assert status(lambda: rl.Plan(np.full((8, 8), 16, np.uint8), rl.default_params(layout=APERTURE))) == 3
    assert status(lambda: rl.Plan(np.full((8, 8), 4, np.uint8), rl.default_params())) == 3
    assert status(lambda: rl.Plan(mask, rl.default_params(layout=2))) == 1
    plan = rl.Plan(mask, rl.default_params(layout=APERTURE))
    import torch
    lr = torch.from_numpy(y).cuda()
    hr = torch.zeros((2 * mask.shape[0], 2 * mask.shape[1]), device="cuda")
    sl = torch.zeros(plan.info()["n_blocks"] * rl.SHORTLIST_BYTES, dtype=torch.uint8, device="cuda")
    # the learned proposal reads opaque-sub-pixel codes
    assert status(lambda: plan.reconstruct_learned(lr, hr, sl, max_missing=1e9)) == 8
