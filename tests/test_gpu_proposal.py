"""GPU tests of the learned candidate proposal (this library's extension):
network gradients against the FP64 reference, the whole-image pass against
per-patch logits, and the shortlist-restricted greedy loop against the FP64
oracle (the loop with q = 0 outside the shortlist is the same problem)."""
import numpy as np
import pytest

import oracle
from oracle import cnn_ref
from paper_2205_02646_gb300 import synth
from parity import compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rl():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_02646_gb300 import build, rljsde
    build.build()
    rljsde.load()
    return rljsde


def _image(h=48, w=64, seed=5):
    f = synth.image(2 * h, 2 * w, 24, 3, 9100 + seed)
    mask = synth.recurrent_mask(h, w, 4, 30 + seed)
    y = synth.measure(f, mask).astype(np.float32)
    return f, mask, y


def test_gradients_match_fp64_reference(rl):
    import torch
    f, mask, y = _image(24, 24)
    net = rl.Net(seed=3)
    rng = np.random.default_rng(0)
    params = net.get_params()
    # larger head weights than the init so every term of the gradient matters
    params[cnn_ref.N_PARAMS - 1026 - 1026 * 288:cnn_ref.N_PARAMS - 1026] = rng.normal(0, 0.05, 1026 * 288)
    net.set_params(params)
    blocks = np.array([[0, 0], [5, 7], [11, 2], [6, 11]], np.int32)
    lr = torch.from_numpy(y).cuda()
    md = torch.from_numpy(mask).cuda()
    bd = torch.from_numpy(blocks).cuda()
    x = rl.Net.patches(lr, md, bd)
    targets = (rng.random((4, 1024)) < 0.07).astype(np.uint8)
    nus = rng.random(4).astype(np.float32)
    mass = (rng.random((4, 1024)) * (rng.random((4, 1024)) < 0.1)).astype(np.float32)
    g, loss = net.gradient(x, bd, mask.shape, torch.from_numpy(targets).cuda(), torch.from_numpy(nus).cuda(),
                           torch.from_numpy(mass).cuda())
    xs, origins = zip(*[cnn_ref.patch(y, mask, int(bi), int(bj)) for bi, bj in blocks])
    np.testing.assert_allclose(x.cpu().numpy(), np.array(xs), rtol=0, atol=1e-7)
    ref_loss, ref_g = cnn_ref.loss_and_grads(cnn_ref.unflatten(params), list(xs), list(origins), mask.shape,
                                             list(targets.astype(float)), list(nus.astype(float)),
                                             list(mass.astype(float)))
    assert abs(loss - ref_loss) <= 1e-4 * abs(ref_loss)
    got = cnn_ref.unflatten(g.cpu().numpy())
    for name, _ in cnn_ref.SHAPES:
        a, b = got[name], ref_g[name]
        scale = np.abs(b).max() + 1e-12
        assert np.abs(a - b).max() <= 2e-3 * scale, (name, np.abs(a - b).max(), scale)


def test_whole_image_shortlists_match_patch_logits(rl):
    import torch
    f, mask, y = _image()
    net = rl.Net(seed=7)
    plan = rl.Plan(mask, rl.default_params(nu_max=10))
    lr = torch.from_numpy(y).cuda()
    buf = plan.propose(net, lr)
    torch.cuda.synchronize()
    nbh, nbw = mask.shape[0] // 2, mask.shape[1] // 2
    idx, missing, nu_frac = rl.shortlist_view(buf, nbh * nbw)
    for row in idx:
        assert len(set(row.tolist())) == 64 and row.max() < 1024
    blocks = np.array([[0, 0], [3, 5], [nbh - 1, nbw - 1], [10, 0], [7, 20]], np.int32)
    z = net.logits(rl.Net.patches(lr, torch.from_numpy(mask).cuda(), torch.from_numpy(blocks).cuda()),
                   torch.from_numpy(blocks).cuda(), mask.shape).cpu().numpy()
    for (bi, bj), zb in zip(blocks, z):
        top = set(np.argsort(-zb[:1024], kind="stable")[:64].tolist())
        got = set(idx[bi * nbw + bj].tolist())
        assert len(top & got) >= 56          # head features go through bf16 in the whole-image pass
        assert abs(nu_frac[bi * nbw + bj] - zb[1024]) < 0.05 * (1 + abs(zb[1024]))


@pytest.mark.parametrize("shape", [(40, 56), (36, 560)])
def test_tensor_core_convolutions_match_fp64_features(rl, shape):
    """conv2 and conv3 of the whole-image pass run on the tensor cores
    (tcgen05, bfloat16 taps, FP32 accumulation in tensor memory; input rows
    staged by TMA, 128 output positions of a row per tile).  A head whose
    iteration row selects one feature turns each block's iteration output
    into that feature, which must equal the FP64 reference's up to bfloat16
    rounding of the activations.  The second shape has block rows of 280
    positions: two full tiles and a ragged one, checked at the tile seams."""
    import torch
    f, mask, y = _image(h=shape[0], w=shape[1], seed=8)
    net = rl.Net(seed=11)
    base = cnn_ref.unflatten(net.get_params())
    plan = rl.Plan(mask, rl.default_params(nu_max=10))
    lr = torch.from_numpy(y).cuda()
    nbh, nbw = mask.shape[0] // 2, mask.shape[1] // 2
    rng = np.random.default_rng(4)
    blocks = [(0, 0), (0, nbw - 1), (nbh - 1, 0), (nbh - 1, nbw - 1), (1, 2)] + \
        [tuple(b) for b in rng.integers(0, [nbh, nbw], (20, 2))]
    if nbw > 128:
        blocks += [(0, 127), (0, 128), (nbh - 1, 255), (nbh - 1, 256), (nbh // 2, nbw - 2), (3, 129)]
    ref = {}
    for bi, bj in blocks:
        x, origin = cnn_ref.patch(y, mask, bi, bj)
        ref[(bi, bj)] = cnn_ref.forward(base, x, origin, mask.shape)[1][-1]      # the 288 head features
    scale = max(np.abs(v).max() for v in ref.values())
    assert scale > 0.1
    for fi in (0, 4, 148, 287):                                                # channel 0 / 16 / 31, several taps
        p = {k: v.copy() for k, v in base.items()}
        p["head.w"][:] = 0.0
        p["head.w"][1024, fi] = 1.0
        p["head.b"][:] = 0.0
        net.set_params(cnn_ref.flatten(p).astype(np.float32))
        _, _, nu_frac = rl.shortlist_view(plan.propose(net, lr), nbh * nbw)
        plan.check()
        for (bi, bj), fr in ref.items():
            got = float(nu_frac[bi * nbw + bj])
            assert abs(got - fr[fi]) <= 0.02 * scale + 0.01 * abs(fr[fi]), (fi, bi, bj, got, fr[fi])


@pytest.mark.parametrize("c_supply", [0, 2])        # Gram columns read from the stored C / rebuilt
@pytest.mark.parametrize("seed", [1, 2])
def test_restricted_loop_matches_oracle_with_q_zero_outside(rl, seed, c_supply):
    import torch
    f, mask, y = _image(24, 24, seed)
    nbh, nbw = 12, 12
    nb = nbh * nbw
    nu = 40
    rng = np.random.default_rng(seed)
    idx = np.stack([rng.choice(1024, 64, replace=False) for _ in range(nb)])
    buf = torch.from_numpy(rl.shortlist_from_indices(idx)).cuda()
    plan = rl.Plan(mask, rl.default_params(nu_max=nu, c_supply=c_supply))
    assert (plan.info()["n_stored_c_tables"] == plan.info()["n_tables"]) == (c_supply == 0)
    lr = torch.from_numpy(y).cuda()
    hr = torch.zeros((48, 48), device="cuda")
    sel = torch.zeros(nb * nu, dtype=torch.int16, device="cuda")
    dc = torch.zeros(nb * nu * 2, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    plan.reconstruct_learned(lr, hr, buf, max_missing=1e9, sel=sel, dc=dc, counter=cnt)
    plan.check()
    assert int(cnt.item()) == nb
    g_hr, g_sel = hr.cpu().numpy(), sel.cpu().numpy().reshape(nb, nu)
    qd = oracle.frequency_weight(oracle.Params()).ravel()
    blocks = list(range(0, nb, 5))
    o_hr = np.full((48, 48), np.nan)
    o_sel, o_gap = [], []
    for b in blocks:
        qt = np.zeros(1024)
        qt[idx[b]] = qd[idx[b]]
        h_b, tr = oracle.reconstruct(y.astype(np.float64), mask, oracle.Params(nu_max=nu, q_mode=2, q_table=qt),
                                     blocks=[b], trace=True)
        bi, bj = divmod(b, nbw)
        o_hr[4 * bi:4 * bi + 4, 4 * bj:4 * bj + 4] = h_b[4 * bi:4 * bi + 4, 4 * bj:4 * bj + 4]
        o_sel.append(tr["sel"][0])
        o_gap.append(tr["gap"][0])
    res = compare(g_hr, g_sel[blocks], o_hr, np.array(o_sel), np.array(o_gap), blocks, nbw, tol=1e-4, tie=1e-4)
    assert not res["fails"], res["fails"][:3]


@pytest.mark.parametrize("c_supply", [0, 2])
def test_shortlist_of_plain_selections_reproduces_plain_loop(rl, c_supply):
    """If the shortlist holds every candidate the full loop selects, the
    restricted argmax makes the same choices."""
    import torch
    f, mask, y = _image(32, 32, 4)
    nu = 40
    nb = 16 * 16
    plan = rl.Plan(mask, rl.default_params(nu_max=nu, c_supply=c_supply))
    lr = torch.from_numpy(y).cuda()
    hr = torch.zeros((64, 64), device="cuda")
    sel = torch.zeros(nb * nu, dtype=torch.int16, device="cuda")
    dc = torch.zeros(nb * nu * 2, device="cuda")
    plan.reconstruct_trace(lr, hr, sel, dc)
    ps = sel.cpu().numpy().reshape(nb, nu).astype(np.int64) & 0xFFFF
    idx = np.zeros((nb, 64), np.int64)
    for b in range(nb):
        seen = list(dict.fromkeys(ps[b].tolist()))
        rest = [k for k in range(1024) if k not in seen]
        idx[b] = (seen + rest)[:64]
    buf = torch.from_numpy(rl.shortlist_from_indices(idx)).cuda()
    hr2 = torch.zeros_like(hr)
    sel2 = torch.zeros_like(sel)
    dc2 = torch.zeros_like(dc)
    plan.reconstruct_learned(lr, hr2, buf, max_missing=1e9, sel=sel2, dc=dc2)
    plan.check()
    s2 = sel2.cpu().numpy().reshape(nb, nu).astype(np.int64) & 0xFFFF
    same = (s2 == ps).all(axis=1)
    assert same.mean() >= 0.97
    d = np.abs(hr2.cpu().numpy() - hr.cpu().numpy()).reshape(16, 4, 16, 4).max(axis=(1, 3)).ravel()
    assert d[same].max() <= 1e-4


def test_training_lowers_the_loss(rl):
    import torch
    f, mask, y = _image(64, 64, 9)
    nu = 30
    nb = 32 * 32
    plan = rl.Plan(mask, rl.default_params(nu_max=nu))
    lr = torch.from_numpy(y).cuda()
    hr = torch.zeros((128, 128), device="cuda")
    sel = torch.zeros(nb * nu, dtype=torch.int16, device="cuda")
    dc = torch.zeros(nb * nu * 2, device="cuda")
    plan.reconstruct_trace(lr, hr, sel, dc)
    s = sel.cpu().numpy().reshape(nb, nu).astype(np.int64) & 0xFFFF
    targets = np.zeros((nb, 1024), np.uint8)
    for b in range(nb):
        targets[b, list(dict.fromkeys(s[b].tolist()))[:64]] = 1
    blocks = np.array([[b // 32, b % 32] for b in range(nb)], np.int32)
    bd = torch.from_numpy(blocks).cuda()
    x = rl.Net.patches(lr, torch.from_numpy(mask).cuda(), bd)
    td = torch.from_numpy(targets).cuda()
    nud = torch.ones(nb, device="cuda")
    net = rl.Net(seed=1)
    losses = [net.train_step(x, bd, mask.shape, td, nud, lr=2e-3) for _ in range(40)]      # no gate term
    assert losses[-1] < 0.8 * losses[0], losses[::8]


@pytest.mark.parametrize("c_supply", [0, 2])
@pytest.mark.parametrize("tau", [-1.0, 0.1, 0.5, 0.97, 2.0])
def test_mixed_fallback_matches_both_passes(rl, tau, c_supply):
    """With the confidence gate between the extremes, every block is
    reconstructed either by the shortlist loop (left-out mass <= tau) or by
    the full loop (the rest), whatever the other blocks of its chunk take:
    restricted blocks equal the all-restricted run bit for bit, the others
    match the plain loop."""
    import torch
    f, mask, y = _image(96, 128, 7)
    nbh, nbw = 48, 64
    nb = nbh * nbw
    nu = 24
    rng = np.random.default_rng(11)
    idx = np.stack([rng.choice(1024, 64, replace=False) for _ in range(nb)])
    missing = rng.random(nb).astype(np.float32)
    buf = torch.from_numpy(rl.shortlist_from_indices(idx, missing=missing)).cuda()
    plan = rl.Plan(mask, rl.default_params(nu_max=nu, c_supply=c_supply))
    lr = torch.from_numpy(y).cuda()
    hr_p = torch.zeros((2 * 96, 2 * 128), device="cuda")
    plan.reconstruct(lr, hr_p)
    hr_r = torch.zeros_like(hr_p)
    plan.reconstruct_learned(lr, hr_r, buf, max_missing=2.0)
    hr_m = torch.full_like(hr_p, float("nan"))
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    plan.reconstruct_learned(lr, hr_m, buf, max_missing=tau, counter=cnt)
    plan.check()
    restricted = missing <= np.float32(tau)
    assert int(cnt.item()) == int(restricted.sum())
    blk = lambda t: t.cpu().numpy().reshape(nbh, 4, nbw, 4).transpose(0, 2, 1, 3).reshape(nb, 16)
    m, r, p = blk(hr_m), blk(hr_r), blk(hr_p)
    assert np.isfinite(m).all()                       # every block written by one of the passes
    assert np.array_equal(m[restricted], r[restricted])
    d = np.abs(m[~restricted] - p[~restricted]).max(axis=1) if (~restricted).any() else np.zeros(0)
    assert (d <= 1e-4).mean() >= 0.99 if d.size else True


@pytest.mark.parametrize("c_supply", [0, 2])
def test_restricted_loop_with_repeated_candidates(rl, c_supply):
    """A shortlist that names some candidates twice searches the distinct
    candidates it names: the same as the oracle with q = 0 outside them."""
    import torch
    f, mask, y = _image(24, 24, 3)
    nbh, nbw = 12, 12
    nb = nbh * nbw
    nu = 30
    rng = np.random.default_rng(8)
    idx = np.zeros((nb, 64), np.int64)
    for b in range(nb):
        distinct = rng.choice(1024, 48, replace=False)
        idx[b] = np.concatenate([distinct, rng.choice(distinct, 16, replace=True)])
        rng.shuffle(idx[b])
    buf = torch.from_numpy(rl.shortlist_from_indices(idx)).cuda()
    plan = rl.Plan(mask, rl.default_params(nu_max=nu, c_supply=c_supply))
    lr = torch.from_numpy(y).cuda()
    hr = torch.zeros((48, 48), device="cuda")
    sel = torch.zeros(nb * nu, dtype=torch.int16, device="cuda")
    dc = torch.zeros(nb * nu * 2, device="cuda")
    plan.reconstruct_learned(lr, hr, buf, max_missing=1e9, sel=sel, dc=dc)
    plan.check()
    g_hr, g_sel = hr.cpu().numpy(), sel.cpu().numpy().reshape(nb, nu)
    qd = oracle.frequency_weight(oracle.Params()).ravel()
    blocks = list(range(0, nb, 7))
    o_hr = np.full((48, 48), np.nan)
    o_sel, o_gap = [], []
    for b in blocks:
        qt = np.zeros(1024)
        qt[idx[b]] = qd[idx[b]]
        h_b, tr = oracle.reconstruct(y.astype(np.float64), mask, oracle.Params(nu_max=nu, q_mode=2, q_table=qt),
                                     blocks=[b], trace=True)
        bi, bj = divmod(b, nbw)
        o_hr[4 * bi:4 * bi + 4, 4 * bj:4 * bj + 4] = h_b[4 * bi:4 * bi + 4, 4 * bj:4 * bj + 4]
        o_sel.append(tr["sel"][0])
        o_gap.append(tr["gap"][0])
    res = compare(g_hr, g_sel[blocks], o_hr, np.array(o_sel), np.array(o_gap), blocks, nbw, tol=1e-4, tie=1e-4)
    assert not res["fails"], res["fails"][:3]
    assert all(set(g_sel[b].tolist()) <= set(idx[b].tolist()) for b in blocks)


def _key15(z):
    """15-bit ranking key of FP32 logits: z on a fixed-point grid of step
    2^-9 over [-32, 32), rounded down and clamped."""
    t = np.clip((np.asarray(z, np.float32) + np.float32(32.0)) * np.float32(512.0), 0.0, 32767.0)
    return np.floor(t).astype(np.int64)


def _bias_pattern(name, rng):
    if name == "normal":
        return rng.normal(-2.0, 1.5, 1026)
    if name == "ties":                                # few distinct values: exact ties at the threshold
        return rng.choice(np.array([-3.0, -1.0, 0.5, 2.0]), 1026, p=[0.6, 0.3, 0.06, 0.04])
    if name == "below_step":                          # distinct FP32 values within one 2^-9 key step
        return 1.0 + 2.0 ** -20 * rng.integers(0, 64, 1026) - 2.0 * (rng.random(1026) < 0.9)
    if name == "clamped":                             # beyond the key range: ties at its ends
        return np.where(rng.random(1026) < 0.1, 40.0 + rng.random(1026), -40.0 - rng.random(1026))
    return np.full(1026, 0.25)                        # all equal: the 64 lowest indices


@pytest.mark.parametrize("pattern", ["normal", "ties", "below_step", "clamped", "equal"])
def test_fused_selection_exact_on_bias_logits(rl, pattern):
    """With a zero head matrix every block's logits are the head biases
    exactly, so the fused head's shortlist must be the 64 largest biases by
    their 15-bit keys (fixed-point step 2^-9 over [-32, 32)), ties to the
    lower index, in increasing index order, on every block; the iteration
    output is the bias of row 1024 exactly, and the gate the sigmoid of the
    bias of row 1025."""
    import torch
    f, mask, y = _image(40, 56, 2)
    net = rl.Net(seed=4)
    p = cnn_ref.unflatten(net.get_params())
    b = _bias_pattern(pattern, np.random.default_rng(17))
    p["head.w"][:] = 0.0
    p["head.b"][:] = b
    net.set_params(cnn_ref.flatten(p).astype(np.float32))
    plan = rl.Plan(mask, rl.default_params(nu_max=10))
    lr = torch.from_numpy(y).cuda()
    nb = 20 * 28
    idx, missing, nu_frac = rl.shortlist_view(plan.propose(net, lr), nb)
    plan.check()
    b32 = b.astype(np.float32)
    k = _key15(b32[:1024])
    order = np.lexsort((np.arange(1024), -k))         # key descending, then index ascending
    want = np.sort(order[:64])
    assert np.array_equal(idx.astype(np.int64), np.broadcast_to(want, (nb, 64)))
    assert np.all(nu_frac == b32[1024])
    gate = 1.0 / (1.0 + np.exp(-np.float64(b32[1025])))
    np.testing.assert_allclose(missing, gate, rtol=1e-5, atol=1e-7)
