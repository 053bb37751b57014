"""What the trained proposal network gains over the method without it (an
untrained network of the same shape), on a seconds-scale training run: the
library's own kernels label generator images with the plain loop, train the
network, and run the proposal and the shortlist loop on held-out data.

Checked: the trained network's shortlists hold more of the plain loop's
selections than an untrained one's; the shortlist loop with the trained
network stays close to the plain loop's PSNR on a held-out image while the
untrained network loses several dB; and the gate (the network's predicted
share of the plain loop's coefficient mass its shortlist leaves out) ranks
held-out blocks like the true share."""
import numpy as np
import pytest

from paper_2205_02646_gb300 import synth

pytestmark = pytest.mark.gpu

NU = 60


@pytest.fixture(scope="module")
def trained():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_02646_gb300 import build, proposal, rljsde
    build.build()
    tiles = [synth.recurrent_mask(128, 128, 4, 500 + t) for t in range(4)]
    data = proposal.make_dataset(360, size=256, blocks_per_image=96, nu_max=NU, tiles=tiles, seed=11)
    held = proposal.make_dataset(8, size=256, blocks_per_image=256, nu_max=NU, tiles=tiles, seed=12)
    net = rljsde.Net(seed=2)
    losses = proposal.train(net, data, epochs=12, batch=1024, lr=3e-3)
    untrained = rljsde.Net(seed=2)
    return dict(rl=rljsde, proposal=proposal, net=net, untrained=untrained, held=held, losses=losses, tiles=tiles)


def _held_out_image(tiles):
    f = synth.image(512, 512, 256, 32, 424242, 0.005)
    mask = np.ascontiguousarray(np.tile(tiles[1][:4, :4], (64, 64)))
    return f, mask, synth.measure(f, mask).astype(np.float32)


def test_trained_network_finds_more_of_the_plain_selections(trained):
    rec_t = trained["proposal"].recall(trained["net"], trained["held"])
    rec_u = trained["proposal"].recall(trained["untrained"], trained["held"])
    print("held-out recall@64: trained %.3f, untrained %.3f; loss %.4f -> %.4f"
          % (rec_t, rec_u, trained["losses"][0], trained["losses"][-1]))
    assert rec_t >= rec_u + 0.08
    assert rec_t >= 1.5 * rec_u


def test_shortlist_loop_psnr_trained_vs_untrained(trained):
    import torch
    rl, proposal = trained["rl"], trained["proposal"]
    f, mask, y = _held_out_image(trained["tiles"])
    plan = rl.Plan(mask, rl.default_params(nu_max=NU))
    lr = torch.from_numpy(y).cuda()
    truth = torch.from_numpy(f).cuda()
    hr = torch.zeros((512, 512), device="cuda")
    plan.reconstruct(lr, hr)
    p_plain = proposal.psnr(hr.double(), truth)
    out = {}
    for name in ("net", "untrained"):
        sl = plan.propose(trained[name], lr)
        plan.reconstruct_learned(lr, hr, sl, max_missing=1e9)
        plan.check()
        out[name] = proposal.psnr(hr.double(), truth)
    print("PSNR plain %.3f, trained shortlists %.3f, untrained shortlists %.3f" % (p_plain, out["net"], out["untrained"]))
    assert out["net"] >= p_plain - 0.25
    assert out["net"] >= out["untrained"] + 3.0


def test_gate_ranks_blocks(trained):
    """The gate predicts, per block, the share of the plain loop's
    coefficient mass its shortlist leaves out.  On held-out patches its
    ranking agrees with the true share (Spearman correlation), which an
    untrained gate's does not, and it spreads across blocks by more than
    +-1 % of its median."""
    proposal = trained["proposal"]
    rho_t = proposal.gate_rank_correlation(trained["net"], trained["held"])
    rho_u = proposal.gate_rank_correlation(trained["untrained"], trained["held"])
    import torch
    rl = trained["rl"]
    f, mask, y = _held_out_image(trained["tiles"])
    plan = rl.Plan(mask, rl.default_params(nu_max=NU))
    _, missing, _ = rl.shortlist_view(plan.propose(trained["net"], torch.from_numpy(y).cuda()), 128 * 128)
    plan.check()
    q10, q50, q90 = np.quantile(missing, [0.1, 0.5, 0.9])
    print("gate rank correlation with the left-out share: trained %.3f, untrained %.3f; gate p10/p50/p90 on the "
          "held-out image %.4f %.4f %.4f" % (rho_t, rho_u, q10, q50, q90))
    assert rho_t >= 0.1
    assert rho_t >= rho_u + 0.1
    assert (q90 - q10) / q50 > 0.02
