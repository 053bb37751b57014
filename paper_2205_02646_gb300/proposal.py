"""Training data, training loop and evaluation of the learned candidate
proposal (the network itself and every step of its arithmetic live in the
CUDA library; this module only moves tensors between those calls).

Labels come from the plain method: for every block of a training image the
GPU loop runs with ``nu_max`` iterations and records its selections; the
block's target set is the first 64 distinct candidates it selected (the
shortlist that would reproduce most of its model), and its iteration target
is the number of iterations after which the remaining coefficient changes
|gamma delta| add up to less than ``eps`` (as a fraction of ``nu_max``); the
benchmark's learned study picks ``eps`` on validation images, never on the
image it reports.  The per-candidate coefficient mass trains the gate.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import rljsde, synth

SHORTLIST = 64


def tail_mass(dc):
    """Per block, the sum of |gamma delta| from each iteration to the end:
    tail[b, i] = sum_{j >= i} |dc[b, j]| (dc: (n, nu_max, 2))."""
    import torch
    mag = torch.sqrt(dc[..., 0] ** 2 + dc[..., 1] ** 2)
    return torch.flip(torch.cumsum(torch.flip(mag, [1]), 1), [1])


def nu_targets(tail, eps: float, nu_max: int):
    """Iteration target (fraction of nu_max): the iterations whose remaining
    |gamma delta| still adds up to eps or more."""
    return (tail >= eps).sum(1).float() / nu_max


def mass_from_trace(sel, dc):
    """Per block and candidate, the plain loop's coefficient mass: the sum of
    |gamma delta| over the iterations that selected it ((n, 1024) float)."""
    import torch
    n = sel.shape[0]
    mag = torch.sqrt(dc[..., 0] ** 2 + dc[..., 1] ** 2)
    out = torch.zeros((n, 1024), dtype=torch.float32, device=sel.device)
    out.scatter_add_(1, sel.long() & 0xFFFF, mag)
    return out


def labels_from_trace(sel, dc, nu_max: int, k: int = SHORTLIST, eps: float = 0.2):
    """Targets (n, 1024) uint8 and iteration fractions (n,) from a trace."""
    import torch
    n = sel.shape[0]
    s = sel.long() & 0xFFFF
    it = torch.arange(nu_max, device=sel.device).expand(n, nu_max)
    first = torch.full((n, 1024), nu_max, dtype=torch.long, device=sel.device)
    first.scatter_reduce_(1, s, it, reduce="amin")
    order = torch.topk(-first, k, dim=1).indices
    chosen = torch.gather(first, 1, order) < nu_max
    targets = torch.zeros((n, 1024), dtype=torch.uint8, device=sel.device)
    targets.scatter_(1, order, chosen.to(torch.uint8))
    return targets, nu_targets(tail_mass(dc), eps, nu_max)


def make_dataset(n_images: int, size: int = 512, blocks_per_image: int = 256, nu_max: int = 100,
                 tiles=None, seed: int = 0, n_sin: int = 256, n_edges: int = 32, device: str = "cuda",
                 keep_tail: bool = False, eps: float = 0.2):
    """Patches, block coordinates, targets and iteration targets for
    ``blocks_per_image`` random blocks of each of ``n_images`` synthetic
    size x size images (mask tiles cycled from ``tiles``).  With
    ``keep_tail`` a last entry holds every sample's tail |gamma delta| sums
    (n, nu_max), from which ``nu_targets`` gives the iteration targets of any
    other threshold.  Entries: patches, blocks, targets, iteration targets,
    image shape, per-candidate mass (``mass_from_trace``), [tails]."""
    import torch
    lr = size // 2
    nb_side = lr // 2
    tiles = tiles if tiles is not None else [synth.recurrent_mask(lr, lr, 4, 1000 + t) for t in range(16)]
    plans = [rljsde.Plan(m, rljsde.default_params(nu_max=nu_max)) for m in tiles]
    masks_d = [torch.from_numpy(m).to(device) for m in tiles]
    nb = nb_side * nb_side
    sel = torch.empty(nb * nu_max, dtype=torch.int16, device=device)
    dc = torch.empty(nb * nu_max * 2, dtype=torch.float32, device=device)
    hr = torch.empty((size, size), device=device)
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    xs, bs, ts, ns, ms, tails = [], [], [], [], [], []
    for i in range(n_images):
        t = i % len(tiles)
        f = synth.image_torch(size, size, n_sin, n_edges, seed * 100003 + i, 0.005, device)
        y = synth.measure_torch(f, masks_d[t]).float().contiguous()
        plans[t].reconstruct_trace(y, hr, sel, dc)
        pick = torch.randperm(nb, generator=g, device=device)[:blocks_per_image]
        dcp = dc.view(nb, nu_max, 2)[pick]
        selp = sel.view(nb, nu_max)[pick]
        tg, nu_t = labels_from_trace(selp, dcp, nu_max, eps=eps)
        ms.append(mass_from_trace(selp, dcp))
        blk = torch.stack([pick // nb_side, pick % nb_side], 1).int().contiguous()
        xs.append(rljsde.Net.patches(y, masks_d[t], blk))
        bs.append(blk)
        ts.append(tg)
        ns.append(nu_t)
        if keep_tail:
            tails.append(tail_mass(dcp))
    for p in plans:
        p.check()
    out = (torch.cat(xs), torch.cat(bs), torch.cat(ts), torch.cat(ns), (lr, lr), torch.cat(ms))
    return out + (torch.cat(tails),) if keep_tail else out


def train(net, data, epochs: int = 8, batch: int = 4096, lr: float = 2e-3, seed: int = 0, log=None,
          gate_weight: float = 10.0):
    """Adam with cosine decay over ``epochs`` passes of ``data`` (patches,
    blocks, targets, iteration targets, shape, mass).  The share the gate
    predicts varies little across blocks (standard deviation about 0.04
    around 0.26 on generator images), so its squared error weighs 10: at 1
    the gate learned a constant (rank correlation with the share -0.04 on
    held-out patches), at 10 it ranks them (0.20), at 50 it saturated."""
    import torch
    x, blocks, targets, nu_t, shape, mass = data[:6]
    n = x.shape[0]
    g = torch.Generator(device=x.device)
    g.manual_seed(seed)
    steps = epochs * max(1, n // batch)
    step = 0
    losses = []
    for e in range(epochs):
        perm = torch.randperm(n, generator=g, device=x.device)
        for i in range(0, n - batch + 1, batch):
            idx = perm[i:i + batch]
            rate = lr * 0.5 * (1.0 + math.cos(math.pi * step / steps))
            losses.append(net.train_step(x[idx].contiguous(), blocks[idx].contiguous(), shape,
                                         targets[idx].contiguous(), nu_t[idx].contiguous(), mass[idx].contiguous(),
                                         lr=rate, gate_weight=gate_weight))
            step += 1
        if log:
            log("epoch %d loss %.4f" % (e, float(np.mean(losses[-max(1, n // batch):]))))
    return losses


def gate_rank_correlation(net, data, k: int = SHORTLIST):
    """Spearman correlation, over the samples of ``data``, between the gate
    (sigmoid of head row 1025) and the share of the sample's mass that falls
    outside the network's own top-k logits, the quantity it is trained to
    predict."""
    import torch
    x, blocks, targets, nu_t, shape, mass = data[:6]
    gs, ss = [], []
    for i in range(0, x.shape[0], 8192):
        z = net.logits(x[i:i + 8192].contiguous(), blocks[i:i + 8192].contiguous(), shape)
        top = torch.topk(z[:, :1024], k, dim=1).indices
        inside = torch.zeros_like(mass[i:i + 8192], dtype=torch.bool)
        inside.scatter_(1, top, True)
        m = mass[i:i + 8192]
        ss.append(((m * (~inside)).sum(1) / m.sum(1).clamp_min(1e-12)).cpu().numpy())
        gs.append(torch.sigmoid(z[:, 1025]).cpu().numpy())
    g, s = np.concatenate(gs), np.concatenate(ss)
    rg, rs = np.argsort(np.argsort(g)), np.argsort(np.argsort(s))
    return float(np.corrcoef(rg, rs)[0, 1])


def recall(net, data, k: int = SHORTLIST):
    """Mean fraction of each block's target set found in its top-k logits."""
    import torch
    x, blocks, targets, nu_t, shape = data[:5]
    hits, total = 0, 0
    for i in range(0, x.shape[0], 8192):
        z = net.logits(x[i:i + 8192].contiguous(), blocks[i:i + 8192].contiguous(), shape)
        top = torch.topk(z[:, :1024], k, dim=1).indices
        hits += int(torch.gather(targets[i:i + 8192], 1, top).sum())
        total += int(targets[i:i + 8192].sum())
    return hits / max(total, 1)


def psnr(a, b):
    mse = float(((a - b) ** 2).mean())
    return 10.0 * math.log10(1.0 / mse) if mse > 0 else float("inf")
