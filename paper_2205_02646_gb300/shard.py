"""Splitting RL-JSDE work across GPUs (one process per GPU).

Every 4x4 target block is reconstructed independently from its own 32x32
model window (Sec. III-IV), so the work partitions with no exchange on the
data path:

* a batch of images is split by images, balancing HR pixels per rank;
* one large image is split by block rows.  Rank r keeps block rows
  [a, b) and reconstructs the LR rows [2a - 8, 2b + 8) (clipped to the image):
  the window of block row i spans LR rows [2i - 7, 2i + 9), so a halo of 7
  rows suffices, and 8 keeps the sub-image aligned to the 4-pixel block grid.
  The halo is read once before the launch; the kept HR rows of different
  ranks are disjoint.

Only host-side arithmetic on indices lives here, plus a max-over-ranks
helper for timing.
"""
from __future__ import annotations

HALO_LR = 8


def split_images(sizes, world: int, rank: int):
    """Indices of the images (given as (h, w)) that ``rank`` reconstructs:
    greedy largest-first assignment to the least-loaded rank."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    order = sorted(range(len(sizes)), key=lambda i: (-sizes[i][0] * sizes[i][1], i))
    load = [0] * world
    owner = [0] * len(sizes)
    for i in order:
        r = min(range(world), key=lambda j: (load[j], j))
        owner[i] = r
        load[r] += sizes[i][0] * sizes[i][1]
    return [i for i in range(len(sizes)) if owner[i] == rank]


def split_rows(lr_h: int, world: int, rank: int):
    """Row shard of an image with ``lr_h`` LR rows (even).

    Returns ``(lr0, lr1, keep0, keep1)``: reconstruct the sub-image of LR rows
    [lr0, lr1); its HR rows [keep0, keep1) are this rank's part of the output,
    at full-image HR rows [2 lr0 + keep0, 2 lr0 + keep1).
    """
    if lr_h % 2 or lr_h < 4:
        raise ValueError("lr_h must be even and >= 4")
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    nbh = lr_h // 2
    a = nbh * rank // world
    b = nbh * (rank + 1) // world
    lr0 = max(0, 2 * a - HALO_LR)
    lr1 = min(lr_h, 2 * b + HALO_LR)
    return lr0, lr1, 4 * a - 2 * lr0, 4 * b - 2 * lr0


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a float over all ranks of the default process group (the
    slowest rank sets the measured time)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
