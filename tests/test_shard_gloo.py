"""Multi-process (gloo, CPU) checks of the work split across GPUs: row shards
with halos reproduce the full-image reconstruction exactly, image shards
cover a batch once, and timing takes the max over ranks."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2205_02646_gb300 import shard, synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    import torch
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import oracle
    from paper_2205_02646_gb300 import shard, synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        f = synth.image(48, 40, 16, 2, 123)
        mask = synth.recurrent_mask(24, 20, 4, 5)
        y = synth.measure(f, mask)
        p = oracle.Params(nu_max=12)
        lr0, lr1, k0, k1 = shard.split_rows(mask.shape[0], world, rank)
        sub = oracle.reconstruct(np.ascontiguousarray(y[lr0:lr1]), np.ascontiguousarray(mask[lr0:lr1]), p,
                                 n_threads=1)
        part = torch.from_numpy(np.ascontiguousarray(sub[k0:k1]))
        rows = torch.tensor([2 * lr0 + k0, 2 * lr0 + k1])
        sizes = [torch.zeros(2, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(sizes, rows)
        parts = [torch.zeros((int(s[1] - s[0]), part.shape[1]), dtype=part.dtype) for s in sizes]
        dist.all_gather(parts, part)
        batch = [(64, 32), (16, 16), (128, 96), (40, 40), (8, 200)]
        own = shard.split_images(batch, world, rank)
        mine = torch.tensor(own + [-1] * (len(batch) - len(own)))
        alls = [torch.zeros_like(mine) for _ in range(world)]
        dist.all_gather(alls, mine)
        tmax = shard.max_over_ranks(1.0 + rank)
        if rank == 0:
            full = oracle.reconstruct(y, mask, p, n_threads=1)
            got = np.concatenate([x.numpy() for x in parts], axis=0)
            spans = [tuple(int(v) for v in s) for s in sizes]
            imgs = sorted(int(v) for a in alls for v in a if v >= 0)
            q.put(dict(equal=bool(np.array_equal(got, full)), spans=spans, imgs=imgs, tmax=tmax))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_row_and_image_shards_gloo(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    import queue
    import time
    out = None
    t0 = time.time()
    while out is None and time.time() - t0 < 120:
        try:
            out = q.get(timeout=1)
        except queue.Empty:
            if any(p.exitcode not in (None, 0) for p in procs):
                break
    for p in procs:
        p.join(timeout=60)
        if p.is_alive():
            p.kill()
        assert p.exitcode == 0
    assert out is not None
    assert out["equal"]
    spans = out["spans"]
    assert spans[0][0] == 0 and spans[-1][1] == 48
    assert all(spans[i][1] == spans[i + 1][0] for i in range(world - 1))
    assert out["imgs"] == [0, 1, 2, 3, 4]
    assert out["tmax"] == float(world)


def test_split_rows_edges():
    for lr_h in (4, 6, 30, 64):
        for world in (1, 2, 5):
            cover = []
            for r in range(world):
                lr0, lr1, k0, k1 = shard.split_rows(lr_h, world, r)
                assert lr0 % 2 == 0 and 0 <= lr0 < lr1 <= lr_h
                assert k0 % 4 == 0 and k1 % 4 == 0 and 0 <= k0 <= k1 <= 2 * (lr1 - lr0)
                cover += list(range(2 * lr0 + k0, 2 * lr0 + k1))
            assert cover == list(range(2 * lr_h))
    with pytest.raises(ValueError):
        shard.split_rows(7, 2, 0)
    assert sorted(sum((shard.split_images([(8, 8)] * 7, 3, r) for r in range(3)), [])) == list(range(7))
