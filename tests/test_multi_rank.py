"""Multi-rank host logic on the CPU: gloo ranks shard a batch, compute heights independently, and the gathered
result equals the single-process one (the engine itself is covered per GPU by the parity tests)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2502_12428_gb300 import inputs
from paper_2502_12428_gb300.shard import shard_range, weak_rows


def test_shard_range_covers_exactly():
    for n in (0, 1, 7, 100, 65536):
        for world in (1, 2, 3, 8):
            parts = [shard_range(n, world, r) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
            sizes = [e - b for b, e in parts]
            assert max(sizes) - min(sizes) <= 1


def test_weak_rows_match_one_shot_generation():
    n = 300
    full = inputs.dense(7, 2 * n, 99)
    for r in range(2):
        b, e = weak_rows(n, r)
        assert np.array_equal(inputs.dense(7, n, 99, row0=b), full[b:e])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, p, n, seed, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    f = inputs.dense(p, n, seed)
    b, e = shard_range(n, world, rank)
    mine = torch.from_numpy(oracle.heights(p, f[b:e], threads=1).astype(np.int64))
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, torch.tensor([e - b]))
    width = int(max(s.item() for s in sizes))
    padded = torch.full((width,), -9, dtype=torch.int64)
    padded[:e - b] = mine
    buf = [torch.zeros(width, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(buf, padded)
    buf = [x[:int(s.item())] for x, s in zip(buf, sizes)]
    # max-over-ranks reduction used for timing
    t = torch.tensor([float(rank + 1)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        np.save(out_path, np.concatenate([x.numpy() for x in buf] + [np.array([t.item()])]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_gloo_shards_concatenate_to_single_run(tmp_path, world):
    import oracle
    oracle.build()
    p, n, seed = 5, 203, 4321
    out = str(tmp_path / "heights.npy")
    mp.start_processes(_worker, args=(world, _free_port(), p, n, seed, out), nprocs=world, start_method="spawn")
    got = np.load(out)
    assert got[-1] == world
    assert np.array_equal(got[:-1], oracle.heights(p, inputs.dense(p, n, seed)).astype(np.int64))
