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


# ------------------------------------------------------------------------------------- bench.py's own rank setup
import importlib.util  # noqa: E402
import json  # noqa: E402
import subprocess  # noqa: E402
import sys  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench_module():
    spec = importlib.util.spec_from_file_location("qfs_bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _bench_worker(rank, world, port, out_path):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    bench = _bench_module()
    w, r, local = bench.dist_setup()
    bench.init_ranks("gloo", w)
    slowest = bench.max_over_ranks(10.0 * (r + 1), w)      # each rank's step time; the line takes the largest
    rows = bench.config_batch(2, r)[3]                     # weak scaling: rank r classifies its own rows
    sizes = [torch.zeros(1) for _ in range(w)]
    dist.all_gather(sizes, torch.tensor([float(rows[:, 0].sum())]))
    bench.barrier(w)
    if r == 0:
        np.save(out_path, np.array([w, slowest] + [float(x.item()) for x in sizes]))
    dist.destroy_process_group()


def test_bench_rank_setup_over_gloo(tmp_path):
    out = str(tmp_path / "bench_ranks.npy")
    mp.start_processes(_bench_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
    world, slowest, s0, s1 = np.load(out)
    assert world == 2 and slowest == 20.0
    p, n = 5, 65536
    assert s0 == float(inputs.dense(p, n, inputs.config_seed(2))[:, 0].sum())
    assert s1 == float(inputs.dense(p, n, inputs.config_seed(2), row0=n)[:, 0].sum())


def test_bench_gpus_flag_launches_its_ranks():
    # without torchrun, --gpus 2 re-runs bench.py under torch.distributed.run with two ranks; the reference arm
    # needs no GPU, so both ranks run here over gloo and rank 0 alone prints the line
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "3", "--cpu-sample", "2"], capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    assert lines[0]["n_gpus"] == 2 and lines[0]["impl"] == "reference"


def test_bench_gpus_flag_refuses_more_gpus_than_visible():
    if torch.cuda.is_available():
        pytest.skip("this host has GPUs")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "2"], capture_output=True,
                       text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 2 and "visible" in r.stderr


def test_tensor_tile_count_matches_definition():
    # the tensor form's executed MACs in the bench line: tiles per product from the kernel's enumeration, each 8
    # m16n8k32 tiles of 4096 MACs; for one product of degree m_out every existing (column, 8-output) group of a
    # 16-column group is covered, so tiles >= the word pairs of the data and every tile covers 16 x 8 outputs
    bench = _bench_module()
    for m_out in (8, 28, 96, 168):
        t = bench.tc_tiles(m_out)
        outputs = sum((s + 1) for u in range(m_out + 1) for s in range(u + 1))
        assert t * 16 * 8 >= outputs
    assert bench.tc_executed_macs_per_survivor(7) > 256 / 35 * bench.chain_macs(7, 1, 41) * 0.9
