"""The several-GPU host logic (replicas and ensemble shards) with world size 2 over gloo on CPU."""
import os
import socket

import pytest

from paper_2305_09020_gb300 import replicas


def test_shard_is_balanced_disjoint_and_complete():
    for n in (0, 1, 5, 256, 257):
        for world in (1, 2, 3, 8):
            parts = [replicas.shard(n, r, world) for r in range(world)]
            flat = [u for p in parts for u in p]
            assert flat == list(range(n))
            assert max(len(p) for p in parts) - min(len(p) for p in parts) <= 1
    with pytest.raises(ValueError):
        replicas.shard(4, 2, 2)


def test_single_process_fallbacks():
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.gather_counts(7) == [7]
    assert replicas.job_rate([10, 30], 2.0) == 20.0


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, n_runs, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = replicas.shard(n_runs, rank, world)
        t = 1.0 + rank                                 # rank 1 is the slow one
        tmax = replicas.max_over_ranks(t)
        counts = replicas.gather_counts(len(mine))
        rate = replicas.job_rate(counts, tmax)
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
            f.write(f"{mine.start} {mine.stop} {tmax} {' '.join(map(str, counts))} {rate}\n")
    finally:
        dist.destroy_process_group()


def test_two_ranks_over_gloo(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    world, n_runs = 2, 257
    mp.start_processes(_rank_main, args=(world, _free_port(), n_runs, str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    lines = [open(tmp_path / f"r{r}.txt").read().split() for r in range(world)]
    (s0, e0, t0, c00, c01, r0), (s1, e1, t1, c10, c11, r1) = lines
    assert (int(s0), int(e0), int(s1), int(e1)) == (0, 129, 129, 257)     # disjoint, complete shards
    assert float(t0) == float(t1) == 2.0                                   # both see the slowest time
    assert [int(c00), int(c01)] == [int(c10), int(c11)] == [129, 128]
    assert float(r0) == float(r1) == pytest.approx(257 / 2.0)
