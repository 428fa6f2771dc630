"""The N > 1 path on CPU: two gloo ranks, each with its own shard of rows.

Rows are independent, so sharding needs no collective on the data path;
torch.distributed only carries the barrier and the max over ranks of the
timings.  Checked here: the per-rank shards are the bench's (seed 2 + rank),
the max-over-ranks reduction is the bench's, and per-rank results (the oracle,
CPU) equal a single-process run over the concatenated shards.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    import oracle
    from paper_2606_17065_gb300 import workloads

    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = workloads.stress_batch(512, seed=bench.shard_seed(rank))
    P, _ = oracle.black_price(b.F, b.K, b.T, b.sigma_star, b.flag)
    P = workloads.merge_prices(b, P)
    sig, st = oracle.implied_vol(b.F, b.K, b.T, P, b.flag)
    bench.barrier(world)
    t_max = bench.max_over_ranks(float(rank + 1) * 1.5, world)
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), sig=sig, st=st, t_max=t_max)
    dist.destroy_process_group()


def test_two_rank_shards_match_single_process(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    import bench
    import oracle
    from paper_2606_17065_gb300 import workloads

    for rank in range(world):
        got = np.load(tmp_path / f"rank{rank}.npz")
        assert float(got["t_max"]) == 1.5 * world  # max over ranks
        b = workloads.stress_batch(512, seed=bench.shard_seed(rank))
        P, _ = oracle.black_price(b.F, b.K, b.T, b.sigma_star, b.flag)
        P = workloads.merge_prices(b, P)
        sig, st = oracle.implied_vol(b.F, b.K, b.T, P, b.flag)
        assert np.array_equal(got["st"], st)
        assert np.array_equal(got["sig"], sig, equal_nan=True)
    # the shards are distinct rows
    a = workloads.stress_batch(512, seed=bench.shard_seed(0))
    c = workloads.stress_batch(512, seed=bench.shard_seed(1))
    assert not np.array_equal(a.K, c.K)
