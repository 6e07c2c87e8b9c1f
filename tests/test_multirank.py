"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2).

The path shards by target: every rank draws its own target batches (seeded by
rank) and traces its own paths, with no data exchange; the job's time is the
slowest rank's (max over ranks).  The test checks both on two gloo ranks.
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
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(10.0 + 5.0 * rank)
    _, batches = bench.workload_batches(rank)
    targets = np.concatenate([b[0] for b in batches])
    np.save(os.path.join(out_dir, f"r{rank}.npy"), np.concatenate([[t], targets.astype(np.float64)]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_and_take_max(tmp_path):
    port = _free_port()
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    r0 = np.load(tmp_path / "r0.npy")
    r1 = np.load(tmp_path / "r1.npy")
    assert r0[0] == 15.0 and r1[0] == 15.0                 # both ranks see the slowest rank's time
    assert not np.array_equal(r0[1:], r1[1:])             # each rank draws its own targets
