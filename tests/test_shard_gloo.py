"""Host logic of the multi-GPU path on CPU with two gloo ranks: the
trajectory shares cover every id once, and the all-reduced combination of
per-rank means equals the mean over all trajectories."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2504_21440_gb300.shard import trajectory_shard


@pytest.mark.parametrize("ntraj,world", [(1000, 2), (7, 2), (1, 2), (2001, 8), (0, 3)])
def test_shares_cover_every_trajectory_once(ntraj, world):
    ids = []
    for r in range(world):
        first, count = trajectory_shard(ntraj, r, world)
        ids += list(range(first, first + count))
    assert ids == list(range(ntraj))
    counts = [trajectory_shard(ntraj, r, world)[1] for r in range(world)]
    assert max(counts) - min(counts) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, per_traj, q):
    import torch.distributed as dist
    from paper_2504_21440_gb300.shard import combine_means, trajectory_shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    first, count = trajectory_shard(len(per_traj), rank, world)
    local = per_traj[first:first + count].mean(axis=0) if count else np.zeros(per_traj.shape[1:], complex)
    mean, tot = combine_means(local, count)
    q.put((rank, mean, tot))
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_two_ranks_combine_to_the_full_mean():
    rng = np.random.default_rng(0)
    per_traj = rng.normal(size=(37, 2, 5)) + 1j * rng.normal(size=(37, 2, 5))
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, per_traj, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    full = per_traj.mean(axis=0)
    for rank, mean, tot in out:
        assert tot == 37
        assert np.max(np.abs(mean - full)) < 1e-14
