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


class _OracleSystem:
    """Stands in for qtl.System on a CPU rank: the same mcsolve signature
    (trajectory offset included), answered by the FP64 oracle."""

    def __init__(self, s):
        self.s = s
        self.n_e = len(s.e_ops)

    def mcsolve(self, psi0, tlist, ntraj, seed, traj_offset=0, **kw):
        from oracle.mcsolve import mcsolve
        s = self.s
        return mcsolve(s.H, s.c_ops, s.e_ops, psi0, tlist, ntraj=ntraj, seed=seed,
                       traj_ids=range(traj_offset, traj_offset + ntraj))


def _rank_sharded(rank, world, port, q):
    import torch.distributed as dist
    import workloads as W
    from paper_2504_21440_gb300.shard import mcsolve_sharded
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    s = W.jaynes_cummings(N=3, nt=6, t_end=30.0, kappa=0.2, gamma=0.1)
    mean, tot = mcsolve_sharded(_OracleSystem(s), s.psi0, s.tlist, 13, 4, rank, world)
    q.put((rank, mean, tot))
    dist.barrier()
    dist.destroy_process_group()


def test_mcsolve_sharded_over_two_gloo_ranks_equals_one_ensemble():
    """mcsolve_sharded end to end on two CPU ranks: each rank runs its own
    contiguous trajectory range (through the trajectory offset, so the Philox
    streams are those of the full ensemble), and the all-reduced mean equals
    the single ensemble of 13 trajectories."""
    import workloads as W
    from oracle.mcsolve import mcsolve
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_sharded, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    s = W.jaynes_cummings(N=3, nt=6, t_end=30.0, kappa=0.2, gamma=0.1)
    full = mcsolve(s.H, s.c_ops, s.e_ops, s.psi0, s.tlist, ntraj=13, seed=4)["expect"]
    assert len(out) == 2
    for rank, mean, tot in out:
        assert tot == 13
        assert np.max(np.abs(mean - full)) < 1e-13
