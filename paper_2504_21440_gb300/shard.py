"""Multi-GPU sharding of the quantum-trajectory ensemble.

Trajectories are independent (Sec. 3.3): rank r of W integrates its own
contiguous range of trajectory ids (the Philox stream of trajectory j does
not depend on which rank or process runs it), and one all-reduce of the
per-rank sums of <psi|O|psi>/<psi|psi> gives the ensemble mean on every
rank.  A single master-equation solve is not sharded (one GPU runs it).
"""
import numpy as np


def trajectory_shard(ntraj, rank, world):
    """(first id, count) of rank's contiguous share of ntraj trajectories;
    the shares cover 0..ntraj-1 exactly once and differ by at most one."""
    if world < 1 or not 0 <= rank < world or ntraj < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(ntraj, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def combine_means(local_mean, local_count, group=None):
    """Ensemble mean from per-rank means: all-reduce of mean * count (complex
    values carried as real pairs) and of the counts, over torch.distributed."""
    import torch
    import torch.distributed as dist
    m = np.asarray(local_mean, dtype=np.complex128)
    buf = torch.from_numpy(np.concatenate([(m * local_count).real.ravel(), (m * local_count).imag.ravel(),
                                           [float(local_count)]]))
    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    k = m.size
    tot = buf[-1].item()
    return ((buf[:k].numpy() + 1j * buf[k:2 * k].numpy()) / tot).reshape(m.shape), int(tot)


def mcsolve_sharded(system, psi0, tlist, ntraj, seed, rank, world, group=None, **opts):
    """mcsolve of this rank's trajectory share on its GPU, then the
    ensemble mean over all ranks (identical on every rank)."""
    first, count = trajectory_shard(ntraj, rank, world)
    out = system.mcsolve(psi0, tlist, count, seed, traj_offset=first, **opts) if count else None
    local = out["expect"] if out is not None else np.zeros((system.n_e, len(tlist)), complex)
    return combine_means(local, count, group)
