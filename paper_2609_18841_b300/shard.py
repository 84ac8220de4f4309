"""Trajectory sharding across ranks (one process per GPU).

Quantum trajectories are independent samples of the unravelled Lindblad
evolution (Section 5: the density matrix is the average over trajectories), so
the ensemble partitions into contiguous ranges of global trajectory ids with no
exchange during the evolution.  The jump draws of a trajectory are keyed by its
global id (Philox counter traj_offset + local index), so a sharded run samples
exactly the trajectories an unsharded run would.  The only collective is the
final reduction of the ensemble statistics: per observable the count, the sum
and the centred second moment, merged with Chan et al.'s pairwise update so
that the result is the mean and CLT error sqrt(var / n) of the whole ensemble
(Eq. ErrorCLT).
"""
import numpy as np


def shard_range(n_total, rank, world):
    """Contiguous share of n_total trajectories for `rank` of `world`:
    returns (traj_offset, n_local); the first n_total % world ranks take one
    extra trajectory."""
    if world < 1 or not (0 <= rank < world) or n_total < 0:
        raise ValueError("bad shard request: n_total=%r rank=%r world=%r" % (n_total, rank, world))
    base, extra = divmod(n_total, world)
    n_local = base + (1 if rank < extra else 0)
    offset = rank * base + min(rank, extra)
    return offset, n_local


def local_moments(mean, sem, n):
    """(n, mean, M2) of one shard from the mean and CLT error that
    lt_measure_density reports (sem = sqrt(var / n), var the population
    variance), so M2 = n * var = n^2 * sem^2."""
    mean = np.asarray(mean, dtype=np.float64)
    sem = np.asarray(sem, dtype=np.float64)
    return float(n), mean, (n * sem) ** 2 if n > 1 else np.zeros_like(mean)


def merge_moments(a, b):
    """Pairwise merge of (n, mean, M2) triples (Chan, Golub and LeVeque)."""
    na, ma, qa = a
    nb, mb, qb = b
    n = na + nb
    if n == 0:
        return 0.0, ma, qa
    d = mb - ma
    mean = ma + d * (nb / n)
    m2 = qa + qb + d * d * (na * nb / n)
    return n, mean, m2


def combine_mean_sem(mean, sem, n, group=None, device=None):
    """Ensemble mean and CLT error over all ranks of `group` from each rank's
    (mean, sem, n).  Without an initialised process group it returns the local
    values.  `device` is where the exchanged tensors live (a CUDA device for
    NCCL, the CPU for gloo)."""
    import torch
    import torch.distributed as dist

    n_loc, m_loc, q_loc = local_moments(mean, sem, n)
    if not (dist.is_available() and dist.is_initialized()):
        sem_loc = np.sqrt(q_loc / n_loc / n_loc) if n_loc > 1 else np.zeros_like(m_loc)
        return m_loc.copy(), sem_loc, int(n_loc)
    world = dist.get_world_size(group)
    M = m_loc.size
    row = torch.zeros(1 + 2 * M, dtype=torch.float64, device=device or "cpu")
    row[0] = n_loc
    row[1:1 + M] = torch.from_numpy(m_loc.reshape(-1))
    row[1 + M:] = torch.from_numpy(np.asarray(q_loc, dtype=np.float64).reshape(-1))
    rows = [torch.empty_like(row) for _ in range(world)]
    dist.all_gather(rows, row, group=group)
    acc = (0.0, np.zeros(M), np.zeros(M))
    for r in rows:  # rank order: the same merge order, hence the same rounding, on every rank
        v = r.cpu().numpy()
        acc = merge_moments(acc, (float(v[0]), v[1:1 + M], v[1 + M:]))
    n_tot, m_tot, q_tot = acc
    shape = m_loc.shape
    sem_tot = np.sqrt(q_tot / n_tot / n_tot) if n_tot > 1 else np.zeros(M)
    return m_tot.reshape(shape), sem_tot.reshape(shape), int(n_tot)
