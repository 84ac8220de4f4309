"""Trajectory sharding (one rank per GPU): the shard ranges partition the
ensemble, a sharded oracle run samples exactly the trajectories of the
unsharded one (jump draws keyed by the global trajectory id), and the
cross-rank reduction of (mean, CLT error) equals the statistics of the whole
ensemble.  The multi-rank part runs as two gloo processes on the CPU."""
import os
import socket

import numpy as np
import pytest

from paper_2609_18841_b300 import shard


def test_shard_ranges_partition_the_ensemble():
    for n_total in (0, 1, 7, 64, 4097):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                off, n = shard.shard_range(n_total, r, world)
                seen.extend(range(off, off + n))
            assert seen == list(range(n_total))
    with pytest.raises(ValueError):
        shard.shard_range(4, 2, 2)


def test_merge_moments_equals_whole_sample_statistics():
    rng = np.random.default_rng(3)
    x = rng.random((37, 5))
    parts = [x[:10], x[10:11], x[11:30], x[30:]]
    acc = (0.0, np.zeros(5), np.zeros(5))
    for p in parts:
        var = p.var(axis=0)
        sem = np.sqrt(var / len(p)) if len(p) > 1 else np.zeros(5)
        acc = shard.merge_moments(acc, shard.local_moments(p.mean(axis=0), sem, len(p)))
    n, m, q = acc
    assert n == 37
    assert np.allclose(m, x.mean(axis=0), rtol=0, atol=1e-15)
    assert np.allclose(np.sqrt(q / n / n), np.sqrt(x.var(axis=0) / 37), rtol=1e-13, atol=0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, n_total, out_dir):
    import torch.distributed as dist
    from oracle import tebd
    import workloads

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    L = 4
    cfg = tebd.TrajectoryConfig(L, J=1.0, dt=0.05, chi_max=4, svd_cut=1e-12, gamma_loss=0.8,
                                occupation=workloads.occupation(L, "neel"), seed=11)
    off, n = shard.shard_range(n_total, rank, world)
    res = tebd.run_trajectories(cfg, 6, list(range(off, off + n)))
    dens = res["density"]
    mean = dens.mean(axis=0)
    sem = np.sqrt(dens.var(axis=0) / n) if n > 1 else np.zeros(L)
    m, s, ntot = shard.combine_mean_sem(mean, sem, n)
    np.savez(os.path.join(out_dir, "rank%d.npz" % rank), mean=m, sem=s, n=ntot,
             jumps=res["jumps"], density=dens, offset=off)
    dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_unsharded_ensemble(tmp_path):
    import torch.multiprocessing as mp
    from oracle import tebd
    import workloads

    n_total, world = 7, 2
    mp.start_processes(_rank_main, args=(world, _free_port(), n_total, str(tmp_path)),
                       nprocs=world, join=True, start_method="spawn")
    L = 4
    cfg = tebd.TrajectoryConfig(L, J=1.0, dt=0.05, chi_max=4, svd_cut=1e-12, gamma_loss=0.8,
                                occupation=workloads.occupation(L, "neel"), seed=11)
    whole = tebd.run_trajectories(cfg, 6, list(range(n_total)))
    ranks = [np.load(tmp_path / ("rank%d.npz" % r)) for r in range(world)]
    # each shard sampled the same trajectories (same jump records, same states)
    jumps = np.concatenate([r["jumps"] for r in ranks])
    dens = np.concatenate([r["density"] for r in ranks])
    assert np.array_equal(jumps, whole["jumps"])
    assert np.array_equal(dens, whole["density"])
    assert whole["jumps"].max() >= 0, "the case should contain jumps"
    mean, sem = tebd.ensemble_stats(whole["density"])
    for r in ranks:
        assert int(r["n"]) == n_total
        assert np.allclose(r["mean"], mean, rtol=0, atol=1e-14)
        assert np.allclose(r["sem"], sem, rtol=1e-12, atol=1e-15)
    assert np.array_equal(ranks[0]["mean"], ranks[1]["mean"])
