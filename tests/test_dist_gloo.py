"""The multi-GPU ensemble's host logic with two gloo ranks on the CPU.

Ranks solve disjoint blocks of sample ids with no data exchange; the job's
throughput is all ranks' work over the slowest rank's time.  Checked here:
the blocks are disjoint and cover the ensemble, a sample's random cloud does
not depend on which rank (or how many ranks) draws it, and the MAX/SUM
aggregation and throughput formula used by the benchmark."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import workloads as W  # noqa: E402
from paper_1705_04374_gb300 import sharding  # noqa: E402

PER_RANK = 5
WORLD = 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        from paper_1705_04374_gb300 import api
        ids = sharding.rank_sample_ids(rank, PER_RANK)
        cloud = W.cfg2("fp32").cloud
        clouds = np.stack([api.sample_cloud(cloud, W.BASE_SEED, sid) for sid in ids])
        gathered = [None] * WORLD
        dist.all_gather_object(gathered, (ids, clouds))
        # rank r took (r + 1) s and did 10 (r + 1) units of work
        elapsed, work = sharding.aggregate(1.0 + rank, 10.0 * (rank + 1), WORLD)
        if rank == 0:
            np.save(os.path.join(out_dir, "ids.npy"), np.array([g[0] for g in gathered]))
            np.save(os.path.join(out_dir, "clouds.npy"), np.stack([g[1] for g in gathered]))
            np.save(os.path.join(out_dir, "agg.npy"), np.array([elapsed, work, sharding.job_rate(elapsed, work)]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_partition_and_aggregate(tmp_path):
    mp.start_processes(_rank_main, args=(_free_port(), str(tmp_path)), nprocs=WORLD, start_method="spawn")
    ids = np.load(tmp_path / "ids.npy")
    flat = ids.ravel().tolist()
    assert len(set(flat)) == len(flat) == WORLD * PER_RANK          # disjoint
    assert sorted(flat) == list(range(WORLD * PER_RANK))            # covering
    # a sample's cloud is the same whichever rank draws it
    from paper_1705_04374_gb300 import api
    cloud = W.cfg2("fp32").cloud
    single = np.stack([api.sample_cloud(cloud, W.BASE_SEED, sid) for sid in range(WORLD * PER_RANK)])
    clouds = np.load(tmp_path / "clouds.npy").reshape(single.shape)
    assert np.array_equal(clouds, single)
    elapsed, work, rate = np.load(tmp_path / "agg.npy")
    assert elapsed == 2.0 and work == 30.0 and rate == 15.0


def test_single_rank_needs_no_process_group():
    assert sharding.aggregate(3.0, 7.0, 1) == (3.0, 7.0)
    assert sharding.rank_sample_ids(0, 3) == [0, 1, 2]
    assert sharding.rank_sample_ids(2, 3) == [6, 7, 8]
    with pytest.raises(ValueError):
        sharding.job_rate(0.0, 1.0)


def _estimator_rank(rank, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        pairs = W.toy_levels([301, 41, 9], 2, 0.5, 1.0, seed=23)
        local = [p[list(sharding.pair_shard(len(p), rank, WORLD))] for p in pairs]
        est = sharding.distributed_estimate(local, [1.0, 17.0, 272.0], WORLD)
        np.save(os.path.join(out_dir, f"est{rank}.npy"),
                np.concatenate([est["alpha"], est["sigma2"], est["cov"], est["sigma_tilde2"], [est["mean"], est["eps2"]]]))
        fit = sharding.distributed_estimate(local, [1.0, 17.0, 272.0], WORLD, fit=True)
        np.save(os.path.join(out_dir, f"fit{rank}.npy"),
                np.concatenate([fit["alpha"], fit["cov"], fit["sigma_tilde2"], fit["V_fit"], [fit["mean"], fit["eps2"]]]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_estimate_equals_single_process(tmp_path):
    """Each rank summarises its level-stratified share of the pairs; after one
    all-gather of the summaries both ranks hold the single-process estimate."""
    mp.start_processes(_estimator_rank, args=(_free_port(), str(tmp_path)), nprocs=WORLD, start_method="spawn")
    from paper_1705_04374_gb300 import api
    pairs = W.toy_levels([301, 41, 9], 2, 0.5, 1.0, seed=23)
    ref = api.estimate(pairs, [1.0, 17.0, 272.0])
    want = np.concatenate([ref["alpha"], ref["sigma2"], ref["cov"], ref["sigma_tilde2"], [ref["mean"], ref["eps2"]]])
    e0, e1 = np.load(tmp_path / "est0.npy"), np.load(tmp_path / "est1.npy")
    assert np.array_equal(e0, e1)                      # every rank holds the same numbers
    assert np.allclose(e0, want, rtol=1e-11, atol=1e-14)
    # step 3's variance fit from the combined summaries
    rf = api.estimate(pairs, [1.0, 17.0, 272.0], fit=True)
    want = np.concatenate([rf["alpha"], rf["cov"], rf["sigma_tilde2"], rf["V_fit"], [rf["mean"], rf["eps2"]]])
    f0, f1 = np.load(tmp_path / "fit0.npy"), np.load(tmp_path / "fit1.npy")
    assert np.array_equal(f0, f1)
    assert np.allclose(f0, want, rtol=1e-11, atol=1e-14)
    shards = [set(sharding.pair_shard(41, r, WORLD)) for r in range(WORLD)]
    assert not (shards[0] & shards[1]) and shards[0] | shards[1] == set(range(41))
