"""The multi-process host logic of bench.py on CPU (gloo, world size 2): the
path does not shard, so N GPUs run N replicas with event ids offset by rank;
the job's time is the slowest replica's and its value counts every rank's
photons; the reference arm runs on rank 0 only."""
import argparse
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        assert bench.dist_env() == (rank, world, rank)
        b = bench.replica_batch(rank, n_events=20)
        ids = torch.from_numpy(b.event_ids.astype(np.int64))
        got = [torch.zeros_like(ids) for _ in range(world)]
        dist.all_gather(got, ids)
        all_ids = torch.cat(got).numpy()
        # same work per rank (weak scaling), distinct events: every replica draws its own photons
        photons = torch.tensor([b.total_photons()], dtype=torch.int64)
        ph = [torch.zeros_like(photons) for _ in range(world)]
        dist.all_gather(ph, photons)
        slowest = bench.max_over_ranks(100.0 + 7.0 * rank, "cpu")
        value = bench.aggregate_value(world, b.total_photons(), 3, slowest)
        # the reference arm: only rank 0 runs the oracle
        args = argparse.Namespace(events=2, cpu_sample_photons=1000, warmup=0, steps=1, gpus=world)
        ref_ran = rank == 0
        if rank != 0:
            assert bench.run_reference(args) is None
        q.put((rank, len(np.unique(all_ids)) == len(all_ids), len({int(p) for p in ph}) == 1,
               slowest, value, b.total_photons(), ref_ran))
    finally:
        dist.destroy_process_group()


def test_replicas_two_ranks_on_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for rank, distinct, same_work, slowest, value, photons, _ in out:
        assert distinct and same_work
        assert slowest == pytest.approx(107.0)                # the slowest rank's time
        assert value == pytest.approx(2 * photons * 3 / 0.107)
