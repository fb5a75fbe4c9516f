"""The N>1 bench path on CPU: world_size-2 gloo ranks.  Events are independent, so ranks shard the
batch by seed with no data exchange; the only collectives are the timing aggregation (max of the
step time, sum of the clusters) and barriers.  The reference arm runs on rank 0 alone."""
import hashlib
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_1712_09434_gb300 import synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seed0 = bench.shard_seed0(rank)
        cfgs = synth.batch_configs(n_events=2, seed0=seed0)
        # a rank's own events, small enough to generate here (2 events, the bench's recipe)
        evs = [synth.make_event(c) for c in cfgs]
        units = sum(e.n_clusters for e in evs)
        digest = hashlib.sha1(b"".join(e.pad_fp.tobytes() + e.time_fp.tobytes() for e in evs)).hexdigest()
        ms_local = 10.0 + 5.0 * rank
        ms, total = bench.aggregate(ms_local, units, world)
        got = [None] * world
        dist.all_gather_object(got, (rank, seed0, units, digest, ms, total))
        if rank == 0:
            q.put(got)
    finally:
        dist.destroy_process_group()


def test_two_rank_weak_sharding_and_aggregation():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(got)
    seeds = [g[1] for g in got]
    assert seeds == [bench.shard_seed0(0), bench.shard_seed0(1)] and seeds[0] != seeds[1]
    assert got[0][3] != got[1][3]                         # different events on the two ranks
    total = sum(g[2] for g in got)
    for g in got:
        assert g[4] == 15.0                                # max over ranks of 10 and 15 ms
        assert g[5] == total                               # clusters summed over ranks


def test_single_rank_aggregation_needs_no_group():
    assert bench.aggregate(3.5, 7, 1) == (3.5, 7)


def test_shard_seeds_do_not_overlap():
    # each rank's 64 events take seeds seed0 .. seed0+63; ranks are 1000 seeds apart
    spans = [set(range(bench.shard_seed0(r), bench.shard_seed0(r) + 64)) for r in range(8)]
    for i in range(8):
        for j in range(i + 1, 8):
            assert not spans[i] & spans[j]


def test_reference_arm_runs_on_rank_zero_only(capsys):
    class A:
        events, steps, warmup = 1, 1, 0
    bench.run_reference(A, rank=1, world=2)
    assert capsys.readouterr().out == ""
