"""Multi-GPU runs are replicas (no collective on the data path): every rank
runs its own workload with its own seed; the only collective is the
max-over-ranks reduction of the timed region.  Checked with two gloo ranks
on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2005_01945_gb300 import synth
    local_ms = 100.0 * (rank + 1)                     # rank 1 is the slow one
    slowest = bench.max_over_ranks(local_ms, dist)
    rate = bench.whole_job_rate(39424, 5, world, slowest)
    seed = synth.MASTER_SEED + 1000 * rank            # the replica seed rule of bench.py
    a, _ = synth.int_pairs(4, 32, seed + 1, "add32")
    out.put((rank, slowest, rate, int(a[0])))
    dist.destroy_process_group()


def test_two_rank_replicas_max_reduction():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    assert res[0][1] == res[1][1] == 200.0                   # both see the slowest rank
    assert res[0][2] == res[1][2] == pytest.approx(39424 * 5 * 2 / 0.2)
    assert res[0][3] != res[1][3]                            # replicas draw their own inputs
