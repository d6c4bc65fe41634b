"""The multi-process path of bench.py on CPU (gloo, world size 2): process-group
set-up from the torchrun environment, the barrier, and the max-over-ranks
reduction of the per-rank times.  By default the benchmark runs independent
replicas (one problem per GPU, no data-path collective); its sharded mode's
collectives (halo exchange, all-to-all of the spectrum, all-reduce of the
residual norm) are tested in test_shard_exchange.py."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, q):
    os.environ.update(WORLD_SIZE="2", RANK=str(rank), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), PD_BENCH_GLOO="1")
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    ws, r, local = bench.dist_setup()
    bench.barrier(ws)
    ms = bench.max_over_ranks(ws, 1.5 + rank, "cpu")
    bench.barrier(ws)
    q.put((r, local, ws, ms))
    dist.destroy_process_group()


def test_two_rank_barrier_and_max_over_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    assert [o[0] for o in out] == [0, 1]
    assert all(o[2] == 2 for o in out)
    assert all(o[3] == 2.5 for o in out)     # the slowest rank's time on every rank
