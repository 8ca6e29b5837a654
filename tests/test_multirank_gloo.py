"""Multi-process path of bench.py on CPU (gloo, world size 2): every rank replays its own
block of traces (weak scaling, no data-path collective) and the elapsed time is the
maximum over ranks."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    w, r, _ = bench.dist_setup()
    assert (w, r) == (world, rank)
    ts = bench.rank_traces(rank, n_traces=8, n=1000)
    bench.barrier(w)
    elapsed = bench.max_over_ranks(w, 1.0 + rank, torch.device("cpu"))
    first = ts.trace(0)[:16].tolist()
    q.put((rank, elapsed, first, ts.n_samples))
    dist.destroy_process_group()


def test_two_ranks_shard_traces_and_take_max_time():
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    # max over ranks seen by both
    assert out[0][1] == out[1][1] == 2.0
    # disjoint trace blocks (different seeds per trace id), equal per-rank work
    assert out[0][2] != out[1][2]
    assert out[0][3] == out[1][3] == 8 * 1000


def test_rank_blocks_match_single_process_generation():
    sys.path.insert(0, ROOT)
    import bench
    import tracegen
    both = tracegen.batched(n_traces=16, n=500)
    r1 = bench.rank_traces(1, n_traces=8, n=500)
    assert np.array_equal(r1.trace(0), both.trace(8))
