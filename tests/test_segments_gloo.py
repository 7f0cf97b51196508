"""Multi-rank layout on CPU (gloo, world size 2): each rank owns a contiguous,
overlapping window segment (the paper's no-communication design), runs its
windows independently, and only the timing aggregation (max over ranks) and a
barrier cross ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2603_22274_gb300.segments import rank_windows, segment_windows


def test_paper_example_and_cover():
    # windows 1..15 on two GPUs: [1, 8] and [8, 15] (1-based)
    assert segment_windows(15, 2) == [(0, 7), (7, 14)]
    for K in (2, 12, 42, 73, 80):
        for n in (1, 2, 3, 4, 8):
            segs = segment_windows(K, n)
            covered = set()
            for a, b in segs:
                assert 0 <= a <= b < K
                covered |= set(range(a, b + 1))
            assert covered == set(range(K))
            for (a0, b0), (a1, b1) in zip(segs, segs[1:]):
                assert a1 == b0 or (a1, b1) == (a0, b0)   # shared boundary window


def _worker(rank, world, port, K, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = rank_windows(K, world, rank)
    # each rank's "work": a quantity computed from its own windows only
    local = torch.tensor([float(sum(mine)), float(len(mine)), 0.1 * (rank + 1)], dtype=torch.float64)
    dist.barrier()
    t = local[2:3].clone()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)      # the bench's max-over-ranks timing
    n = local[1:2].clone()
    dist.all_reduce(n, op=dist.ReduceOp.SUM)      # windows processed by all ranks
    out[rank] = (mine, float(t.item()), float(n.item()))
    dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_two_rank_segments_gloo():
    K = 42
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, K, out)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    w0, t0, n0 = out[0]
    w1, t1, n1 = out[1]
    assert w0[-1] == w1[0]                      # duplicated boundary window
    assert set(w0) | set(w1) == set(range(K))
    assert t0 == t1 == pytest.approx(0.2)       # max over ranks
    assert n0 == n1 == len(w0) + len(w1)
