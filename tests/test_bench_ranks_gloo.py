"""bench.py's multi-rank path on CPU (gloo, world size 2): the reference arm
under torchrun prints one JSON line from rank 0 only; the timing helpers take
the max and the sum over ranks; every rank gets its own ligands with the same
window layout (weak scaling, no data-path collective)."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_reference_arm_under_torchrun_prints_once():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "tiny",
           "--steps", "1", "--warmup", "1", "--gpus", "2"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [x for x in out.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1, out.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    ws, r, local = bench.dist_setup()
    bench.barrier(ws)
    t = bench.allmax(ws, 0.1 * (rank + 1))
    n = bench.allsum(ws, 10.0 + rank)
    w = bench.make_workload("batch", r)
    lig = w.systems[0]
    out[rank] = (ws, r, t, n, w.n_replicas, lig.pos[lig.is_ligand.astype(bool)][:3].tolist())
    import torch.distributed as dist
    dist.destroy_process_group()


def test_rank_helpers_and_per_rank_workloads():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(300)
        assert p.exitcode == 0
    (ws0, r0, t0, n0, nr0, x0), (ws1, r1, t1, n1, nr1, x1) = out[0], out[1]
    assert (ws0, r0, ws1, r1) == (2, 0, 2, 1)
    assert t0 == t1 == pytest.approx(0.2)          # max over ranks
    assert n0 == n1 == pytest.approx(21.0)         # sum over ranks
    assert nr0 == nr1 == 1152                      # same window layout on every rank
    assert not np.allclose(x0, x1)                 # but each rank's own ligands
