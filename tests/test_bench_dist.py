"""The benchmark's multi-process plumbing on CPU (gloo, world size 2): the
barrier, the max over ranks that sets the whole-job time, the whole-job value
(snapshots of all replicas over the slowest rank's time), and that only rank 0
runs the reference arm.  No GPU and no data-path collective are involved."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    d = bench.Dist(world)
    assert d.pg is not None and d.pg.get_backend() == "gloo"
    d.barrier()
    ms = 10.0 + 5.0 * rank                      # per-rank step time
    ms_max = d.max(ms)
    value = d.world * bench.N_SNAP / (ms_max * 1e-3)
    ref = bench.run_reference(None, d) if rank != 0 else "rank0"
    d.barrier()
    d.close()
    out[rank] = (ms_max, value, ref)


def test_two_gloo_ranks_max_and_whole_job_value():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    import bench
    for r in range(2):
        ms_max, value, ref = out[r]
        assert ms_max == 15.0                   # the slowest rank sets the time
        assert value == pytest.approx(2 * bench.N_SNAP / 15e-3)
    assert out[1][2] is None                    # only rank 0 runs the reference arm
