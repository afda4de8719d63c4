"""The N > 1 path of the benchmark on CPU: independent replicas over a world-size-2 gloo group
(rendezvous on 127.0.0.1); the job's step time is the slowest rank's, its throughput all ranks'
flops over that time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    assert bench.dist_env() == (ws, rank, rank)
    ms, value = bench.replicas_result(1.0 + rank, 2.0e9, ws, torch.device("cpu"))
    out.put((rank, ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_max_over_ranks_gloo():
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get() for _ in range(ws))
    for rank, ms, value in got:
        assert ms == 2.0                                  # the slowest rank's step
        assert value == pytest.approx(2 * 2.0e9 / 2.0e-3 / 1e9)  # both ranks' flops over it


def test_single_replica_needs_no_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.replicas_result(0.5, 1.0e9, 1, None)
    assert ms == 0.5 and value == pytest.approx(2000.0)
