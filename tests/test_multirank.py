"""Multi-process host logic of the benchmark (replicas, no collective in the data path), run as two
gloo ranks on the CPU: the whole-job value is the units of all ranks over the slowest rank's time,
the barrier joins both ranks, and only rank 0 of the reference arm does any work."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, ws: int, port: int, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import bench
        assert bench._dist() == (ws, rank, rank)
        value = bench.whole_job_value(1000.0, 4, 1.0 + rank, ws)  # rank r took 1 + r seconds
        slowest = bench._max_over_ranks(1.0 + rank, ws)
        bench._barrier(ws)

        class Args:
            workload, steps, warmup, gpus = "pp_500", 1, 0, ws
        ref = bench.run_reference(Args, ws, rank) if rank == 1 else None  # rank 1: no work, no output
        q.put((rank, value, slowest, ref))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_whole_job_value():
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, slowest, ref in out:
        assert slowest == 2.0
        assert value == pytest.approx(1000.0 * 2 * 4 / 2.0)
        assert ref is None
