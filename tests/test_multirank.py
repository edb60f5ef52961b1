"""The N > 1 host logic of bench.py on CPU ranks (gloo, world size 2, 127.0.0.1).

With several GPUs bench.py runs one independent replica of the workload per rank (the
step needs no data exchange between replicas); the only collectives are the barrier around
the timed region and the max over ranks of the elapsed time.  The reference arm runs on
rank 0 only; the other ranks exit without work.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        r, w, _ = bench.dist_env()
        bench.barrier(w)
        slowest = bench.max_over_ranks(10.0 + rank, w)

        class Args:
            steps, warmup, gpus, workload = 2, 1, world, "pulse1024_f32_varD_mms"

        line = bench.run_reference(Args()) if rank == 1 else "skipped"
        q.put((rank, r, w, slowest, line))
    finally:
        dist.destroy_process_group()


def test_two_cpu_ranks_max_timing_and_rank0_reference():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, r, w, slowest, line in results:
        assert r == rank and w == world
        assert slowest == 11.0  # every rank sees the slowest rank's time
    # rank 1 ran the reference arm's entry and returned without doing work
    assert results[1][4] is None
