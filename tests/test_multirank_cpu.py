"""The N > 1 path of the benchmark is N independent replicas (the node-aware
SpMV is simulated on one GPU; nothing is exchanged between GPUs).  Its host
logic, max-over-ranks time and the whole-job value, runs here on world_size-2
gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 + 5.0 * rank  # rank 1 is the slowest
    dist.barrier()
    mx = bench.max_over_ranks(ms)
    ws, r, local = bench.dist_env()
    val = bench.job_value(ws, 1e9, 100, 4, mx)
    q.put((rank, mx, ws, r, val))
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_job_value():
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
    for rank, mx, ws, r, val in out:
        assert mx == 15.0 and ws == 2 and r == rank
        # 2 replicas x 1e9 B x 100 applies x 4 steps over the slowest 15 ms
        assert val == pytest.approx(2 * 1e9 * 400 / 0.015 / 1e9)


def test_single_process_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_value(1, 2e9, 10, 5, 100.0) == pytest.approx(1000.0)
