"""Sharding of the node-aware apply over several devices (whole simulated nodes
per device, one exchange of the inter-node messages per apply), run as
world_size-2 and -3 gloo process groups on the CPU: every rank holds only its
nodes' part of g_send, filled from v with the oracle's inter-node message list;
after the exchange its part of g_recv must hold exactly what the oracle's plan
delivers to its nodes (each message's values, in the (receiver, sender)
layout).  Also: the exchange plan's bookkeeping against the message list."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle as O
from paper_1612_08060_gb300 import inputs as I
from paper_1612_08060_gb300 import shard

CASES = [("poisson3d", 16, 32, 4), ("random", 300, 24, 3), ("banded", 2000, 16, 2)]


def _matrix(kind, n):
    if kind == "poisson3d":
        return I.poisson3d(n)
    if kind == "random":
        return I.random_pattern(n, 0.03, 11)
    return I.banded_random(n, 12)


def _expected_grecv(src, dst, ptr, idx, v):
    order = sorted(range(len(src)), key=lambda k: (dst[k], src[k]))
    return np.concatenate([v[idx[ptr[k]:ptr[k + 1]]] for k in order]) if order else np.zeros(0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, case, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    kind, n, n_p, ppn = case
    A = _matrix(kind, n)
    src, dst, ptr, idx = O.OraclePlan(A.row_ptr, A.col, n_p, ppn).list(O.INTER)
    v = I.vector(A.n, 7)
    n_nodes = -(-n_p // ppn)
    X = shard.exchange_plan(src, dst, ptr, ppn, n_nodes, world)[rank]
    gsend = torch.from_numpy(v[idx[X.gs_lo:X.gs_hi]].copy())
    grecv = torch.full((X.gr_hi - X.gr_lo,), float("nan"), dtype=torch.float64)
    shard.exchange(gsend, grecv, X)
    want = _expected_grecv(src, dst, ptr, idx, v)[X.gr_lo:X.gr_hi]
    q.put((rank, bool(np.array_equal(grecv.numpy(), want)), len(X.send), len(X.recv)))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_sharded_exchange_matches_oracle(case, world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, case, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert all(ok for _, ok, _, _ in out), out
    assert any(ns > 0 for _, _, ns, _ in out)  # the exchange crosses ranks


@pytest.mark.parametrize("world", [1, 2, 4, 7])
def test_exchange_plan_covers_every_message_once(world):
    """Every message is either local to one rank or sent by its sender's rank
    and received by its receiver's rank; spans are contiguous and tile g_send
    and g_recv; nodes are dealt in contiguous blocks."""
    A = I.poisson2d(40)
    n_p, ppn = 40, 3
    src, dst, ptr, idx = O.OraclePlan(A.row_ptr, A.col, n_p, ppn).list(O.INTER)
    n_nodes = -(-n_p // ppn)
    starts = shard.node_blocks(n_nodes, world)
    assert starts[0] == 0 and starts[-1] == n_nodes and np.all(np.diff(starts) >= n_nodes // world)
    plan = shard.exchange_plan(src, dst, ptr, ppn, n_nodes, world)
    seen = {}
    for X in plan:
        for a, b, g in X.local:
            seen[a] = seen.get(a, 0) + 1
        for peer, segs in X.send.items():
            assert segs == plan[peer].recv[X.rank]
            for a, b, g in segs:
                seen[a] = seen.get(a, 0) + 1
    starts_gs = [int(ptr[k]) for k in range(len(src)) if ptr[k + 1] > ptr[k]]
    assert sorted(seen) == starts_gs and set(seen.values()) == {1}
    assert [X.gs_lo for X in plan] + [plan[-1].gs_hi] == sorted([X.gs_lo for X in plan] + [plan[-1].gs_hi])
    assert sum(X.gs_hi - X.gs_lo for X in plan) == ptr[-1] == sum(X.gr_hi - X.gr_lo for X in plan)
