"""Sharding of the node-aware apply over several devices: whole simulated nodes
per device.

Every step of Algorithm NAPSpMV (Sec. 4) but one stays inside a node: the
on_node -> on_node and on_node -> off_node gathers (Eqs. IL2, IL0), the packing
of g_send and the off_node -> on_node forwarding (Eq. IL1) only touch the
processes of one node, and the three-block SpMV only the receiving process.
Only the inter-node messages of Eq. I cross nodes.  Giving device d a
contiguous block of simulated nodes therefore leaves one exchange per apply:
the messages whose sending node lives on another device than their receiving
node.  Messages between nodes of one device stay a local copy.

This module computes that exchange from the plan's inter-node message list and
carries it out over a torch.distributed process group (one rank per device),
point to point: each rank sends, per peer, the g_send segments of the messages
that peer receives, concatenated in g_send order, and scatters what it receives
into its own g_recv positions.  Layouts follow the plan: g_send holds the
messages in (sending process, receiving process) order, g_recv in (receiving
process, sending process) order (the library's NAPSPMV_LIST_INTER order).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def node_blocks(n_nodes: int, world: int):
    """First node of every rank's block, [world + 1]: ranks get n_nodes / world
    nodes, the first n_nodes mod world one more."""
    q, rem = divmod(n_nodes, world)
    starts = [0]
    for r in range(world):
        starts.append(starts[-1] + q + (1 if r < rem else 0))
    return np.array(starts, np.int64)


@dataclass
class RankExchange:
    """One rank's part of the exchange.  Element ranges are into the global
    g_send / g_recv; the rank holds g_send[gs_lo:gs_hi] and g_recv[gr_lo:gr_hi]."""
    rank: int
    gs_lo: int = 0
    gs_hi: int = 0
    gr_lo: int = 0
    gr_hi: int = 0
    send: dict = field(default_factory=dict)   # peer -> list of (gs_lo, gs_hi, gr_lo)
    recv: dict = field(default_factory=dict)   # peer -> list of (gs_lo, gs_hi, gr_lo)
    local: list = field(default_factory=list)  # list of (gs_lo, gs_hi, gr_lo)

    def count(self, table, peer):
        return int(sum(b - a for a, b, _ in table.get(peer, [])))


def exchange_plan(src, dst, ptr, ppn, n_nodes, world):
    """The exchange of every rank.  src, dst: sending / receiving process of
    each inter-node message in g_send order; ptr: their offsets ([m + 1])."""
    src = np.asarray(src, np.int64)
    dst = np.asarray(dst, np.int64)
    ptr = np.asarray(ptr, np.int64)
    m = len(src)
    starts = node_blocks(n_nodes, world)
    owner = lambda node: int(np.searchsorted(starts, node, side="right") - 1)  # noqa: E731
    lens = ptr[1:] - ptr[:-1]
    # g_recv offsets: messages in (dst, src) order
    rorder = sorted(range(m), key=lambda k: (dst[k], src[k]))
    gr_off = np.zeros(m, np.int64)
    o = 0
    for k in rorder:
        gr_off[k] = o
        o += lens[k]
    out = [RankExchange(r) for r in range(world)]
    for r in range(world):
        lo_node, hi_node = starts[r], starts[r + 1]
        mine_s = [k for k in range(m) if lo_node <= src[k] // ppn < hi_node]
        mine_r = [k for k in range(m) if lo_node <= dst[k] // ppn < hi_node]
        X = out[r]
        if mine_s:
            X.gs_lo, X.gs_hi = int(ptr[mine_s[0]]), int(ptr[mine_s[-1] + 1])
        else:
            first = next((k for k in range(m) if src[k] // ppn >= hi_node), m)
            X.gs_lo = X.gs_hi = int(ptr[first])
        if mine_r:
            X.gr_lo = int(min(gr_off[k] for k in mine_r))
            X.gr_hi = int(max(gr_off[k] + lens[k] for k in mine_r))
        else:
            X.gr_lo = X.gr_hi = int(next((gr_off[k] for k in rorder if dst[k] // ppn >= hi_node), o))
    for k in range(m):
        a, b = owner(src[k] // ppn), owner(dst[k] // ppn)
        seg = (int(ptr[k]), int(ptr[k + 1]), int(gr_off[k]))
        if a == b:
            out[a].local.append(seg)
        else:
            out[a].send.setdefault(b, []).append(seg)
            out[b].recv.setdefault(a, []).append(seg)
    return out


def exchange(gsend_local, grecv_local, X: RankExchange, group=None):
    """Carry out one rank's exchange: local messages are copied, remote ones
    sent and received point to point (every rank calls this once per apply).
    gsend_local / grecv_local: the rank's slices of g_send and g_recv
    (torch tensors on the device the process group's backend serves)."""
    import torch
    import torch.distributed as dist
    for a, b, g in X.local:
        grecv_local[g - X.gr_lo:g - X.gr_lo + (b - a)] = gsend_local[a - X.gs_lo:b - X.gs_lo]
    reqs, bufs = [], {}
    for peer in sorted(X.recv):
        bufs[peer] = torch.empty(X.count(X.recv, peer), dtype=grecv_local.dtype,
                                 device=grecv_local.device)
        reqs.append(dist.irecv(bufs[peer], src=peer, group=group))
    for peer in sorted(X.send):
        parts = [gsend_local[a - X.gs_lo:b - X.gs_lo] for a, b, _ in X.send[peer]]
        reqs.append(dist.isend(torch.cat(parts).contiguous(), dst=peer, group=group))
    for q in reqs:
        q.wait()
    for peer, buf in bufs.items():
        o = 0
        for a, b, g in X.recv[peer]:
            grecv_local[g - X.gr_lo:g - X.gr_lo + (b - a)] = buf[o:o + (b - a)]
            o += b - a
    return grecv_local
