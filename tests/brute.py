"""Brute-force evaluation of the paper's set definitions with Python sets.

Used by the tests to pin the C oracle on tiny inputs (N <= ~48): every set is
built by enumerating all ranks, nodes and stored entries, exactly as the
equations of Secs. 2, 2.1, 4.1 and 4.2 of Bienz, Gropp, Olson (arXiv 1612.08060)
state them, with the same readings of the open points as the oracle (listed in the
oracle's header).  Nothing here is fast or clever on purpose.
"""
from __future__ import annotations


def partition(n, n_p, strided=False):
    """R(r) as explicit sets; the first n mod n_p ranks get one more row.
    strided: R(r) = {i : i mod n_p = r} (the strided partition of Sec. 5)."""
    if strided:
        return [set(range(r, n, n_p)) for r in range(n_p)]
    q, rem = divmod(n, n_p)
    R, start = [], 0
    for r in range(n_p):
        size = q + (1 if r < rem else 0)
        R.append(set(range(start, start + size)))
        start += size
    return R


def _groups(P, K, from_top):
    """Node splitting: the processes (local ids) of a node with P processes given
    to its K partners in order, floor(P/K) + (k < P mod K) each; counted up from
    process 0, or down from process P-1 (from_top)."""
    out, lo, hi = [], 0, P
    for k in range(K):
        size = P // K + (1 if k < P % K else 0)
        if from_top:
            out.append(list(range(hi - size, hi)))
            hi -= size
        else:
            out.append(list(range(lo, lo + size)))
            lo += size
    return out


def brute_plan(n, rows, n_p, ppn, map_text=False, strided=False, majority=False, split=False):
    """rows[i] = set of stored columns of row i.  Returns a dict of dicts:
    STD/J0/J1/J2/INTER: {(src, dst): sorted tuple}; NODE: {(n, m): tuple};
    BLL/BNL/LBUF: {rank: tuple}; T, U: {rank: set of nodes}; G: {rank: set};
    split: list of (on_process, on_node, off_node) counts per row."""
    R = partition(n, n_p, strided)
    nn = (n_p + ppn - 1) // ppn
    node_ranks = [[r for r in range(n_p) if r // ppn == x] for x in range(nn)]
    node_rows = [set().union(*(R[r] for r in node_ranks[x])) for x in range(nn)]
    A = {(i, j) for i in range(n) for j in rows[i]}

    def uses(I_rows, J_cols):
        return {(i, j) for (i, j) in A if i in I_rows and j in J_cols}

    out = {}
    # Eqs. P and D
    STD = {}
    for r in range(n_p):
        for t in range(n_p):
            if r == t:
                continue
            D = {j for (i, j) in uses(R[t], R[r])}
            if D:
                STD[(r, t)] = tuple(sorted(D))
    out["STD"] = STD
    # Eqs. N and E
    NODE = {}
    for a in range(nn):
        for b in range(nn):
            if a == b:
                continue
            E = {j for (i, j) in uses(node_rows[b], node_rows[a])}
            if E:
                NODE[(a, b)] = tuple(sorted(E))
    out["NODE"] = NODE
    # T and U: the mapping rule (largest |E| first on the sending side; on the
    # receiving side ascending |E| from the last process, as the tables show)
    T = {r: set() for r in range(n_p)}
    U = {r: set() for r in range(n_p)}
    if majority:
        # the alternative named after Eq. U: m maps to the process of a that
        # stores the most of E(a, m); on the receiving side a maps to the
        # process of m whose rows use the most of E(a, m); ties: lowest process
        for (a, m), E in NODE.items():
            own = [len(set(E) & R[r]) for r in node_ranks[a]]
            T[node_ranks[a][own.index(max(own))]].add(m)
            use = [len(set(E) & {j for (i, j) in A if i in R[q]}) for q in node_ranks[m]]
            U[node_ranks[m][use.index(max(use))]].add(a)
    for a in ([] if majority else range(nn)):
        P = len(node_ranks[a])
        sends = sorted([m for (x, m) in NODE if x == a], key=lambda m: (-len(NODE[(a, m)]), m))
        for k, m in enumerate(sends):
            T[node_ranks[a][k % P]].add(m)
        recvs = [x for (x, m) in NODE if m == a]
        if map_text:
            recvs.sort(key=lambda x: (-len(NODE[(x, a)]), x))
        else:
            recvs.sort(key=lambda x: (len(NODE[(x, a)]), x))
        for k, x in enumerate(recvs):
            U[node_ranks[a][P - 1 - (k % P)]].add(x)
    # Eq. G and Eq. I
    G = {r: set() for r in range(n_p)}
    INTER = {}
    if split:
        # the text after Eq. U: a node with fewer partners than processes maps
        # each partner to a group of its processes; E(a, m) is cut into
        # max(|S|, |R|) contiguous pieces, piece i from S[i mod |S|] to
        # R[i mod |R|]
        T = {r: set() for r in range(n_p)}
        U = {r: set() for r in range(n_p)}
        sgrp, rgrp = {}, {}
        for a in range(nn):
            P = len(node_ranks[a])
            sends = sorted([m for (x, m) in NODE if x == a],
                           key=lambda m: (-len(NODE[(a, m)]), m))
            if len(sends) < P:
                for m, g in zip(sends, _groups(P, len(sends), False)):
                    sgrp[(a, m)] = [node_ranks[a][p] for p in g]
            else:
                for k, m in enumerate(sends):
                    sgrp[(a, m)] = [node_ranks[a][k % P]]
            recvs = [x for (x, m) in NODE if m == a]
            if map_text:
                recvs.sort(key=lambda x: (-len(NODE[(x, a)]), x))
            else:
                recvs.sort(key=lambda x: (len(NODE[(x, a)]), x))
            if len(recvs) < P:
                for x, g in zip(recvs, _groups(P, len(recvs), True)):
                    rgrp[(x, a)] = [node_ranks[a][p] for p in g]
            else:
                for k, x in enumerate(recvs):
                    rgrp[(x, a)] = [node_ranks[a][P - 1 - (k % P)]]
        for (x, m), E in NODE.items():
            S, Rg = sgrp[(x, m)], rgrp[(x, m)]
            for r in S:
                T[r].add(m)
            for q in Rg:
                U[q].add(x)
            c, e = max(len(S), len(Rg)), len(E)
            for i in range(c):
                piece = E[i * e // c:(i + 1) * e // c]
                if piece:
                    G[S[i % len(S)]].add(Rg[i % len(Rg)])
                    INTER[(S[i % len(S)], Rg[i % len(Rg)])] = tuple(piece)
    else:
        for r in range(n_p):
            for q in range(n_p):
                m, x = q // ppn, r // ppn
                if m in T[r] and x in U[q]:
                    G[r].add(q)
                    INTER[(r, q)] = NODE[(x, m)]
    out["T"], out["U"] = T, U
    out["G"], out["INTER"] = G, INTER
    # Eq. IL0: on_node -> off_node
    J0 = {}
    for s in range(n_p):
        sent = set()
        for q in G[s]:
            sent |= set(INTER[(s, q)])
        for p in node_ranks[s // ppn]:
            if p == s:
                continue
            J = {j for j in sent if j in R[p]}
            if J:
                J0[(p, s)] = tuple(sorted(J))
    out["J0"] = J0
    # Eq. IL1: off_node -> on_node
    J1 = {}
    for q in range(n_p):
        recv = set()
        for (r, d), idx in INTER.items():
            if d == q:
                recv |= set(idx)
        for s in node_ranks[q // ppn]:
            if s == q:
                continue
            J = {j for (i, j) in A if i in R[s] and j in recv}
            if J:
                J1[(q, s)] = tuple(sorted(J))
    out["J1"] = J1
    # Eq. IL2: on_node -> on_node
    J2 = {}
    for p in range(n_p):
        for s in node_ranks[p // ppn]:
            if s == p:
                continue
            J = {j for (i, j) in uses(R[s], R[p])}
            if J:
                J2[(p, s)] = tuple(sorted(J))
    out["J2"] = J2
    # receive layouts of each rank and the aggregator buffers
    BLL, BNL, LBUF = {}, {}, {}
    for t in range(n_p):
        own_node = node_rows[t // ppn]
        on = {j for (i, j) in A if i in R[t] and j in own_node and j not in R[t]}
        off = {j for (i, j) in A if i in R[t] and j not in own_node}
        if on:
            BLL[t] = tuple(sorted(on))
        if off:
            BNL[t] = tuple(sorted(off))
        lb = set()
        for (p, s), idx in J0.items():
            if s == t:
                lb |= set(idx)
        if lb:
            LBUF[t] = tuple(sorted(lb))
    out["BLL"], out["BNL"], out["LBUF"] = BLL, BNL, LBUF
    split = []
    for i in range(n):
        t = next(r for r in range(n_p) if i in R[r])
        c = [0, 0, 0]
        for j in rows[i]:
            if j in R[t]:
                c[0] += 1
            elif j in node_rows[t // ppn]:
                c[1] += 1
            else:
                c[2] += 1
        split.append(tuple(c))
    out["split"] = split
    return out
