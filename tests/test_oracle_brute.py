"""The CPU oracle's plans against a literal Python evaluation of the set
definitions (tests/brute.py) on tiny random patterns, for many (n_p, ppn),
including uneven partitions and a partial last node; and its products against
dense numpy products."""
import itertools

import numpy as np
import pytest

import oracle as O
from brute import brute_plan
from paper_1612_08060_gb300.inputs import random_pattern

LISTS = [("STD", O.STD), ("NODE", O.NODE), ("INTER", O.INTER), ("J0", O.J0), ("J1", O.J1),
         ("J2", O.J2)]
LAYOUTS = [("BLL", O.BLL), ("BNL", O.BNL), ("LBUF", O.LBUF)]

CASES = []
for seed, (n, dens) in enumerate([(7, 0.3), (12, 0.25), (17, 0.2), (24, 0.15), (31, 0.1),
                                   (40, 0.08), (48, 0.3)]):
    for n_p, ppn in [(1, 1), (2, 1), (3, 2), (5, 2), (6, 3), (7, 4), (n, 1), (n, 4),
                     (min(n, 9), 9), (min(n, 11), 3), (min(n, 16), 5)]:
        if n_p <= n:
            CASES.append((n, dens, seed, n_p, ppn))


def _rows(A):
    return [set(A.col[A.row_ptr[i]:A.row_ptr[i + 1]].tolist()) for i in range(A.n)]


@pytest.mark.parametrize("n,dens,seed,n_p,ppn", CASES)
def test_plans_match_set_definitions(n, dens, seed, n_p, ppn):
    A = random_pattern(n, dens, seed)
    plan = O.OraclePlan(A.row_ptr, A.col, n_p, ppn)
    b = brute_plan(n, _rows(A), n_p, ppn)
    for name, kind in LISTS:
        assert plan.list_dict(kind) == b[name], name
    for name, kind in LAYOUTS:
        got = {s: idx for (s, d), idx in plan.list_dict(kind).items()}
        assert all(s == d for (s, d) in plan.list_dict(kind))
        assert got == b[name], name
    assert [tuple(r) for r in plan.split().tolist()] == b["split"]


@pytest.mark.parametrize("n_p,ppn", [(6, 2), (9, 4), (12, 5)])
def test_map_text_rule(n_p, ppn):
    A = random_pattern(36, 0.12, 77)
    plan = O.OraclePlan(A.row_ptr, A.col, n_p, ppn, flags=O.MAP_TEXT)
    b = brute_plan(36, _rows(A), n_p, ppn, map_text=True)
    assert plan.list_dict(O.INTER) == b["INTER"]
    assert plan.list_dict(O.J0) == b["J0"]
    assert plan.list_dict(O.J1) == b["J1"]


@pytest.mark.parametrize("n,dens,seed,n_p,ppn", CASES[::3])
def test_napspmv_and_spmv_equal_dense(n, dens, seed, n_p, ppn):
    A = random_pattern(n, dens, seed)
    v = np.random.default_rng(seed + 100).uniform(-1, 1, n)
    ref = A.to_dense() @ v
    scale = np.abs(A.to_dense()) @ np.abs(v)
    w1 = O.spmv(A.row_ptr, A.col, A.val, v)
    plan = O.OraclePlan(A.row_ptr, A.col, n_p, ppn)
    w2 = plan.napspmv(A.row_ptr, A.col, A.val, v)
    tol = 4 * np.finfo(float).eps * scale + 1e-300
    assert np.all(np.abs(w1 - ref) <= tol)
    assert np.all(np.abs(w2 - ref) <= tol)


def test_invariants_random():
    """E(n,m) is the union of D(r,t) over r on n, t on m; one inter-node message
    per node pair; node-aware inter-node counts never exceed the standard ones;
    every intra-node message stays on its node; nobody sends to itself."""
    for seed, (n, n_p, ppn) in enumerate([(40, 10, 3), (48, 16, 4), (45, 9, 2), (30, 30, 7)]):
        A = random_pattern(n, 0.15, 300 + seed)
        plan = O.OraclePlan(A.row_ptr, A.col, n_p, ppn)
        D = plan.list_dict(O.STD)
        E = plan.list_dict(O.NODE)
        U = {}
        for (r, t), idx in D.items():
            if r // ppn != t // ppn:
                U.setdefault((r // ppn, t // ppn), set()).update(idx)
        assert {k: tuple(sorted(v)) for k, v in U.items()} == E
        inter = plan.list_dict(O.INTER)
        assert len(inter) == len(E)
        assert sorted(inter.values()) == sorted(E.values())
        s = plan.stats()
        assert s["nap_inter_msgs"] <= s["std_inter_msgs"]
        assert s["nap_inter_vals"] <= s["std_inter_vals"]
        for kind in (O.J0, O.J1, O.J2):
            for (a, b) in plan.list_dict(kind):
                assert a != b and a // ppn == b // ppn
        for (a, b) in itertools.chain(D, inter):
            assert a != b


@pytest.mark.parametrize("n,dens,seed,n_p,ppn", CASES[::2])
def test_strided_plans_match_set_definitions(n, dens, seed, n_p, ppn):
    """The strided partition (row i on rank i mod n_p, Sec. 5): every list,
    layout and row split against the literal set evaluation."""
    A = random_pattern(n, dens, seed)
    plan = O.OraclePlan(A.row_ptr, A.col, n_p, ppn, flags=O.STRIDED)
    b = brute_plan(n, _rows(A), n_p, ppn, strided=True)
    for name, kind in LISTS:
        assert plan.list_dict(kind) == b[name], name
    for name, kind in LAYOUTS:
        got = {s: idx for (s, d), idx in plan.list_dict(kind).items()}
        assert got == b[name], name
    assert [tuple(r) for r in plan.split().tolist()] == b["split"]


@pytest.mark.parametrize("n,dens,seed,n_p,ppn", CASES[1::4])
def test_strided_napspmv_equals_dense(n, dens, seed, n_p, ppn):
    A = random_pattern(n, dens, seed)
    v = np.random.default_rng(seed + 200).uniform(-1, 1, n)
    ref = A.to_dense() @ v
    scale = np.abs(A.to_dense()) @ np.abs(v)
    plan = O.OraclePlan(A.row_ptr, A.col, n_p, ppn, flags=O.STRIDED)
    w = plan.napspmv(A.row_ptr, A.col, A.val, v)
    assert np.all(np.abs(w - ref) <= 4 * np.finfo(float).eps * scale + 1e-300)


@pytest.mark.parametrize("n_p,ppn,k", [(5, 2, 4), (8, 4, 3), (12, 3, 5), (3, 1, 7)])
def test_strided_tridiagonal_closed_form(n_p, ppn, k):
    """1D 3-point operator, n = k n_p.  Strided: row i (rank i mod n_p) needs
    i-1 from rank (t-1) mod n_p and i+1 from rank (t+1) mod n_p, so every rank
    receives two messages; |D((t-1) mod n_p, t)| = k, one less when that sender
    is rank n_p-1 (column n-1 is not needed to the left), and |D((t+1) mod
    n_p, t)| = k, one less when the sender is rank 0 (column 0 is not needed
    to the right): 2 n_p messages carrying 2n - 2 values.  Contiguous: only
    the 2 (n_p - 1) block boundaries communicate, one value each."""
    n = k * n_p
    rows = [[j for j in (i - 1, i, i + 1) if 0 <= j < n] for i in range(n)]
    rp = np.zeros(n + 1, np.int64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    col = np.array([j for r in rows for j in r], np.int32)
    D = O.OraclePlan(rp, col, n_p, ppn, flags=O.STRIDED).list_dict(O.STD)
    want = {}
    for t in range(n_p):
        left, right = (t - 1) % n_p, (t + 1) % n_p
        want[(left, t)] = k - (1 if left == n_p - 1 else 0)
        want[(right, t)] = k - (1 if right == 0 else 0)
    assert {key: len(v) for key, v in D.items()} == want
    assert sum(len(v) for v in D.values()) == 2 * n - 2
    Dc = O.OraclePlan(rp, col, n_p, ppn).list_dict(O.STD)
    assert len(Dc) == 2 * (n_p - 1) and all(len(v) == 1 for v in Dc.values())


@pytest.mark.parametrize("n,dens,seed,n_p,ppn", CASES[::3])
@pytest.mark.parametrize("strided", [False, True])
def test_majority_mapping_matches_set_definitions(n, dens, seed, n_p, ppn, strided):
    """The majority mapping (node m to the process storing most of E(n,m), and
    the receiving process whose rows use most of it), with both partitions."""
    A = random_pattern(n, dens, seed)
    flags = O.MAP_MAJORITY | (O.STRIDED if strided else 0)
    plan = O.OraclePlan(A.row_ptr, A.col, n_p, ppn, flags=flags)
    b = brute_plan(n, _rows(A), n_p, ppn, strided=strided, majority=True)
    for name, kind in LISTS:
        assert plan.list_dict(kind) == b[name], name
    for name, kind in LAYOUTS:
        got = {s: idx for (s, d), idx in plan.list_dict(kind).items()}
        assert got == b[name], name
    v = np.random.default_rng(seed).uniform(-1, 1, n)
    w = plan.napspmv(A.row_ptr, A.col, A.val, v)
    ref = A.to_dense() @ v
    assert np.all(np.abs(w - ref) <= 4 * np.finfo(float).eps * (np.abs(A.to_dense()) @ np.abs(v)))


def test_majority_mapping_minimises_per_pair_forwarding():
    """Per node pair, the values of E(n,m) that its sending process does not own
    (they reach it through the on->off step) and the values its receiving
    process does not use (they only pass through it) are each the smallest
    over all processes of the node under the majority mapping: summed over the
    pairs, never more than under the table mapping.  Inter-node traffic is the
    same under both."""
    for seed, (n, n_p, ppn) in enumerate([(48, 12, 4), (60, 10, 5), (45, 9, 3), (80, 20, 4)]):
        A = random_pattern(n, 0.12, 500 + seed)
        rows = _rows(A)
        owner = {}
        for r in range(n_p):
            q, rem = divmod(n, n_p)
            start = r * q + min(r, rem)
            for i in range(start, start + q + (1 if r < rem else 0)):
                owner[i] = r

        def forwarded(flags):
            P = O.OraclePlan(A.row_ptr, A.col, n_p, ppn, flags=flags)
            E = P.list_dict(O.NODE)
            sp, rp = P.tu()
            keys = sorted(E)
            not_owned = not_used = 0
            for k, (a_, m) in enumerate(keys):
                s_ = a_ * ppn + int(sp[k])
                q_ = m * ppn + int(rp[k])
                used = {j for i in range(n) if owner[i] == q_ for j in rows[i]}
                not_owned += sum(1 for j in E[(a_, m)] if owner[j] != s_)
                not_used += sum(1 for j in E[(a_, m)] if j not in used)
            return not_owned, not_used, P.stats()["nap_inter_vals"]

        t_own, t_use, t_inter = forwarded(0)
        m_own, m_use, m_inter = forwarded(O.MAP_MAJORITY)
        assert m_own <= t_own and m_use <= t_use and m_inter == t_inter


def test_majority_with_map_text_rejected():
    A = random_pattern(12, 0.3, 1)
    with pytest.raises(ValueError):
        O.OraclePlan(A.row_ptr, A.col, 4, 2, flags=O.MAP_MAJORITY | O.MAP_TEXT)



# ------------------------------------------------------------------ node splitting
@pytest.mark.parametrize("n,dens,seed,n_p,ppn", CASES[::2])
@pytest.mark.parametrize("text", [False, True])
def test_split_matches_set_definitions(n, dens, seed, n_p, ppn, text):
    """Node splitting (the text after Eq. U): the oracle's plans against the
    literal set evaluation of the same reading."""
    A = random_pattern(n, dens, seed)
    flags = O.MAP_SPLIT | (O.MAP_TEXT if text else 0)
    plan = O.OraclePlan(A.row_ptr, A.col, n_p, ppn, flags=flags)
    b = brute_plan(n, _rows(A), n_p, ppn, map_text=text, split=True)
    for name, kind in LISTS:
        assert plan.list_dict(kind) == b[name], name
    for name, kind in LAYOUTS:
        got = {s: idx for (s, d), idx in plan.list_dict(kind).items()}
        assert got == b[name], name
    v = np.random.default_rng(seed).uniform(-1, 1, n)
    w = plan.napspmv(A.row_ptr, A.col, A.val, v)
    ref = A.to_dense() @ v
    assert np.all(np.abs(w - ref) <= 4 * np.finfo(float).eps * (np.abs(A.to_dense()) @ np.abs(v)))


def test_split_worked_example_by_hand():
    """The paper's worked example under node splitting, derived by hand from the
    reading: node 2 sends only to node 0 and node 1 receives only from node 0,
    so both are split over their two processes; the other pairs keep the
    tables' processes.  Seven inter-node messages of one value each, and every
    process sends and receives."""
    import golden_example as G
    ex = G.load()
    n = len(ex["rows"])
    rp = np.zeros(n + 1, np.int64)
    cols = []
    for i in range(n):
        c = sorted(ex["rows"][i])
        cols += c
        rp[i + 1] = rp[i] + len(c)
    plan = O.OraclePlan(rp, np.array(cols, np.int32), ex["np"], ex["ppn"], flags=O.MAP_SPLIT)
    # ranks: (p, n) = n * 2 + p
    assert plan.list_dict(O.INTER) == {(0, 2): (0,), (0, 3): (1,), (1, 5): (0,), (2, 1): (3,),
                                       (3, 4): (2,), (4, 0): (4,), (5, 0): (5,)}
    assert plan.list_dict(O.J0) == {(0, 1): (0,), (1, 0): (1,), (3, 2): (3,), (2, 3): (2,)}
    assert plan.list_dict(O.J1) == {(0, 1): (4,), (1, 0): (3,), (2, 3): (0,), (5, 4): (0,)}
    sp, rpn = plan.tu()  # node pairs (0,1) (0,2) (1,0) (1,2) (2,0): first process of each group
    assert list(sp) == [0, 1, 0, 1, 0] and list(rpn) == [0, 1, 1, 0, 0]
    st = plan.stats()
    assert st["nap_inter_msgs"] == 7 and st["nap_inter_vals"] == 7


def test_split_every_process_communicates():
    """2D 5-point 16 x 16, one grid line per process, four processes per node,
    four nodes: every node has fewer partner nodes (one or two) than processes,
    so under node splitting every process sends and receives at least one
    inter-node message; unsplit, only one process per node pair does.  The
    values moved between nodes are the same (a grid line per node pair), cut
    into pieces of 4 (a one-partner node, four ways) or 8 values (two ways)."""
    from paper_1612_08060_gb300.inputs import poisson2d
    A = poisson2d(16)
    split = O.OraclePlan(A.row_ptr, A.col, 16, 4, flags=O.MAP_SPLIT)
    plain = O.OraclePlan(A.row_ptr, A.col, 16, 4)
    I = split.list_dict(O.INTER)
    assert {s for (s, d) in I} == set(range(16)) == {d for (s, d) in I}
    assert len({s for (s, d) in plain.list_dict(O.INTER)}) == 6
    assert sorted({len(v) for v in I.values()}) == [4, 8]
    # pieces of a pair are contiguous and cover E(n, m) exactly
    E = split.list_dict(O.NODE)
    for (a, m), vals in E.items():
        got = sorted(j for (s, d), idx in I.items() if s // 4 == a and d // 4 == m for j in idx)
        assert got == list(vals)
    assert split.stats()["nap_inter_vals"] == plain.stats()["nap_inter_vals"] == 6 * 16


def test_split_with_majority_rejected():
    A = random_pattern(12, 0.3, 1)
    with pytest.raises(ValueError):
        O.OraclePlan(A.row_ptr, A.col, 4, 2, flags=O.MAP_MAJORITY | O.MAP_SPLIT)


def test_unknown_flag_bits_rejected():
    """A flag bit the oracle does not define is refused, not ignored."""
    A = random_pattern(12, 0.3, 1)
    for bad in (1, 32, 64, 1 << 20):
        with pytest.raises(Exception):
            O.OraclePlan(A.row_ptr, A.col, 4, 2, flags=bad)
