"""The CPU oracle against the paper's worked example (Example "simple_matrix",
tables of Secs. 2.1, 4.1, 4.2), with the printed errata named cell by cell."""
import numpy as np
import pytest

import oracle as O
import golden_example
from brute import brute_plan
from paper_1612_08060_gb300.inputs import CSR


@pytest.fixture(scope="module")
def ex():
    g = golden_example.load()
    n = len(g["rows"])
    cols = [sorted(g["rows"][i]) for i in range(n)]
    row_ptr = np.zeros(n + 1, np.int64)
    row_ptr[1:] = np.cumsum([len(c) for c in cols])
    col = np.array([j for c in cols for j in c], np.int32)
    # values are not given; any distinct numbers do: A_ij = 1 + i + 10 j
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    val = 1.0 + rows + 10.0 * col
    plan = O.OraclePlan(row_ptr, col, g["np"], g["ppn"])
    return g, CSR(row_ptr, col, val), plan


def _by_src(d):
    out = {}
    for (s, t), idx in d.items():
        out.setdefault(s, set()).add(t)
    return out


def test_table_P_D(ex):
    g, A, plan = ex
    D = plan.list_dict(O.STD)
    assert D == {k: v for k, v in g["D"].items()}
    P = _by_src(D)
    for r in range(g["np"]):
        assert P.get(r, set()) == set(g["P"][r])


def test_table_N_E(ex):
    g, A, plan = ex
    E = plan.list_dict(O.NODE)
    assert E == g["E"]
    N = _by_src(E)
    for n in g["N"]:
        assert N[n] == set(g["N"][n])


def test_table_T_U_G(ex):
    g, A, plan = ex
    s, d, _, _ = plan.list(O.NODE)
    sp, rp = plan.tu()
    ppn = g["ppn"]
    T = {r: set() for r in range(g["np"])}
    U = {r: set() for r in range(g["np"])}
    for k in range(len(s)):
        T[int(s[k]) * ppn + int(sp[k])].add(int(d[k]))
        U[int(d[k]) * ppn + int(rp[k])].add(int(s[k]))
    for r in range(g["np"]):
        assert T[r] == set(g["T"][r]), r
        assert U[r] == set(g["U"][r]), r
    G = _by_src(plan.list_dict(O.INTER))
    for r in range(g["np"]):
        assert G.get(r, set()) == set(g["G"][r])


@pytest.mark.parametrize("kind,table", [(O.INTER, "I"), (O.J0, "J0"), (O.J1, "J1"),
                                        (O.J2, "J2")])
def test_tables_I_J(ex, kind, table):
    g, A, plan = ex
    assert plan.list_dict(kind) == {k: v for k, v in g[table].items() if v}


@pytest.mark.parametrize("kind,table", [(O.J0, "L0"), (O.J1, "L1"), (O.J2, "L2")])
def test_tables_L(ex, kind, table):
    g, A, plan = ex
    L = _by_src(plan.list_dict(kind))
    for r in range(g["np"]):
        assert L.get(r, set()) == set(g[table][r]), (table, r)


def test_printed_errata_are_exactly_the_corrected_cells(ex):
    """Every PRINTED cell differs from what the equations give; every other
    printed cell agrees (checked by the tests above)."""
    g, A, plan = ex
    lists = {"I": O.INTER, "J0": O.J0, "J1": O.J1, "J2": O.J2}
    for table, cells in g["printed"].items():
        if table in lists:
            got = plan.list_dict(lists[table])
            for key, printed in cells.items():
                assert got.get(key, ()) != printed, (table, key)
        else:  # L tables
            kind = {"L0": O.J0, "L1": O.J1, "L2": O.J2}[table]
            L = _by_src(plan.list_dict(kind))
            for key, printed in cells.items():
                assert L.get(key, set()) != set(printed), (table, key)
    # nine cells in all: I x2, L0, J0, L1, J1 x2, L2, J2
    assert sum(len(c) for c in g["printed"].values()) == 9


def test_message_statistics(ex):
    """Standard: 11 one-value messages, 3 intra-node and 8 inter-node; rank 0
    sends 3 inter-node messages.  Node-aware: 5 inter-node messages carrying 7
    values (v_0 goes to node 2 once, not twice); at most one inter-node message
    per process; 5 / 3 / 3 intra-node messages in the three local steps."""
    g, A, plan = ex
    s = plan.stats()
    assert (s["std_msgs"], s["std_vals"]) == (11, 11)
    assert (s["std_intra_msgs"], s["std_inter_msgs"], s["std_inter_vals"]) == (3, 8, 8)
    assert s["std_max_inter_msgs_proc"] == 3
    assert (s["nap_inter_msgs"], s["nap_inter_vals"]) == (5, 7)
    assert s["nap_max_inter_msgs_proc"] == 1
    assert (s["j0_msgs"], s["j0_vals"]) == (5, 5)
    assert (s["j1_msgs"], s["j1_vals"]) == (3, 3)
    assert (s["j2_msgs"], s["j2_vals"]) == (3, 3)


def test_brute_force_agrees_on_example(ex):
    g, A, plan = ex
    b = brute_plan(A.n, g["rows"], g["np"], g["ppn"])
    for name, kind in [("STD", O.STD), ("NODE", O.NODE), ("INTER", O.INTER), ("J0", O.J0),
                       ("J1", O.J1), ("J2", O.J2)]:
        assert plan.list_dict(kind) == b[name], name


def test_napspmv_equals_dense_product(ex):
    g, A, plan = ex
    v = np.array([0.5, -1.25, 2.0, 3.5, -0.75, 1.0])
    w = plan.napspmv(A.row_ptr, A.col, A.val, v)
    np.testing.assert_allclose(w, A.to_dense() @ v, rtol=1e-15, atol=0)
