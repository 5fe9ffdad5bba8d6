"""GPU plan build (through the C ABI) against the CPU oracle, bit-exact on every
message list, buffer layout, T/U assignment, block split and statistic."""
import math

import numpy as np
import pytest

import oracle as O
import golden_example
from gpu_util import assert_plans_equal, gpu_plan
from paper_1612_08060_gb300 import inputs as I
from paper_1612_08060_gb300 import napspmv as nap

pytestmark = pytest.mark.gpu


def test_worked_example():
    g = golden_example.load()
    n = len(g["rows"])
    cols = [sorted(g["rows"][i]) for i in range(n)]
    rp = np.zeros(n + 1, np.int64)
    rp[1:] = np.cumsum([len(c) for c in cols])
    A = I.CSR(rp, np.array([j for c in cols for j in c], np.int32), np.ones(int(rp[-1])))
    gp = gpu_plan(A, g["np"], g["ppn"])
    assert_plans_equal(gp, O.OraclePlan(A.row_ptr, A.col, g["np"], g["ppn"]))
    d = {}
    s, t, p, idx = nap.export_list(gp, nap.LIST_INTER)
    for k in range(len(s)):
        d[(int(s[k]), int(t[k]))] = tuple(int(x) for x in idx[p[k]:p[k + 1]])
    assert d == {k: v for k, v in g["I"].items()}


CASES = [(n, dens, seed, n_p, ppn)
         for seed, (n, dens) in enumerate([(9, 0.3), (24, 0.2), (48, 0.15), (97, 0.05),
                                           (200, 0.02)])
         for n_p, ppn in [(1, 1), (2, 1), (3, 2), (7, 3), (n, 1), (n, 4), (min(n, 13), 5),
                          (min(n, 32), 32), (min(n, 40), 8)]]


@pytest.mark.parametrize("n,dens,seed,n_p,ppn", CASES)
def test_random_patterns(n, dens, seed, n_p, ppn):
    A = I.random_pattern(n, dens, seed)
    assert_plans_equal(gpu_plan(A, n_p, ppn), O.OraclePlan(A.row_ptr, A.col, n_p, ppn))


@pytest.mark.parametrize("n_p,ppn", [(6, 2), (12, 5), (30, 4)])
def test_map_text(n_p, ppn):
    A = I.random_pattern(60, 0.08, 11)
    gp = gpu_plan(A, n_p, ppn, nap.MAP_TEXT)
    assert_plans_equal(gp, O.OraclePlan(A.row_ptr, A.col, n_p, ppn, flags=O.MAP_TEXT))


@pytest.mark.parametrize("n,dens,seed,n_p,ppn", CASES[::2])
def test_strided_random_patterns(n, dens, seed, n_p, ppn):
    """Strided partition (row i on process i mod n_p): the same lists, bit for
    bit, as the oracle's literal evaluation."""
    A = I.random_pattern(n, dens, seed)
    gp = gpu_plan(A, n_p, ppn, nap.F32_VALUES | nap.PARTITION_STRIDED)
    assert_plans_equal(gp, O.OraclePlan(A.row_ptr, A.col, n_p, ppn, flags=O.STRIDED))


@pytest.mark.parametrize("cfg,scale", [(1, 1), (2, 4), (3, 16)])
def test_strided_workloads(cfg, scale):
    w = I.workload(cfg, scale)
    A = w.build()
    gp = gpu_plan(A, w.n_p, w.ppn, nap.PARTITION_STRIDED | nap.MAP_TEXT)
    assert_plans_equal(gp, O.OraclePlan(A.row_ptr, A.col, w.n_p, w.ppn,
                                        flags=O.STRIDED | O.MAP_TEXT))


@pytest.mark.parametrize("n,dens,seed,n_p,ppn", CASES[1::3])
@pytest.mark.parametrize("strided", [False, True])
def test_majority_mapping(n, dens, seed, n_p, ppn, strided):
    """The majority mapping of node pairs (NAPSPMV_MAP_MAJORITY), both
    partitions: bit-exact against the oracle."""
    A = I.random_pattern(n, dens, seed)
    gflags = nap.MAP_MAJORITY | (nap.PARTITION_STRIDED if strided else 0)
    oflags = O.MAP_MAJORITY | (O.STRIDED if strided else 0)
    assert_plans_equal(gpu_plan(A, n_p, ppn, gflags),
                       O.OraclePlan(A.row_ptr, A.col, n_p, ppn, flags=oflags))


@pytest.mark.parametrize("cfg,scale", [(1, 1), (2, 4), (4, 64)])
def test_majority_mapping_workloads(cfg, scale):
    w = I.workload(cfg, scale)
    A = w.build()
    assert_plans_equal(gpu_plan(A, w.n_p, w.ppn, nap.MAP_MAJORITY),
                       O.OraclePlan(A.row_ptr, A.col, w.n_p, w.ppn, flags=O.MAP_MAJORITY))


@pytest.mark.parametrize("n,dens,seed,n_p,ppn", CASES[::2])
@pytest.mark.parametrize("extra", [0, 1])
def test_split_mapping(n, dens, seed, n_p, ppn, extra):
    """Node splitting (NAPSPMV_MAP_SPLIT, the text after Eq. U), alone and with
    the prose's receive order or the strided partition: bit-exact against the
    oracle."""
    A = I.random_pattern(n, dens, seed)
    gx, ox = [(nap.MAP_TEXT, O.MAP_TEXT), (nap.PARTITION_STRIDED, O.STRIDED)][extra]
    assert_plans_equal(gpu_plan(A, n_p, ppn, nap.MAP_SPLIT | gx),
                       O.OraclePlan(A.row_ptr, A.col, n_p, ppn, flags=O.MAP_SPLIT | ox))


@pytest.mark.parametrize("cfg,scale", [(1, 1), (2, 1), (3, 1), (4, 64)])
def test_split_mapping_workloads(cfg, scale):
    """Node splitting on the workloads, bit-exact against the oracle at full
    size.  In the 3D 7-point 128^3 and the Q1 2048^2 workloads an inner node has
    2 partner nodes and 16 processes (groups of 8 on both sides: 8 messages per
    pair); the first and the last node have one partner (a group of 16: the 4
    pairs that touch them carry 16 messages each)."""
    w = I.workload(cfg, scale)
    A = w.build()
    gp = gpu_plan(A, w.n_p, w.ppn, nap.MAP_SPLIT)
    op = O.OraclePlan(A.row_ptr, A.col, w.n_p, w.ppn, flags=O.MAP_SPLIT)
    assert_plans_equal(gp, op)
    if cfg in (2, 3):
        plain = O.OraclePlan(A.row_ptr, A.col, w.n_p, w.ppn).stats()
        st = op.stats()
        assert st["nap_inter_vals"] == plain["nap_inter_vals"]
        assert st["nap_inter_msgs"] == 8 * (plain["nap_inter_msgs"] - 4) + 16 * 4


def test_empty_matrix_and_empty_rows():
    n = 50
    A = I.CSR(np.zeros(n + 1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    assert_plans_equal(gpu_plan(A, 10, 3), O.OraclePlan(A.row_ptr, A.col, 10, 3))
    B = I.random_pattern(40, 0.1, 3, diag=False)
    assert_plans_equal(gpu_plan(B, 8, 3), O.OraclePlan(B.row_ptr, B.col, 8, 3))


@pytest.mark.parametrize("cfg,scale", [(1, 1), (2, 4), (3, 8), (4, 64)])
def test_workloads(cfg, scale):
    w = I.workload(cfg, scale)
    A = w.build()
    assert_plans_equal(gpu_plan(A, w.n_p, w.ppn), O.OraclePlan(A.row_ptr, A.col, w.n_p, w.ppn))


def test_config2_full_size():
    """3D 7-point 128^3, n_p = 1024, ppn = 16: bit-exact against the oracle and
    the closed-form counts (3,824 messages, 1,008 inter-node; 126 node pairs)."""
    w = I.workload(2)
    A = w.build()
    gp = gpu_plan(A, w.n_p, w.ppn)
    assert_plans_equal(gp, O.OraclePlan(A.row_ptr, A.col, w.n_p, w.ppn))
    s = nap.napspmv_plan_stats(gp)
    assert (s["std_msgs"], s["std_inter_msgs"], s["std_inter_vals"]) == (3824, 1008, 2064384)
    assert (s["nap_inter_msgs"], s["nap_inter_vals"]) == (126, 2064384)


def test_config3_full_size_counts():
    """2D Q1 2048^2, n_p = 4096, ppn = 16: counts from the stencil geometry
    (20,472 messages, 2,040 inter-node with 1,045,500 values; 510 node pairs
    with 1,044,480 values)."""
    w = I.workload(3)
    A = w.build()
    s = nap.napspmv_plan_stats(gpu_plan(A, w.n_p, w.ppn))
    assert (s["std_msgs"], s["std_intra_msgs"], s["std_inter_msgs"]) == (20472, 18432, 2040)
    assert s["std_inter_vals"] == 1045500
    assert (s["nap_inter_msgs"], s["nap_inter_vals"]) == (510, 1044480)


def test_invalid_inputs_rejected():
    A = I.poisson2d(8)
    with pytest.raises(nap.NapError) as e:
        nap.napspmv_plan(A.row_ptr, A.col, A.val, 4, 2, 64)  # unknown flag bit
    assert e.value.code == nap.ERR_ARG
    with pytest.raises(nap.NapError) as e:
        nap.napspmv_plan(A.row_ptr, A.col, A.val, 4, 2, nap.MAP_MAJORITY | nap.MAP_TEXT)
    assert e.value.code == nap.ERR_ARG
    bad = A.col.copy()
    bad[3] = 64
    with pytest.raises(nap.NapError) as e:
        nap.napspmv_plan(A.row_ptr, bad, A.val, 4, 2)
    assert e.value.code == nap.ERR_ARG
    dup = A.col.copy()
    dup[1] = dup[0]
    with pytest.raises(nap.NapError):
        nap.napspmv_plan(A.row_ptr, dup, A.val, 4, 2)
    rp = A.row_ptr.copy()
    rp[5] = rp[6] + 1
    with pytest.raises(nap.NapError):
        nap.napspmv_plan(rp, A.col, A.val, 4, 2)
    for n_p, ppn in [(0, 1), (65, 1), (4, 0)]:
        with pytest.raises(nap.NapError):
            nap.napspmv_plan(A.row_ptr, A.col, A.val, n_p, ppn)
