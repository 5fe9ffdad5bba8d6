"""Sec. 3 cost models with the paper's Blue Waters parameters, checked by hand on
single messages and on the worked example's plans (via the oracle)."""
import math

import numpy as np
import pytest

import oracle as O
import golden_example
from paper_1612_08060_gb300 import model as M


def test_single_message_formulas():
    # 64 KiB rendezvous inter-node message, ppn = 16:
    # T = 2e-5 + 16 * 65536 / min(5.5e9, 6.1e8 + 15 * 3.6e9)
    s = 65536
    want = 2.0e-5 + 16 * s / min(5.5e9, 6.1e8 + 15 * 3.6e9)
    assert M.inter_time(s, 16) == pytest.approx(want, rel=1e-15)
    # ppn = 1 reduces to the postal model alpha + s / B_max
    assert M.inter_time(s, 1) == pytest.approx(2.0e-5 + s / 6.1e8, rel=1e-15)
    # eager intra-node: 1.6e-6 + 4096 / 7.4e8
    assert M.intra_time(4096) == pytest.approx(1.6e-6 + 4096 / 7.4e8, rel=1e-15)
    # short, ppn = 1: the printed B_max is negative -> latency only
    assert M.inter_time(8, 1) == 4.0e-6
    assert M.protocol(512) == "short" and M.protocol(513) == "eager"
    assert M.protocol(8193) == "rend"


def test_worked_example_node_aware_beats_standard():
    g = golden_example.load()
    n = len(g["rows"])
    cols = [sorted(g["rows"][i]) for i in range(n)]
    rp = np.zeros(n + 1, np.int64)
    rp[1:] = np.cumsum([len(c) for c in cols])
    col = np.array([j for c in cols for j in c], np.int32)
    P = O.OraclePlan(rp, col, g["np"], g["ppn"])
    lists = {k: P.list(getattr(O, k))[:3] for k in ("STD", "INTER", "J0", "J1", "J2")}
    m = M.modelled(lists, g["ppn"], g["np"])
    # rank 0 sends three one-value inter-node messages (short, ppn = 2):
    # 3 * (4e-6 + 2 * 8 / (-1.8e7 + 6.3e8)); every other rank sends fewer
    per = 4.0e-6 + 2 * 8 / (-1.8e7 + 6.3e8)
    assert m["std_max_s"] == pytest.approx(3 * per, rel=1e-12)
    # node-aware: at most one inter-node message per process, the largest with
    # two values
    assert m["nap_inter_max_s"] == pytest.approx(4.0e-6 + 2 * 16 / (-1.8e7 + 6.3e8), rel=1e-12)
    assert m["nap_inter_max_s"] < m["std_max_s"]
    assert math.isfinite(m["nap_max_s"])
