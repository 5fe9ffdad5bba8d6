"""Randomised search for disagreements between the oracle's plans and the
literal evaluation of the set definitions (tests/brute.py): random sizes,
densities (empty rows included), partitions and every flag combination the
oracle accepts; the node-aware product against the dense one on the same
draws.  Derandomised, so every run draws the same examples.  CPU only."""
import numpy as np
import pytest

import oracle as O
from brute import brute_plan

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")

FLAGS = [0, O.MAP_TEXT, O.STRIDED, O.MAP_MAJORITY, O.STRIDED | O.MAP_TEXT,
         O.STRIDED | O.MAP_MAJORITY, O.MAP_SPLIT, O.MAP_SPLIT | O.MAP_TEXT,
         O.STRIDED | O.MAP_SPLIT]


@st.composite
def problems(draw):
    n = draw(st.integers(1, 40))
    dens = draw(st.sampled_from([0.0, 0.05, 0.1, 0.2, 0.4]))
    diag = draw(st.booleans())
    seed = draw(st.integers(0, 2**31 - 1))
    n_p = draw(st.integers(1, n))
    ppn = draw(st.integers(1, 8))
    flags = draw(st.sampled_from(FLAGS))
    rng = np.random.default_rng(seed)
    m = rng.random((n, n)) < dens
    if diag:
        np.fill_diagonal(m, True)
    rows, cols = np.nonzero(m)
    row_ptr = np.zeros(n + 1, np.int64)
    np.cumsum(m.sum(axis=1), out=row_ptr[1:])
    val = rng.uniform(-1.0, 1.0, len(cols))
    return n, row_ptr, cols.astype(np.int32), val, n_p, ppn, flags, seed


@hyp.settings(max_examples=300, deadline=None, derandomize=True,
              suppress_health_check=list(hyp.HealthCheck))
@hyp.given(problems())
def test_oracle_agrees_with_set_definitions(prob):
    n, row_ptr, col, val, n_p, ppn, flags, seed = prob
    rows = [set(col[row_ptr[i]:row_ptr[i + 1]].tolist()) for i in range(n)]
    plan = O.OraclePlan(row_ptr, col, n_p, ppn, flags=flags)
    b = brute_plan(n, rows, n_p, ppn, map_text=bool(flags & O.MAP_TEXT),
                   strided=bool(flags & O.STRIDED), majority=bool(flags & O.MAP_MAJORITY),
                   split=bool(flags & O.MAP_SPLIT))
    for name, kind in [("STD", O.STD), ("NODE", O.NODE), ("INTER", O.INTER), ("J0", O.J0),
                       ("J1", O.J1), ("J2", O.J2)]:
        assert plan.list_dict(kind) == b[name], name
    for name, kind in [("BLL", O.BLL), ("BNL", O.BNL), ("LBUF", O.LBUF)]:
        assert {s: idx for (s, d), idx in plan.list_dict(kind).items()} == b[name], name
    assert [tuple(r) for r in plan.split().tolist()] == b["split"]
    v = np.random.default_rng(seed + 1).uniform(-1.0, 1.0, n)
    dense = np.zeros((n, n))
    dense[np.repeat(np.arange(n), np.diff(row_ptr)), col] = val
    w = plan.napspmv(row_ptr, col, val, v)
    tol = 4 * np.finfo(float).eps * (np.abs(dense) @ np.abs(v)) + 1e-300
    assert np.all(np.abs(w - dense @ v) <= tol)
