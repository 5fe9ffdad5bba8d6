"""The continuous-batching server: every request's result is the same (bit for
bit) served alone and in a mix, SpMV results match the oracle, CG-IR solves
reach 1e-10 (recomputed by the oracle), and admission respects a memory budget."""
import numpy as np
import pytest

import oracle as O
from paper_1612_08060_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _specs(count=24, seed=5, n_hi=3e4):
    return I.serving_requests(count, rate_hz=2000.0, seed=seed, n_lo=200, n_hi=n_hi, p_spmv=0.6)


def _matrix(spec):
    return I.poisson2d(spec["side"]) if spec["dim"] == 2 else I.poisson3d(spec["side"])


def test_alone_equals_mix_and_correct():
    from paper_1612_08060_gb300 import serve
    specs = _specs()
    mixed = serve.Server(max_active=64, keep_results=True).run(specs, realtime=True)
    alone = serve.Server(max_active=1, keep_results=True).run(specs, realtime=False)
    by_id = {r.id: r for r in alone}
    assert {r.kind for r in mixed} == {"spmv", "cg"}
    for r in mixed:
        a = by_id[r.id]
        assert np.array_equal(r.result, a.result), r.id
        A = _matrix(r.spec)
        rhs = I.vector(A.n, r.spec["seed"])
        if r.kind == "spmv":
            ref = O.spmv(A.row_ptr, A.col, A.val, rhs)
            assert np.linalg.norm(r.result - ref) <= 1e-13 * np.linalg.norm(ref)
        else:
            res = rhs - O.spmv(A.row_ptr, A.col, A.val, r.result)
            assert np.linalg.norm(res) <= 1e-10 * np.linalg.norm(rhs), r.id


def test_memory_budget_admission():
    from paper_1612_08060_gb300 import serve
    specs = _specs(count=12, seed=9, n_hi=5e4)
    srv = serve.Server(mem_budget=12 << 20, max_active=64, keep_results=True)
    reqs = srv.run(specs, realtime=False)
    assert all(r.state == "done" for r in reqs)
    assert max(srv.batch_sizes) < len(specs)  # the budget held some requests back
    assert srv.mem_used <= srv.budget


def test_solo_matrices_alone_equals_mix():
    """Requests on matrices of at least SOLO_NNZ entries take the phased engine
    (SpMV and batched CG alike) in a group of their own on the second stream,
    with solo_iters_per_step CG iterations a step; the rest share the fused
    launch at iters_per_step.  Results stay the same bits served alone or in a
    mix, and correct."""
    from paper_1612_08060_gb300 import napspmv as nap, serve
    shapes = [(3, 44, "cg"), (2, 330, "spmv"), (3, 44, "spmv"), (2, 40, "cg"), (3, 14, "spmv"),
              (2, 90, "cg"), (2, 330, "cg")]
    specs = []
    for q, (dim, side, kind) in enumerate(shapes):
        n = side ** dim
        specs.append(dict(id=q, arrival=0.0002 * q, kind=kind, dim=dim, side=side, n=n,
                          n_p=max(1, round(n / 2048)), ppn=16, seed=1000 + q))
    big = [s for s in specs if _matrix(s).nnz >= nap.SOLO_NNZ]
    assert {s["kind"] for s in big} == {"spmv", "cg"} and len(big) < len(specs)
    srv = serve.Server(max_active=64, keep_results=True)
    mixed = srv.run(specs, realtime=True)
    alone = serve.Server(max_active=1, keep_results=True).run(specs, realtime=False)
    by_id = {r.id: r for r in alone}
    for r in mixed:
        if r.kind == "cg":
            # inner iterations come in whole steps of the request's own group
            step = srv.solo_iters if r.m.solo else srv.iters
            assert r.inner > 0 and r.inner % step == 0, (r.id, r.inner)
            assert r.inner == by_id[r.id].inner and r.outer == by_id[r.id].outer
        assert np.array_equal(r.result, by_id[r.id].result), r.id
        A = _matrix(r.spec)
        rhs = I.vector(A.n, r.spec["seed"])
        if r.kind == "spmv":
            ref = O.spmv(A.row_ptr, A.col, A.val, rhs)
            assert np.linalg.norm(r.result - ref) <= 1e-13 * np.linalg.norm(ref)
        else:
            res = rhs - O.spmv(A.row_ptr, A.col, A.val, r.result)
            assert np.linalg.norm(res) <= 1e-10 * np.linalg.norm(rhs), r.id


def test_caller_matrices_and_vectors(tmp_path):
    """Requests may carry the caller's own CSR and right-hand side (here banded
    random matrices with about 20 entries per row, whose plans default to two
    lanes per row for the tile pipelines, beside a Poisson spec): the results
    are the same bits alone and in a mix, SpMV within the oracle's bound, CG-IR
    to 1e-10; a tuning cache entry for a matrix is installed on its plan."""
    import json
    from paper_1612_08060_gb300 import autotune, napspmv as nap, serve
    mats = [I.banded_random(2500, 21), I.banded_random(3500, 22)]
    # make the banded matrices symmetric positive definite for the CG requests
    spd = []
    for A in mats:
        d = A.to_dense()
        d = 0.5 * (d + d.T)
        d[np.arange(A.n), np.arange(A.n)] = 1.0 + np.abs(d).sum(axis=1) - np.abs(np.diag(d))
        rows, cols = np.nonzero(d)
        rp = np.zeros(A.n + 1, np.int64)
        np.cumsum(np.bincount(rows, minlength=A.n), out=rp[1:])
        spd.append(I.CSR(rp, cols.astype(np.int32), d[rows, cols]))
    specs = []
    for q in range(10):
        A = spd[q % 2]
        specs.append(dict(id=q, arrival=0.0003 * q, kind="spmv" if q % 3 else "cg", n=A.n,
                          matrix=A, n_p=6 + q % 2, ppn=2, key=f"m{q % 2}",
                          rhs=I.vector(A.n, 50 + q)))
    specs.append(dict(_specs(1, seed=3)[0], id=10))
    cache = str(tmp_path / "tune.json")
    key = autotune.matrix_key(spd[0].row_ptr, 6, 2, nap.PREC_F64)
    opts = {"engine": nap.ENGINE_OVERLAP, "vec": 2, "tile_nnz": 1024, "tile_rows": 256,
            "stages": 2, "pipeline": nap.PIPELINE_SELL, "ctas_per_sm": 0, "chunk": 2048}
    with open(cache, "w") as f:
        json.dump({key: {"opts": opts, "ms": 1.0}}, f)
    srv = serve.Server(max_active=64, keep_results=True, tune_cache=cache)
    mixed = srv.run(specs, realtime=True)
    d = nap.napspmv_get_default_opts(srv.cache["user_m0_np6_ppn2"].plan)
    assert (d.tile_nnz, d.tile_rows, d.chunk) == (1024, 256, 2048)
    alone = serve.Server(max_active=1, keep_results=True, tune_cache=cache).run(specs,
                                                                                  realtime=False)
    by_id = {r.id: r for r in alone}
    for r in mixed:
        assert np.array_equal(r.result, by_id[r.id].result), r.id
        if "matrix" not in r.spec:
            continue
        A, rhs = r.spec["matrix"], r.spec["rhs"]
        if r.kind == "spmv":
            ref = O.spmv(A.row_ptr, A.col, A.val, rhs)
            assert np.linalg.norm(r.result - ref) <= 1e-13 * np.linalg.norm(ref)
        else:
            res = rhs - O.spmv(A.row_ptr, A.col, A.val, r.result)
            assert np.linalg.norm(res) <= 1e-10 * np.linalg.norm(rhs), r.id
