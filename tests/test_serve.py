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
    (SpMV and batched CG alike), the rest share the fused launch; results stay
    the same bits served alone or in a mix, and correct."""
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
    mixed = serve.Server(max_active=64, keep_results=True).run(specs, realtime=True)
    alone = serve.Server(max_active=1, keep_results=True).run(specs, realtime=False)
    by_id = {r.id: r for r in alone}
    for r in mixed:
        assert np.array_equal(r.result, by_id[r.id].result), r.id
        A = _matrix(r.spec)
        rhs = I.vector(A.n, r.spec["seed"])
        if r.kind == "spmv":
            ref = O.spmv(A.row_ptr, A.col, A.val, rhs)
            assert np.linalg.norm(r.result - ref) <= 1e-13 * np.linalg.norm(ref)
        else:
            res = rhs - O.spmv(A.row_ptr, A.col, A.val, r.result)
            assert np.linalg.norm(res) <= 1e-10 * np.linalg.norm(rhs), r.id
