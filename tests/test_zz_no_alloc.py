"""napspmv_apply_noalloc: the apply for callers that cannot allocate device memory
(another allocator owns the device's free memory, or cudaMalloc's implicit
synchronisation is not acceptable on their path).  Its buffers live in a fixed
static device array.  On two calls in a row its result must have the bits of the
allocating fused-engine apply with the same options, match the default apply and
the oracle, and leave the device's free memory unchanged; plans too large for
the array are rejected.

Collected last on purpose (file name) so that a run stopping at the first
failure has already run every other test."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import abs_row_bound, assert_close_fp64, gpu_plan, oracle_chain
from paper_1612_08060_gb300 import inputs as I
from paper_1612_08060_gb300 import napspmv as nap

pytestmark = pytest.mark.gpu

SCRATCH_DOUBLES = 1 << 20


def _scratch_need(plan, A, n_p, ppn, reps):
    """Doubles of the static array one call needs (as the header states)."""
    st = nap.napspmv_plan_stats(plan)
    need = (2 + st["bll_total"] + st["lbuf_total"] + 2 * st["nap_inter_vals"] +
            st["bnl_total"])
    return need + (A.n if reps > 1 else 0)


def _fused_opts_of_noalloc(plan, tile_rows=None, tile_nnz=None, chunk=None):
    """The options napspmv_apply_noalloc runs with: the plan's defaults on the
    fused engine, FP64, and the tile shape of the plan's current row tiles."""
    o = nap.napspmv_get_default_opts(plan)
    o.engine = nap.ENGINE_FUSED
    o.precision = nap.PREC_F64
    if tile_rows:
        o.tile_rows = tile_rows
    if tile_nnz:
        o.tile_nnz = tile_nnz
    if chunk:
        o.chunk = chunk
    return o


def _run_two_calls(A, plan, reps, scale, opts_same, seed=100):
    """Two no-alloc calls in a row, the device's free memory read around them;
    then the allocating applies.  Returns nothing; asserts everything."""
    vs = [torch.from_numpy(I.vector(A.n, seed + c)).cuda() for c in range(2)]
    got = [torch.full_like(vs[0], float("nan")) for _ in range(2)]
    same = [torch.full_like(vs[0], float("nan")) for _ in range(2)]
    dflt = [torch.full_like(vs[0], float("nan")) for _ in range(2)]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for c in range(2):  # two calls in a row share (and reuse) the static area
        nap.napspmv_apply_noalloc(plan, vs[c], got[c], reps, scale)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0, "the no-alloc apply changed free memory"
    assert nap.napspmv_status(plan) == nap.OK
    for c in range(2):
        nap.napspmv_apply_ex(plan, vs[c], same[c], reps, scale, opts_same)
        assert nap.napspmv_status(plan) == nap.OK
        assert torch.equal(got[c], same[c]), f"call {c}: bits differ from the fused apply"
    for c in range(2):
        nap.napspmv_apply_n(plan, vs[c], dflt[c], reps, scale)
        assert nap.napspmv_status(plan) == nap.OK
        g, r = got[c].cpu().numpy(), dflt[c].cpu().numpy()
        assert np.linalg.norm(g - r) <= 1e-13 * max(1.0, reps) * np.linalg.norm(r)
        v = vs[c].cpu().numpy()
        if reps == 1:
            assert_close_fp64(g, O.spmv(A.row_ptr, A.col, A.val, v), abs_row_bound(A, v))
        else:
            ref = oracle_chain(A, v, reps, scale)
            assert np.linalg.norm(g - ref) <= 1e-13 * reps * np.linalg.norm(ref)


@pytest.mark.parametrize("make,n_p,ppn,reps,scale", [
    (lambda: I.poisson2d(64), 16, 4, 1, 1.0),
    (lambda: I.poisson3d(40), 32, 8, 5, 1.0 / 16.0),
    (lambda: I.random_pattern(700, 0.01, 3), 70, 4, 2, 0.5),
    # about 20 entries per row: two lanes per row, warp-tuned 1024 / 2048 tiles
    (lambda: I.banded_random(8000, 5), 8, 2, 1, 1.0),
    (lambda: I.banded_random(8000, 6), 8, 2, 3, 1.0 / 64.0),
])
def test_noalloc_matches_allocating_entry_point(make, n_p, ppn, reps, scale):
    A = make()
    plan = gpu_plan(A, n_p, ppn)
    d = nap.napspmv_get_default_opts(plan)
    if A.nnz > 16 * A.n:
        assert d.vec == 2 and d.tile_nnz == 2048
    assert _scratch_need(plan, A, n_p, ppn, reps) <= SCRATCH_DOUBLES
    # a warm-up call: the first call on a device looks the array's address up
    w0 = torch.empty(A.n, dtype=torch.float64, device="cuda")
    nap.napspmv_apply_noalloc(plan, torch.zeros_like(w0), w0, 1, 1.0)
    _run_two_calls(A, plan, reps, scale, _fused_opts_of_noalloc(plan))


def test_noalloc_after_defaults_changed():
    """napspmv_set_default_opts rebuilt the plan's work items with another tile
    shape: the no-alloc apply runs with those items."""
    A = I.poisson3d(30)
    plan = gpu_plan(A, 12, 4)
    nap.napspmv_set_default_opts(plan, nap.make_opts(tile_rows=128, tile_nnz=512, chunk=1024))
    d = nap.napspmv_get_default_opts(plan)
    assert (d.tile_rows, d.tile_nnz, d.chunk) == (128, 512, 1024)
    _run_two_calls(A, plan, 3, 0.125, _fused_opts_of_noalloc(plan), seed=300)


def test_noalloc_after_a_batch_with_another_tile_shape():
    """A batch given explicit tile options rebuilds the plans' work items; the
    no-alloc apply then runs with the items the plan holds (and its default lane
    count), which the fused apply with the same tile shape reproduces."""
    A = I.banded_random(6000, 9)
    B = I.poisson2d(50)
    pa, pb = gpu_plan(A, 6, 3), gpu_plan(B, 10, 5)
    va = torch.from_numpy(I.vector(A.n, 1)).cuda()
    vb = torch.from_numpy(I.vector(B.n, 2)).cuda()
    o = nap.make_opts(engine=nap.ENGINE_FUSED, tile_rows=64, tile_nnz=256, chunk=512)
    nap.napspmv_apply_batch([pa, pb], [va, vb], [torch.empty_like(va), torch.empty_like(vb)],
                            [1, 1], opts=o)
    assert nap.napspmv_status(pa) == nap.OK and nap.napspmv_status(pb) == nap.OK
    vs = [torch.from_numpy(I.vector(A.n, 400 + c)).cuda() for c in range(2)]
    got = [torch.full_like(va, float("nan")) for _ in range(2)]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for c in range(2):
        nap.napspmv_apply_noalloc(pa, vs[c], got[c], 2, 0.25)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
    assert nap.napspmv_status(pa) == nap.OK
    same = _fused_opts_of_noalloc(pa, tile_rows=64, tile_nnz=256, chunk=512)
    for c in range(2):
        alone = torch.empty_like(va)
        nap.napspmv_apply_ex(pa, vs[c], alone, 2, 0.25, same)
        assert nap.napspmv_status(pa) == nap.OK
        assert torch.equal(alone, got[c]), c
        dflt = torch.empty_like(va)
        nap.napspmv_apply_n(pa, vs[c], dflt, 2, 0.25)
        g, r = got[c].cpu().numpy(), dflt.cpu().numpy()
        assert np.linalg.norm(g - r) <= 2e-13 * np.linalg.norm(r)
        ref = oracle_chain(A, vs[c].cpu().numpy(), 2, 0.25)
        assert np.linalg.norm(g - ref) <= 2e-13 * np.linalg.norm(ref)


def test_noalloc_chain_vector_only_when_chained():
    """One apply needs no chain vector: a plan that fits the array with reps = 1
    but not with the extra N values of reps = 2 is accepted once, refused chained."""
    A = I.poisson3d(100)  # N = 10^6; two processes, one per node: 2 x 10^4 values per buffer
    plan = gpu_plan(A, 2, 1)
    assert _scratch_need(plan, A, 2, 1, 1) <= SCRATCH_DOUBLES < _scratch_need(plan, A, 2, 1, 2)
    v = I.vector(A.n, 7)
    vd = torch.from_numpy(v).cuda()
    wd = torch.full_like(vd, float("nan"))
    nap.napspmv_apply_noalloc(plan, vd, wd, 1, 1.0)
    assert nap.napspmv_status(plan) == nap.OK
    assert_close_fp64(wd.cpu().numpy(), O.spmv(A.row_ptr, A.col, A.val, v), abs_row_bound(A, v))
    with pytest.raises(nap.NapError) as e:
        nap.napspmv_apply_noalloc(plan, vd, wd, 2, 1.0)
    assert e.value.code == nap.ERR_UNSUPPORTED and "static area" in str(e.value)


def test_noalloc_rejects_plans_beyond_the_static_area():
    A = I.poisson3d(104)  # N = 1,124,864 > 2^20 doubles of scratch
    plan = gpu_plan(A, 64, 16)
    assert _scratch_need(plan, A, 64, 16, 1) > SCRATCH_DOUBLES
    vd = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    with pytest.raises(nap.NapError) as e:
        nap.napspmv_apply_noalloc(plan, vd, torch.empty_like(vd))
    assert e.value.code == nap.ERR_UNSUPPORTED
    assert "static area" in str(e.value)
