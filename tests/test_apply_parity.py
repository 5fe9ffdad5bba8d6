"""The node-aware apply on the GPU (through the C ABI) against the CPU oracle.

FP64: elementwise |w - w_ref| <= 1e-13 (|A||v|)_i and normwise relative error
<= 1e-13.  FP32-stored values: within 1e-13 of the oracle's FP32-product /
FP64-sum result and <= 1e-6 normwise of the FP64 product."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import abs_row_bound, assert_close_fp64, gpu_plan, oracle_chain
from paper_1612_08060_gb300 import inputs as I
from paper_1612_08060_gb300 import napspmv as nap

pytestmark = pytest.mark.gpu


def run(plan, v, reps=1, scale=1.0, **opts):
    vd = torch.from_numpy(np.ascontiguousarray(v)).cuda()
    wd = torch.full_like(vd, float("nan"))
    o = nap.make_opts(**opts) if opts else None
    nap.napspmv_apply_ex(plan, vd, wd, reps, scale, o)
    assert nap.napspmv_status(plan) == 0
    return wd.cpu().numpy()


ENGINES = [dict(engine=nap.ENGINE_FUSED), dict(engine=nap.ENGINE_PHASED),
           dict(engine=nap.ENGINE_OVERLAP),
           dict(engine=nap.ENGINE_PHASED, pipeline=nap.PIPELINE_WARP),
           dict(engine=nap.ENGINE_OVERLAP, pipeline=nap.PIPELINE_WARP),
           dict(engine=nap.ENGINE_PHASED, pipeline=nap.PIPELINE_SELL),
           dict(engine=nap.ENGINE_OVERLAP, pipeline=nap.PIPELINE_SELL)]
SHAPES = [dict(vec=v) for v in (1, 2, 4, 8, 32)]


@pytest.mark.parametrize("eng", ENGINES)
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("n,dens,n_p,ppn", [(64, 0.1, 8, 3), (300, 0.02, 37, 4),
                                             (1000, 0.01, 1000, 16), (513, 0.03, 1, 1)])
def test_random_fp64(eng, shape, n, dens, n_p, ppn):
    A = I.random_pattern(n, dens, n + n_p)
    v = I.vector(n, 5)
    w = run(gpu_plan(A, n_p, ppn), v, **eng, **shape)
    assert_close_fp64(w, O.spmv(A.row_ptr, A.col, A.val, v), abs_row_bound(A, v))


@pytest.mark.parametrize("eng", ENGINES)
@pytest.mark.parametrize("chunk,tile", [(32, 1), (64, 7), (4096, 1024), (100000, 8000)])
def test_item_sizes(eng, chunk, tile):
    w_ = I.workload(1)
    A = w_.build()
    v = I.vector(A.n, w_.seed)
    w = run(gpu_plan(A, w_.n_p, w_.ppn), v, chunk=chunk, tile_rows=tile,
            tile_nnz=min(4096, max(32, 5 * tile)), **eng)
    assert_close_fp64(w, O.spmv(A.row_ptr, A.col, A.val, v), abs_row_bound(A, v))


@pytest.mark.parametrize("eng", ENGINES)
@pytest.mark.parametrize("reps,scale", [(2, 1.0 / 12.0), (3, 0.25), (10, 1.0 / 16.0), (4, 1.0)])
def test_chained(eng, reps, scale):
    A = I.poisson3d(20)
    v = I.vector(A.n, 9)
    plan = gpu_plan(A, 40, 4)
    w = run(plan, v, reps=reps, scale=scale, **eng)
    ref = oracle_chain(A, v, reps, scale)
    assert np.linalg.norm(w - ref) <= 1e-13 * reps * np.linalg.norm(ref)


@pytest.mark.parametrize("eng", ENGINES)
def test_fp32_values(eng):
    A = I.aniso_q1(96)
    v = I.vector(A.n, 13)
    plan = gpu_plan(A, 18, 4)
    w = run(plan, v, precision=nap.PREC_F32, **eng)
    ref32 = O.spmv_f32(A.row_ptr, A.col, A.val.astype(np.float32), v)
    ref64 = O.spmv(A.row_ptr, A.col, A.val, v)
    assert np.linalg.norm(w - ref32) <= 1e-13 * np.linalg.norm(ref32)
    assert np.linalg.norm(w - ref64) <= 1e-6 * np.linalg.norm(ref64)


def test_fp32_requires_flag():
    A = I.poisson2d(8)
    plan = nap.napspmv_plan(A.row_ptr, A.col, A.val, 4, 2, 0)
    vd = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    with pytest.raises(nap.NapError) as e:
        nap.napspmv_apply_ex(plan, vd, torch.empty_like(vd), 1, 1.0,
                             nap.make_opts(precision=nap.PREC_F32))
    assert e.value.code == nap.ERR_STATE


@pytest.mark.parametrize("eng", ENGINES)
def test_edge_cases(eng):
    # nnz = 0
    n = 37
    A = I.CSR(np.zeros(n + 1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    w = run(gpu_plan(A, 5, 2), I.vector(n, 1), **eng)
    assert np.array_equal(w, np.zeros(n))
    # empty rows, uneven partition, partial last node, ppn > n_p
    B = I.random_pattern(101, 0.05, 17, diag=False)
    v = I.vector(101, 2)
    for n_p, ppn in [(7, 3), (10, 64), (101, 1), (1, 5)]:
        w = run(gpu_plan(B, n_p, ppn), v, **eng)
        assert_close_fp64(w, O.spmv(B.row_ptr, B.col, B.val, v), abs_row_bound(B, v))
    # one dense row among short ones (long-row lane reduction)
    C = I.random_pattern(200, 0.01, 4)
    rows = [set(C.col[C.row_ptr[i]:C.row_ptr[i + 1]]) for i in range(200)]
    rows[77] = set(range(200))
    rp = np.zeros(201, np.int64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    col = np.array([j for r in rows for j in sorted(r)], np.int32)
    D = I.CSR(rp, col, np.random.default_rng(5).uniform(-1, 1, len(col)))
    v = I.vector(200, 3)
    for vec in (1, 4, 32):
        w = run(gpu_plan(D, 9, 2), v, vec=vec, **eng)
        assert_close_fp64(w, O.spmv(D.row_ptr, D.col, D.val, v), abs_row_bound(D, v))


@pytest.mark.parametrize("reps", [1, 3])
def test_engines_agree_bitwise(reps):
    """With one lane per row every engine evaluates each row's FMA chain in the
    same order (on_process, on_node, off_node; the overlapped engine continues
    the chain from the local partial): identical bits."""
    A = I.aniso_q1(64)
    v = I.vector(A.n, 21)
    plan = gpu_plan(A, 16, 4)
    a = run(plan, v, reps=reps, scale=0.25, engine=nap.ENGINE_FUSED, vec=1)
    b = run(plan, v, reps=reps, scale=0.25, engine=nap.ENGINE_PHASED, vec=1)
    c = run(plan, v, reps=reps, scale=0.25, engine=nap.ENGINE_OVERLAP, vec=1)
    d = run(plan, v, reps=reps, scale=0.25, engine=nap.ENGINE_PHASED, pipeline=nap.PIPELINE_SELL)
    e = run(plan, v, reps=reps, scale=0.25, engine=nap.ENGINE_OVERLAP, pipeline=nap.PIPELINE_SELL)
    assert np.array_equal(a, b) and np.array_equal(a, c)
    assert np.array_equal(a, d) and np.array_equal(a, e)


@pytest.mark.parametrize("reps", [1, 3])
def test_engines_agree_bitwise_fp32(reps):
    """FP32 values: the fused engine rounds each gathered FP64 x to FP32 at the
    product; the phased engines carry FP32 copies of the same values through
    the message steps.  Same floats, same chain order: identical bits."""
    A = I.aniso_q1(64)
    v = I.vector(A.n, 22)
    plan = gpu_plan(A, 16, 4)
    o = dict(reps=reps, scale=0.25, vec=1, precision=nap.PREC_F32)
    a = run(plan, v, engine=nap.ENGINE_FUSED, **o)
    b = run(plan, v, engine=nap.ENGINE_PHASED, **o)
    c = run(plan, v, engine=nap.ENGINE_OVERLAP, **o)
    d = run(plan, v, engine=nap.ENGINE_OVERLAP, pipeline=nap.PIPELINE_WARP, **o)
    e = run(plan, v, engine=nap.ENGINE_OVERLAP, pipeline=nap.PIPELINE_SELL, **o)
    f = run(plan, v, engine=nap.ENGINE_PHASED, pipeline=nap.PIPELINE_SELL, **o)
    assert np.array_equal(a, b) and np.array_equal(a, c) and np.array_equal(a, d)
    assert np.array_equal(a, e) and np.array_equal(a, f)


def _mixed_rows(n=900, seed=31):
    """Rows of very different lengths: empty rows, short rows, rows of 100-250
    entries and a few rows longer than the sliced-row limit (256 entries)."""
    rng = np.random.default_rng(seed)
    lens = rng.choice([0, 1, 3, 7, 20, 120, 250], size=n, p=[.1, .1, .2, .3, .2, .07, .03])
    lens[rng.choice(n, 6, replace=False)] = rng.integers(257, n, 6)
    cols = [np.sort(rng.choice(n, int(k), replace=False)) for k in lens]
    row_ptr = np.zeros(n + 1, np.int64)
    np.cumsum(lens, out=row_ptr[1:])
    col = np.concatenate(cols).astype(np.int32)
    return I.CSR(row_ptr, col, rng.uniform(-1, 1, len(col)))


@pytest.mark.parametrize("prec", [nap.PREC_F64, nap.PREC_F32])
@pytest.mark.parametrize("n_p,ppn,flags", [(9, 3, 0), (30, 4, nap.PARTITION_STRIDED), (1, 1, 0)])
def test_sell_mixed_row_lengths(prec, n_p, ppn, flags):
    """Sliced rows on rows of very different lengths (chunks cut where the
    count halves, empty rows, rows past the 256-entry limit summed by a warp):
    within the oracle's bound; and, rows of at most 256 entries, the same bits as
    one lane per row on the CTA pipeline."""
    A = _mixed_rows()
    plan = nap.napspmv_plan(A.row_ptr, A.col, A.val, n_p, ppn, flags | nap.F32_VALUES)
    v = I.vector(A.n, 17)
    for eng in (nap.ENGINE_PHASED, nap.ENGINE_OVERLAP):
        w = run(plan, v, reps=1, scale=0.5, engine=eng, pipeline=nap.PIPELINE_SELL, precision=prec)
        ref = run(plan, v, reps=1, scale=0.5, engine=eng, pipeline=nap.PIPELINE_CTA, vec=1,
                  tile_nnz=4096, precision=prec)
        short = np.diff(A.row_ptr) <= 256
        assert np.array_equal(w[short], ref[short]), eng
        if prec == nap.PREC_F64:
            assert_close_fp64(w, 0.5 * O.spmv(A.row_ptr, A.col, A.val, v),
                              0.5 * abs_row_bound(A, v))
        else:
            ref32 = 0.5 * O.spmv_f32(A.row_ptr, A.col, A.val.astype(np.float32), v)
            assert np.linalg.norm(w - ref32) <= 1e-13 * np.linalg.norm(ref32)


@pytest.mark.parametrize("eng", ENGINES)
def test_fp32_product_special_values(eng):
    """Rows of one entry: w_i is the FP32 product itself, widened to FP64 (0 +
    p).  Products that are normal, subnormal, +-0, +-inf or NaN must widen
    exactly as the oracle's (C) conversion does: compared bit for bit."""
    a = np.array([1.5, 1e-30, 3.0, -2.0, 1e30, -1e30, 0.0, 2.0 ** -126, 7.0, 1.0, 0.5, 1.0],
                 np.float32)
    x = np.array([0.1, 1e-15, -0.0, 0.0, 1e30, 1e30, np.inf, 0.75, 1.0 / 3.0, np.nan,
                  2.0 ** -140, -3.4e38])
    n = len(a)
    A = I.CSR(np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), a.astype(np.float64))
    w = run(gpu_plan(A, 4, 2), x, precision=nap.PREC_F32, **eng)
    with np.errstate(all="ignore"):
        ref = O.spmv_f32(A.row_ptr, A.col, a, x)
    assert np.array_equal(np.isnan(w), np.isnan(ref))
    ok = ~np.isnan(ref)
    assert np.array_equal(w[ok].view(np.uint64), ref[ok].view(np.uint64)), (w, ref)


@pytest.mark.parametrize("eng", ENGINES)
@pytest.mark.parametrize("n,dens,n_p,ppn", [(300, 0.02, 37, 4), (1000, 0.01, 64, 16),
                                             (97, 0.05, 97, 3)])
def test_strided_partition(eng, n, dens, n_p, ppn):
    """Strided plans (row i on process i mod n_p) on every engine: FP64 and
    FP32-value applies, single and chained, against the oracle."""
    A = I.random_pattern(n, dens, n + 7)
    v = I.vector(n, 8)
    plan = gpu_plan(A, n_p, ppn, nap.F32_VALUES | nap.PARTITION_STRIDED)
    for vec in (1, 4):
        w = run(plan, v, vec=vec, **eng)
        assert_close_fp64(w, O.spmv(A.row_ptr, A.col, A.val, v), abs_row_bound(A, v))
    w = run(plan, v, reps=3, scale=0.5, **eng)
    ref = oracle_chain(A, v, 3, 0.5)
    assert np.linalg.norm(w - ref) <= 3e-13 * np.linalg.norm(ref)
    w = run(plan, v, precision=nap.PREC_F32, **eng)
    ref32 = O.spmv_f32(A.row_ptr, A.col, A.val.astype(np.float32), v)
    assert np.linalg.norm(w - ref32) <= 1e-13 * np.linalg.norm(ref32)


@pytest.mark.parametrize("eng", ENGINES)
def test_majority_mapping_apply(eng):
    A = I.random_pattern(400, 0.02, 31)
    v = I.vector(400, 32)
    plan = gpu_plan(A, 40, 4, nap.F32_VALUES | nap.MAP_MAJORITY)
    w = run(plan, v, reps=2, scale=0.5, **eng)
    ref = oracle_chain(A, v, 2, 0.5)
    assert np.linalg.norm(w - ref) <= 2e-13 * np.linalg.norm(ref)


@pytest.mark.parametrize("eng", ENGINES)
def test_split_mapping_apply(eng):
    """Node splitting (several inter-node messages per node pair): every engine
    within the oracle's bound, one apply and a chain; with one lane per row the
    same bits as the unsplit plan (the received values are the same)."""
    A = I.random_pattern(400, 0.02, 33)
    v = I.vector(400, 34)
    plan = gpu_plan(A, 40, 8, nap.F32_VALUES | nap.MAP_SPLIT)
    w = run(plan, v, reps=1, **eng)
    assert_close_fp64(w, O.spmv(A.row_ptr, A.col, A.val, v), abs_row_bound(A, v))
    w = run(plan, v, reps=3, scale=0.5, **eng)
    ref = oracle_chain(A, v, 3, 0.5)
    assert np.linalg.norm(w - ref) <= 3e-13 * np.linalg.norm(ref)
    B = I.poisson3d(24)
    vb = I.vector(B.n, 35)
    a = run(gpu_plan(B, 27, 9, nap.F32_VALUES | nap.MAP_SPLIT), vb, vec=1, **eng)
    b = run(gpu_plan(B, 27, 9, nap.F32_VALUES), vb, vec=1, **eng)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("strided", [False, True])
@pytest.mark.parametrize("prec", [nap.PREC_F64, nap.PREC_F32])
def test_composed_gathers_same_bits(strided, prec):
    """Composed gathers fetch each receive buffer straight from v; the literal
    exchange delivers the same values through its hops, so every engine gives
    identical bits with either plan."""
    A = I.random_pattern(600, 0.015, 41)
    v = I.vector(600, 42)
    part = nap.PARTITION_STRIDED if strided else 0
    lit = gpu_plan(A, 48, 4, nap.F32_VALUES | part)
    com = gpu_plan(A, 48, 4, nap.F32_VALUES | part | nap.COMPOSED_GATHERS)
    for eng in ENGINES:
        for reps in (1, 3):
            a = run(lit, v, reps=reps, scale=0.5, precision=prec, **eng)
            b = run(com, v, reps=reps, scale=0.5, precision=prec, **eng)
            assert np.array_equal(a, b), (eng, reps)
    ref = oracle_chain(A, v, 3, 0.5)
    if prec == nap.PREC_F64:
        assert np.linalg.norm(b - ref) <= 3e-13 * np.linalg.norm(ref)


@pytest.mark.parametrize("prec", [nap.PREC_F64, nap.PREC_F32])
@pytest.mark.parametrize("vec", [1, 2, 8])
@pytest.mark.parametrize("case", ["random", "poisson3d", "banded"])
def test_halo_staging_same_bits(case, vec, prec):
    """The overlapped engine's remote pass with each process's receive buffers
    staged in shared memory (the default) against gathers from global memory:
    same values in the same order, identical bits; both within the oracle's
    tolerance."""
    if case == "random":
        A, n_p, ppn = I.random_pattern(700, 0.02, 51), 33, 4
    elif case == "poisson3d":
        A, n_p, ppn = I.poisson3d(24), 54, 6
    else:
        w_ = I.workload(4, 64)
        A, n_p, ppn = w_.build(), w_.n_p, w_.ppn
    v = I.vector(A.n, 52)
    plan = gpu_plan(A, n_p, ppn)
    o = dict(engine=nap.ENGINE_OVERLAP, vec=vec, precision=prec, reps=2, scale=0.5,
             pipeline=nap.PIPELINE_CTA)
    a = run(plan, v, halo=nap.HALO_ON, **o)
    b = run(plan, v, halo=nap.HALO_OFF, **o)
    assert np.array_equal(a, b)
    if prec == nap.PREC_F64:
        ref = oracle_chain(A, v, 2, 0.5)
        assert np.linalg.norm(a - ref) <= 2e-13 * np.linalg.norm(ref)


def test_halo_staging_edge_cases():
    """Staged receive buffers with a row longer than a stage (summed by the
    whole CTA from global entries and the staged window) and with processes
    whose rows have no remote entries at all (empty windows)."""
    n, n_p, ppn = 800, 20, 4
    base = I.random_pattern(n, 0.03, 61)
    rows = [set(base.col[base.row_ptr[i]:base.row_ptr[i + 1]].tolist()) for i in range(n)]
    rows[400] = set(range(n))                      # one dense row
    for i in range(0, 160):                        # processes 0-3 own rows 0-159:
        rows[i] = {j for j in rows[i] if j < 40 * (i // 40 + 1) and j >= 40 * (i // 40)} | {i}
    rp = np.zeros(n + 1, np.int64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    col = np.array([j for r in rows for j in sorted(r)], np.int32)
    A = I.CSR(rp, col, np.random.default_rng(62).uniform(-1, 1, len(col)))
    v = I.vector(n, 63)
    plan = gpu_plan(A, n_p, ppn)
    # the staged pass runs CTA tiles; against the CTA pipeline's global-gather
    # pass the bits agree (the warp pipeline sums rows longer than a warp stage
    # in another order, so it is held to the oracle's tolerance instead)
    for prec in (nap.PREC_F64, nap.PREC_F32):
        o = dict(engine=nap.ENGINE_OVERLAP, vec=1, tile_nnz=256, tile_rows=64, precision=prec,
                 reps=2, scale=0.5, pipeline=nap.PIPELINE_CTA)
        a = run(plan, v, halo=nap.HALO_ON, **o)
        b = run(plan, v, halo=nap.HALO_OFF, **o)
        assert np.array_equal(a, b), prec
    ref = oracle_chain(A, v, 1, 1.0)
    for pipe in (nap.PIPELINE_CTA, nap.PIPELINE_WARP):
        for halo in (nap.HALO_ON, nap.HALO_OFF):
            w = run(plan, v, engine=nap.ENGINE_OVERLAP, tile_nnz=256, tile_rows=64,
                    pipeline=pipe, halo=halo)
            assert_close_fp64(w, ref, abs_row_bound(A, v))


@pytest.mark.parametrize("flags", [nap.PARTITION_STRIDED, nap.COMPOSED_GATHERS,
                                   nap.PARTITION_STRIDED | nap.COMPOSED_GATHERS])
def test_strided_and_composed_on_every_entry(flags):
    """Strided and composed-gather plans run on the fused engine too (its levels
    need no contiguous node rows): a fused apply, a batch of two and the
    no-allocation entry point, each against the oracle."""
    A = I.poisson2d(20)
    plan = gpu_plan(A, 10, 3, nap.F32_VALUES | flags)
    plan2 = gpu_plan(A, 10, 3, nap.F32_VALUES | flags)
    v = I.vector(A.n, 4)
    vd = torch.from_numpy(v).cuda()
    ref = O.spmv(A.row_ptr, A.col, A.val, v)
    bound = abs_row_bound(A, v)
    outs = [torch.full_like(vd, float("nan")) for _ in range(4)]
    nap.napspmv_apply_ex(plan, vd, outs[0], 1, 1.0, nap.make_opts(engine=nap.ENGINE_FUSED))
    nap.napspmv_apply_batch([plan, plan2], [vd, vd], [outs[1], outs[2]], [1, 1], [1.0, 1.0])
    nap.napspmv_apply_noalloc(plan, vd, outs[3], 1, 1.0)
    assert nap.napspmv_status(plan) == 0 and nap.napspmv_status(plan2) == 0
    for o in outs:
        assert_close_fp64(o.cpu().numpy(), ref, bound)


@pytest.mark.parametrize("reps", [1, 2, 3])
def test_unaligned_output_vector(reps):
    """An output vector that starts 8 bytes into an allocation (not 16-byte
    aligned, which the bulk copies of the row tiles need) gives the same bits as
    an aligned one: only matrix slices and staged receive buffers are ever
    copied in bulk, never the caller's vectors."""
    A = I.poisson3d(20)
    v = I.vector(A.n, 71)
    plan = gpu_plan(A, 40, 4)
    vd = torch.from_numpy(v).cuda()
    buf = torch.full((A.n + 1,), float("nan"), dtype=torch.float64, device="cuda")
    w_odd = buf[1:]
    assert w_odd.data_ptr() % 16 == 8
    o = nap.make_opts(engine=nap.ENGINE_OVERLAP, vec=1)
    nap.napspmv_apply_ex(plan, vd, w_odd, reps, 0.5, o)
    assert nap.napspmv_status(plan) == 0
    aligned = run(plan, v, reps=reps, scale=0.5, engine=nap.ENGINE_OVERLAP, vec=1)
    assert np.array_equal(w_odd.cpu().numpy(), aligned)
    ref = oracle_chain(A, v, reps, 0.5)
    assert np.linalg.norm(aligned - ref) <= 1e-13 * reps * np.linalg.norm(ref)


@pytest.mark.parametrize("eng", ENGINES)
def test_fp32_narrowing_rounding_cases(eng):
    """x rounded to FP32 before the product: exact halfway cases (ties to
    even, up and down), cases just off a tie, the carry into the exponent, the
    largest finite FP32 value and its halfway point to infinity, the smallest
    normal FP32 exponent and values just below it, compared bit for bit with
    the oracle's C conversion through rows of one entry of value 1."""
    t = 2.0 ** -24
    x = np.array([1 + t, 1 + 3 * t, 1 + t + 2.0 ** -40, 1 + t - 2.0 ** -40, -(1 + t),
                  -(1 + 3 * t), 2 - t, 2 - t / 2, 3.4028234663852886e38,
                  3.4028235677973366e38, 3.4028235677973362e38, 2.0 ** -126 * (1 + t),
                  2.0 ** -126 * (1 + 3 * t), 2.0 ** -126 - 2.0 ** -150, 2.0 ** -149 * 1.5,
                  0.1, -1.0 / 3.0, 7.0e-39])
    n = len(x)
    A = I.CSR(np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), np.ones(n))
    w = run(gpu_plan(A, 6, 2), x, precision=nap.PREC_F32, **eng)
    with np.errstate(all="ignore"):
        ref = O.spmv_f32(A.row_ptr, A.col, np.ones(n, np.float32), x)
    assert np.array_equal(w.view(np.uint64), ref.view(np.uint64)), (w, ref)
    with np.errstate(all="ignore"):
        assert np.array_equal(ref, x.astype(np.float32).astype(np.float64))


def test_host_entry_point():
    A = I.poisson2d(40)
    v = I.vector(A.n, 4)
    plan = gpu_plan(A, 10, 2)
    w = np.zeros(A.n)
    nap.napspmv_apply_host(plan, v, w, 3, 0.125)
    ref = oracle_chain(A, v, 3, 0.125)
    assert np.linalg.norm(w - ref) <= 3e-13 * np.linalg.norm(ref)


@pytest.mark.parametrize("cfg", [1, 2, 3])
def test_workloads_full_size(cfg):
    """Full-size stencil workloads, default (bench) launch options, one apply;
    every output element compared."""
    w_ = I.workload(cfg)
    A = w_.build()
    v = I.vector(A.n, w_.seed)
    plan = gpu_plan(A, w_.n_p, w_.ppn)
    w = run(plan, v)
    assert_close_fp64(w, O.spmv(A.row_ptr, A.col, A.val, v), abs_row_bound(A, v))


def test_config4_full_size():
    """The 2^23-row banded random workload at full size (n_p 8192, ppn 32,
    ~1.7e8 stored entries) with its default launch options (overlapped engine,
    sliced rows, occupancy maximum): one apply and a 3-apply chain, every output
    element compared with the oracle; the warp pipeline (two lanes per row) too."""
    w_ = I.workload(4)
    A = w_.build()
    v = I.vector(A.n, w_.seed)
    plan = gpu_plan(A, w_.n_p, w_.ppn)
    d = nap.napspmv_get_default_opts(plan)
    assert (d.vec, d.pipeline, d.ctas_per_sm) == (2, nap.PIPELINE_SELL, 0)
    ref1 = O.spmv(A.row_ptr, A.col, A.val, v)
    bound = abs_row_bound(A, v)
    w = run(plan, v)
    assert_close_fp64(w, ref1, bound)
    w = run(plan, v, pipeline=nap.PIPELINE_WARP, ctas_per_sm=3)
    assert_close_fp64(w, ref1, bound)
    w = run(plan, v, reps=3, scale=1.0 / 64.0)
    ref = oracle_chain(A, v, 3, 1.0 / 64.0)
    assert np.linalg.norm(w - ref) <= 3e-13 * np.linalg.norm(ref)


def test_config2_chain_bench_configuration():
    """The 3D 7-point 128^3 workload's chain: 100 chained applies x <- A x / 16 in
    the benchmark's launch configuration (default engine, one graph-captured
    chain); every element compared with the oracle's chain against a per-row
    bound carried through the 100 applies.

    Bound: both chains round each row sum of at most L = 7 products with error
    <= gamma s (|A| |x_k|)_i, gamma = L u / (1 - L u), u = 2^-53 (the scale 1/16
    is exact).  An error e_k in x_k reaches x_{k+1} as s |A| |e_k|, so the two
    chains differ by at most b_K, with b_0 = 0 and
    b_{k+1} = s |A| b_k + 2 gamma s |A| |x_k| (x_k: the oracle's iterate, widened
    by b_k to cover the other chain's)."""
    w_ = I.workload(2)
    A = w_.build()
    v = I.vector(A.n, w_.seed)
    plan = gpu_plan(A, w_.n_p, w_.ppn)
    reps, s = 100, 1.0 / 16.0
    w = run(plan, v, reps=reps, scale=s)
    L = int(np.max(np.diff(A.row_ptr)))
    u = 2.0 ** -53
    gamma = L * u / (1 - L * u)
    absA = np.abs(A.val)
    x = v.copy()
    b = np.zeros_like(v)
    for _ in range(reps):
        b = s * O.spmv(A.row_ptr, A.col, absA, b) + \
            2.0 * gamma * s * O.spmv(A.row_ptr, A.col, absA, np.abs(x) + b)
        x = s * O.spmv(A.row_ptr, A.col, A.val, x)
    err = np.abs(w - x)
    assert np.all(err <= b * (1 + 1e-6) + 1e-300), float(np.max(err / (b + 1e-300)))
    assert np.linalg.norm(w - x) <= 1e-12 * np.linalg.norm(x)


def test_config3_fp32_error_stated():
    """Config 3 (rotated anisotropic Q1, 2048^2): FP32-stored values stay within
    1e-6 (normwise) of the FP64 oracle."""
    w_ = I.workload(3)
    A = w_.build()
    v = I.vector(A.n, w_.seed)
    plan = gpu_plan(A, w_.n_p, w_.ppn)
    w = run(plan, v, precision=nap.PREC_F32)
    ref = O.spmv(A.row_ptr, A.col, A.val, v)
    rel = np.linalg.norm(w - ref) / np.linalg.norm(ref)
    assert rel <= 1e-6, rel
