"""Seeded random draws of matrix and launch options (engine, precision, lanes
per row, CTA, warp or sliced-row tiles, tile shape, staged receive buffers, chain length,
partition and mapping flags): every apply matches the oracle within the FP64 bound, or the
oracle's FP32-value product within 1e-13 in FP32 mode."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import abs_row_bound, assert_close_fp64, oracle_chain
from paper_1612_08060_gb300 import inputs as I
from paper_1612_08060_gb300 import napspmv as nap

pytestmark = pytest.mark.gpu

ENGINES = [nap.ENGINE_FUSED, nap.ENGINE_PHASED, nap.ENGINE_OVERLAP]


def _matrix(rng):
    kind = int(rng.integers(0, 3))
    if kind == 0:
        n = int(rng.integers(1, 600))
        return I.random_pattern(n, float(rng.choice([0.005, 0.02, 0.1])),
                                int(rng.integers(0, 2**31 - 1)), diag=bool(rng.random() < 0.8))
    if kind == 1:
        return I.banded_random(int(rng.integers(100, 20000)), int(rng.integers(0, 2**31 - 1)))
    side = int(rng.integers(2, 40))
    return I.poisson3d(side) if rng.random() < 0.5 else I.poisson2d(side * 3)


def _draws(count=60, seed=4242):
    rng = np.random.default_rng(seed)
    for q in range(count):
        A = _matrix(rng)
        n_p = int(rng.integers(1, min(A.n, 300) + 1))
        ppn = int(rng.integers(1, 17))
        flags = int(rng.choice([0, 0, nap.MAP_TEXT, nap.MAP_MAJORITY, nap.PARTITION_STRIDED,
                                nap.MAP_SPLIT]))
        eng = int(rng.choice(ENGINES))
        prec = int(rng.choice([nap.PREC_F64, nap.PREC_F32]))
        opts = dict(engine=eng, precision=prec, vec=int(rng.choice([1, 2, 4, 8, 16, 32])),
                    pipeline=int(rng.choice([nap.PIPELINE_CTA, nap.PIPELINE_WARP, nap.PIPELINE_SELL])),
                    tile_nnz=int(rng.choice([64, 256, 1536])),
                    tile_rows=int(rng.choice([8, 64, 512])),
                    halo=int(rng.choice([nap.HALO_ON, nap.HALO_OFF])))
        reps = 1 if prec == nap.PREC_F32 else int(rng.choice([1, 2, 5]))
        yield q, A, n_p, ppn, flags, opts, reps, int(rng.integers(0, 2**31 - 1))


@pytest.mark.parametrize("draw", list(_draws()), ids=lambda d: f"draw{d[0]}")
def test_random_apply(draw):
    q, A, n_p, ppn, flags, opts, reps, seed = draw
    plan = nap.napspmv_plan(A.row_ptr, A.col, A.val, n_p, ppn, flags | nap.F32_VALUES)
    v = I.vector(A.n, seed)
    vd = torch.from_numpy(v).cuda()
    wd = torch.full_like(vd, float("nan"))
    nap.napspmv_apply_ex(plan, vd, wd, reps, 0.5, nap.make_opts(**opts))
    assert nap.napspmv_status(plan) == nap.OK
    w = wd.cpu().numpy()
    if opts["precision"] == nap.PREC_F32:
        ref32 = 0.5 * O.spmv_f32(A.row_ptr, A.col, A.val.astype(np.float32), v)
        assert np.linalg.norm(w - ref32) <= 1e-13 * np.linalg.norm(ref32) + 1e-300, opts
    elif reps == 1:
        ref = 0.5 * O.spmv(A.row_ptr, A.col, A.val, v)
        assert_close_fp64(w, ref, 0.5 * abs_row_bound(A, v))
    else:
        ref = oracle_chain(A, v, reps, 0.5)
        assert np.linalg.norm(w - ref) <= 1e-13 * reps * np.linalg.norm(ref) + 1e-300, opts
