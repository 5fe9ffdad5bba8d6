"""Seeded random batches of 2 to 12 matrices (equal chain lengths, which take the
level-by-level ticket order, or mixed ones, which run job after job; FP64 or
FP32 values): every entry is bit-identical to the same apply alone with the
batch's options.  A batch resolves unset options against its first plan (one
kernel, one lane count per row), so the apply alone is given those options
explicitly: with its own plan's defaults (another lane count for rows of more
than 16 entries) an FP64 sum may round in another order."""
import numpy as np
import pytest
import torch

from paper_1612_08060_gb300 import inputs as I
from paper_1612_08060_gb300 import napspmv as nap

pytestmark = pytest.mark.gpu


def _draws(count=20, seed=777):
    rng = np.random.default_rng(seed)
    for q in range(count):
        k = int(rng.integers(2, 13))
        mats = []
        for _ in range(k):
            if rng.random() < 0.5:
                A = I.random_pattern(int(rng.integers(1, 400)), float(rng.choice([0.01, 0.05])),
                                     int(rng.integers(0, 2**31 - 1)))
            else:
                side = int(rng.integers(3, 30))
                A = I.poisson3d(side) if rng.random() < 0.5 else I.poisson2d(3 * side)
            mats.append((A, int(rng.integers(1, min(A.n, 200) + 1)), int(rng.integers(1, 17))))
        equal = bool(rng.random() < 0.6)
        reps = [int(rng.integers(1, 4))] * k if equal else [int(x) for x in rng.integers(1, 4, k)]
        prec = int(rng.choice([nap.PREC_F64, nap.PREC_F32]))
        yield q, mats, reps, prec


@pytest.mark.parametrize("draw", list(_draws()), ids=lambda d: f"batch{d[0]}")
def test_random_batch(draw):
    q, mats, reps, prec = draw
    plans = [nap.napspmv_plan(A.row_ptr, A.col, A.val, n_p, ppn, nap.F32_VALUES)
             for (A, n_p, ppn) in mats]
    vs = [torch.from_numpy(I.vector(A.n, 100 * q + k)).cuda() for k, (A, _, _) in enumerate(mats)]
    outs = [torch.full_like(v, float("nan")) for v in vs]
    opts = nap.napspmv_get_default_opts(plans[0])
    opts.engine = nap.ENGINE_FUSED
    opts.precision = prec
    nap.napspmv_apply_batch(plans, vs, outs, reps, [0.5] * len(mats), opts=opts)
    for k in range(len(mats)):
        assert nap.napspmv_status(plans[k]) == nap.OK
        alone = torch.empty_like(vs[k])
        nap.napspmv_apply_ex(plans[k], vs[k], alone, reps[k], 0.5, opts)
        torch.cuda.synchronize()
        assert torch.equal(alone, outs[k]), (q, k)
