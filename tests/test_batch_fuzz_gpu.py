"""Seeded random batches of 2 to 12 matrices (equal chain lengths, which take the
level-by-level ticket order, or mixed ones, which run job after job; FP64 or
FP32 values): every entry is bit-identical to the same apply alone on the fused
engine with that entry's resolved options.  A batch resolves the option fields
it is not given against each entry's own plan and runs one fused launch per
distinct option set; given every field (here: the first plan's defaults), all
entries share those options and one launch."""
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
        own = bool(rng.random() < 0.5)  # only engine and precision given
        yield q, mats, reps, prec, own


@pytest.mark.parametrize("draw", list(_draws()), ids=lambda d: f"batch{d[0]}")
def test_random_batch(draw):
    q, mats, reps, prec, own = draw
    plans = [nap.napspmv_plan(A.row_ptr, A.col, A.val, n_p, ppn, nap.F32_VALUES)
             for (A, n_p, ppn) in mats]
    # a few rows of about 20 entries: another lane count by default
    if own and q % 2 == 0:
        B = I.banded_random(3000, 1000 + q)
        mats.append((B, 6, 2))
        plans.append(nap.napspmv_plan(B.row_ptr, B.col, B.val, 6, 2, nap.F32_VALUES))
        reps = reps + [reps[-1]]
    vs = [torch.from_numpy(I.vector(A.n, 100 * q + k)).cuda() for k, (A, _, _) in enumerate(mats)]
    outs = [torch.full_like(v, float("nan")) for v in vs]
    if own:
        opts = nap.make_opts(engine=nap.ENGINE_FUSED, precision=prec)
    else:
        opts = nap.napspmv_get_default_opts(plans[0])
        opts.engine = nap.ENGINE_FUSED
        opts.precision = prec
    nap.napspmv_apply_batch(plans, vs, outs, reps, [0.5] * len(mats), opts=opts)
    for k in range(len(mats)):
        assert nap.napspmv_status(plans[k]) == nap.OK
        alone = torch.empty_like(vs[k])
        if own:
            o = nap.napspmv_get_default_opts(plans[k])
            o.engine = nap.ENGINE_FUSED
            o.precision = prec
        else:
            o = opts
        nap.napspmv_apply_ex(plans[k], vs[k], alone, reps[k], 0.5, o)
        torch.cuda.synchronize()
        assert torch.equal(alone, outs[k]), (q, k)
