"""One persistent launch over several independent applies (different matrices,
sizes, chain lengths, and one plan twice with two workspaces): every result is
bit-identical to the same apply run alone, and matches the oracle."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import gpu_plan, oracle_chain
from paper_1612_08060_gb300 import inputs as I
from paper_1612_08060_gb300 import napspmv as nap

pytestmark = pytest.mark.gpu


def test_batch_equals_alone():
    mats = [(I.poisson2d(50), 10, 4, 1, 1.0), (I.poisson3d(17), 9, 2, 4, 1 / 12),
            (I.aniso_q1(33), 33, 16, 2, 0.5), (I.random_pattern(300, 0.03, 4), 30, 3, 1, 1.0)]
    plans = [gpu_plan(A, n_p, ppn) for (A, n_p, ppn, _, _) in mats]
    # second use of the first plan through its own workspace
    plans.append(plans[0])
    mats.append(mats[0][:3] + (3, 0.25))
    wss = [None, None, None, None, nap.Workspace(plans[0])]
    vs = [torch.from_numpy(I.vector(m[0].n, 10 + k)).cuda() for k, m in enumerate(mats)]
    outs = [torch.full_like(v, float("nan")) for v in vs]
    reps = [m[3] for m in mats]
    scales = [m[4] for m in mats]
    opts = nap.make_opts(engine=nap.ENGINE_FUSED, vec=4)  # the batched launch's engine
    nap.napspmv_apply_batch(plans, vs, outs, reps, scales, opts=opts, ws=wss)
    assert nap.napspmv_status(plans[0]) == 0
    assert nap.napspmv_ws_status(wss[4]) == 0
    for k, (A, n_p, ppn, r, s) in enumerate(mats):
        alone = torch.empty_like(vs[k])
        nap.napspmv_apply_ex(plans[k], vs[k], alone, r, s, opts)
        torch.cuda.synchronize()
        assert torch.equal(alone, outs[k]), k
        ref = oracle_chain(A, vs[k].cpu().numpy(), r, s)
        got = outs[k].cpu().numpy()
        assert np.linalg.norm(got - ref) <= 1e-13 * r * np.linalg.norm(ref)


@pytest.mark.parametrize("reps,prec", [(1, nap.PREC_F64), (3, nap.PREC_F64), (1, nap.PREC_F32)])
def test_batch_level_order_equals_alone(reps, prec):
    """Jobs that chain equally many applies take their tickets level by level
    across the batch (every job's message steps, then the row tiles); the bits
    stay those of each apply alone."""
    mats = [(I.poisson3d(24), 27, 4), (I.poisson2d(90), 40, 16), (I.poisson3d(13), 1, 1),
            (I.aniso_q1(40), 64, 8), (I.random_pattern(500, 0.02, 7), 12, 3),
            (I.poisson3d(20), 16, 16)]
    plans = [nap.napspmv_plan(A.row_ptr, A.col, A.val, n_p, ppn, flags=nap.F32_VALUES)
             for (A, n_p, ppn) in mats]
    vs = [torch.from_numpy(I.vector(A.n, 30 + k)).cuda() for k, (A, _, _) in enumerate(mats)]
    outs = [torch.full_like(v, float("nan")) for v in vs]
    opts = nap.make_opts(engine=nap.ENGINE_FUSED, precision=prec)
    nap.napspmv_apply_batch(plans, vs, outs, [reps] * len(mats), [0.125] * len(mats), opts=opts)
    for k, (A, _, _) in enumerate(mats):
        assert nap.napspmv_status(plans[k]) == 0
        alone = torch.empty_like(vs[k])
        nap.napspmv_apply_ex(plans[k], vs[k], alone, reps, 0.125, opts)
        torch.cuda.synchronize()
        assert torch.equal(alone, outs[k]), k
        if prec == nap.PREC_F64:
            ref = oracle_chain(A, vs[k].cpu().numpy(), reps, 0.125)
            got = outs[k].cpu().numpy()
            assert np.linalg.norm(got - ref) <= 1e-13 * reps * np.linalg.norm(ref)


def test_batch_rejects_shared_workspace():
    A = I.poisson2d(10)
    p = gpu_plan(A, 4, 2)
    v = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    with pytest.raises(nap.NapError):
        nap.napspmv_apply_batch([p, p], [v, v], [torch.empty_like(v), torch.empty_like(v)],
                                [1, 1])
