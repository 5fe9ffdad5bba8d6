"""Failure detection without a GPU fault: a dependency wait that nothing
satisfies (the debug_stall hook makes the first work item wait on a counter no
item increments) ends after timeout_ms with NAPSPMV_ERR_TIMEOUT, the context
stays usable and the next apply is correct."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import abs_row_bound, assert_close_fp64, gpu_plan
from paper_1612_08060_gb300 import inputs as I
from paper_1612_08060_gb300 import napspmv as nap

pytestmark = pytest.mark.gpu


def test_stalled_wait_times_out_and_recovers():
    A = I.poisson2d(32)
    plan = gpu_plan(A, 8, 2)
    v = I.vector(A.n, 1)
    vd = torch.from_numpy(v).cuda()
    wd = torch.empty_like(vd)
    nap.napspmv_apply_ex(plan, vd, wd, 3, 1.0, nap.make_opts(engine=nap.ENGINE_FUSED, debug_stall=1, timeout_ms=100))
    assert nap.napspmv_status(plan) == nap.ERR_TIMEOUT
    assert nap.napspmv_status(plan) == nap.OK  # the status was cleared
    nap.napspmv_apply(plan, vd, wd)
    assert nap.napspmv_status(plan) == nap.OK
    assert_close_fp64(wd.cpu().numpy(), O.spmv(A.row_ptr, A.col, A.val, v), abs_row_bound(A, v))


def test_sticky_error_skips_work_until_cleared():
    A = I.poisson2d(16)
    plan = gpu_plan(A, 4, 2)
    vd = torch.ones(A.n, dtype=torch.float64, device="cuda")
    wd = torch.full_like(vd, 7.0)
    nap.napspmv_apply_ex(plan, vd, wd, 1, 1.0, nap.make_opts(engine=nap.ENGINE_FUSED, debug_stall=1, timeout_ms=50))
    torch.cuda.synchronize()
    w2 = torch.full_like(vd, 7.0)
    nap.napspmv_apply(plan, vd, w2)  # (default engine) sees the sticky flag, does no work
    nap.napspmv_apply_ex(plan, vd, w2, 2, 1.0, nap.make_opts(engine=nap.ENGINE_FUSED))
    assert nap.napspmv_status(plan) == nap.ERR_TIMEOUT
    assert torch.all(w2 == 7.0)


def test_stalled_job_leaves_the_rest_of_a_batch_intact():
    """In one fused launch over several jobs, the stalled job (the one that owns
    the first ticket) reports ERR_TIMEOUT; the others finish with the bits they
    have alone and report OK."""
    mats = [(I.poisson3d(16), 16, 4), (I.poisson2d(60), 20, 4), (I.poisson3d(12), 8, 2)]
    plans = [gpu_plan(A, n_p, ppn) for (A, n_p, ppn) in mats]
    vs = [torch.from_numpy(I.vector(A.n, 40 + k)).cuda() for k, (A, _, _) in enumerate(mats)]
    outs = [torch.full_like(v, float("nan")) for v in vs]
    stall = nap.make_opts(engine=nap.ENGINE_FUSED, debug_stall=1, timeout_ms=100)
    nap.napspmv_apply_batch(plans, vs, outs, [2, 2, 2], [0.25] * 3, opts=stall)
    assert nap.napspmv_status(plans[0]) == nap.ERR_TIMEOUT
    opts = nap.make_opts(engine=nap.ENGINE_FUSED)
    for k in (1, 2):
        assert nap.napspmv_status(plans[k]) == nap.OK
        alone = torch.empty_like(vs[k])
        nap.napspmv_apply_ex(plans[k], vs[k], alone, 2, 0.25, opts)
        torch.cuda.synchronize()
        assert torch.equal(alone, outs[k]), k
    # the stalled job's plan is usable again once its status was read
    nap.napspmv_apply_ex(plans[0], vs[0], outs[0], 1, 1.0, opts)
    assert nap.napspmv_status(plans[0]) == nap.OK
    A = mats[0][0]
    assert_close_fp64(outs[0].cpu().numpy(), O.spmv(A.row_ptr, A.col, A.val, vs[0].cpu().numpy()),
                      abs_row_bound(A, vs[0].cpu().numpy()))
