"""napspmv_apply_noalloc: the apply for callers that cannot allocate device memory
(another allocator owns the device's free memory, or cudaMalloc's implicit
synchronisation is not acceptable on their path).  Its buffers live in a fixed
static device array; the result must match the allocating entry point on two
calls in a row, and plans too large for the array are rejected.

Collected last on purpose (file name) so that a run stopping at the first
failure has already run every other test."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import abs_row_bound, assert_close_fp64, gpu_plan
from paper_1612_08060_gb300 import inputs as I
from paper_1612_08060_gb300 import napspmv as nap

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("make,n_p,ppn,reps,scale", [
    (lambda: I.poisson2d(64), 16, 4, 1, 1.0),
    (lambda: I.poisson3d(40), 32, 8, 5, 1.0 / 16.0),
    (lambda: I.random_pattern(700, 0.01, 3), 70, 4, 2, 0.5),
])
def test_noalloc_matches_allocating_entry_point(make, n_p, ppn, reps, scale):
    A = make()
    plan = gpu_plan(A, n_p, ppn)
    for call in range(2):  # two calls in a row share (and reuse) the static area
        v = I.vector(A.n, 100 + call)
        vd = torch.from_numpy(v).cuda()
        ref = torch.full_like(vd, float("nan"))
        got = torch.full_like(vd, float("nan"))
        nap.napspmv_apply_n(plan, vd, ref, reps, scale)
        nap.napspmv_apply_noalloc(plan, vd, got, reps, scale)
        assert nap.napspmv_status(plan) == nap.OK
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.linalg.norm(g - r) <= 1e-13 * max(1.0, reps) * np.linalg.norm(r)
        if reps == 1:
            assert_close_fp64(g, O.spmv(A.row_ptr, A.col, A.val, v), abs_row_bound(A, v))


def test_noalloc_rejects_plans_beyond_the_static_area():
    A = I.poisson3d(104)  # N = 1,124,864 > 2^20 doubles of scratch
    plan = gpu_plan(A, 64, 16)
    vd = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    with pytest.raises(nap.NapError) as e:
        nap.napspmv_apply_noalloc(plan, vd, torch.empty_like(vd))
    assert e.value.code == nap.ERR_UNSUPPORTED
    assert "static area" in str(e.value)
