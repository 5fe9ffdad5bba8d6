"""The autotuner picks launch options by measurement, installs them as the plan's
defaults, caches them per matrix key, and the tuned plan still matches the oracle."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import abs_row_bound, assert_close_fp64, gpu_plan
from paper_1612_08060_gb300 import autotune
from paper_1612_08060_gb300 import inputs as I
from paper_1612_08060_gb300 import napspmv as nap

pytestmark = pytest.mark.gpu


def test_tune_installs_and_caches(monkeypatch, tmp_path):
    monkeypatch.setattr(autotune, "CANDIDATES", {
        "engine": [nap.ENGINE_OVERLAP, nap.ENGINE_FUSED], "vec": [1, 2],
        "tile_nnz": [1024, 1536], "tile_rows": [256, 512], "stages": [2], "chunk": [2048]})
    monkeypatch.setattr(autotune, "_cache", {})
    A = I.poisson3d(32)
    plan = gpu_plan(A, 16, 4)
    cache = tmp_path / "tune.json"
    best, ms = autotune.tune(plan, A.row_ptr, reps=4, max_sweeps=1, cache_file=str(cache))
    assert ms > 0 and cache.exists()
    d = nap.napspmv_get_default_opts(plan)
    for k, v in best.items():
        assert getattr(d, k) == v, k
        assert v in autotune.CANDIDATES[k]
    v = I.vector(A.n, 3)
    vd = torch.from_numpy(v).cuda()
    wd = torch.empty_like(vd)
    nap.napspmv_apply(plan, vd, wd)
    assert nap.napspmv_status(plan) == 0
    assert_close_fp64(wd.cpu().numpy(), O.spmv(A.row_ptr, A.col, A.val, v), abs_row_bound(A, v))
    # a second plan of the same matrix takes the cached choice without measuring
    plan2 = gpu_plan(A, 16, 4)
    best2, ms2 = autotune.tune(plan2, A.row_ptr, cache_file=str(cache))
    assert best2 == best and ms2 == ms
