"""Seeded random draws (sizes, densities with empty rows, partitions, every
mapping and partition flag): the GPU plan equals the oracle's bit for bit, and
the default apply matches the oracle's product."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import abs_row_bound, assert_close_fp64, assert_plans_equal
from paper_1612_08060_gb300 import inputs as I
from paper_1612_08060_gb300 import napspmv as nap

pytestmark = pytest.mark.gpu

FLAGS = [0, nap.MAP_TEXT, nap.PARTITION_STRIDED, nap.MAP_MAJORITY,
         nap.PARTITION_STRIDED | nap.MAP_TEXT, nap.PARTITION_STRIDED | nap.MAP_MAJORITY,
         nap.MAP_SPLIT, nap.MAP_SPLIT | nap.MAP_TEXT, nap.PARTITION_STRIDED | nap.MAP_SPLIT]


# the library's and the oracle's flag bits are numbered independently
_TO_ORACLE = {nap.MAP_TEXT: O.MAP_TEXT, nap.PARTITION_STRIDED: O.STRIDED,
              nap.MAP_MAJORITY: O.MAP_MAJORITY, nap.MAP_SPLIT: O.MAP_SPLIT}


def _oracle_flags(flags):
    return sum(o for g, o in _TO_ORACLE.items() if flags & g)


def _draws(count=80, seed=2024):
    rng = np.random.default_rng(seed)
    for q in range(count):
        n = int(rng.integers(1, 300))
        yield (q, n, float(rng.choice([0.0, 0.01, 0.03, 0.1])), bool(rng.random() < 0.8),
               int(rng.integers(1, n + 1)), int(rng.integers(1, 17)),
               int(FLAGS[rng.integers(0, len(FLAGS))]), int(rng.integers(0, 2**31 - 1)))


@pytest.mark.parametrize("q,n,dens,diag,n_p,ppn,flags,seed", list(_draws()))
def test_random_draw(q, n, dens, diag, n_p, ppn, flags, seed):
    A = I.random_pattern(n, dens, seed, diag=diag)
    gp = nap.napspmv_plan(A.row_ptr, A.col, A.val, n_p, ppn, flags | nap.F32_VALUES)
    op = O.OraclePlan(A.row_ptr, A.col, n_p, ppn, flags=_oracle_flags(flags))
    assert_plans_equal(gp, op)
    v = I.vector(n, seed + 1)
    w = torch.empty(n, dtype=torch.float64, device="cuda")
    nap.napspmv_apply(gp, torch.from_numpy(v).cuda(), w)
    assert nap.napspmv_status(gp) == nap.OK
    assert_close_fp64(w.cpu().numpy(), O.spmv(A.row_ptr, A.col, A.val, v), abs_row_bound(A, v))
