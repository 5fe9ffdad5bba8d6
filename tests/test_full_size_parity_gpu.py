"""Full-size parity of the GPU plans and applies against the oracle for the 2D
rotated anisotropic Q1 2048^2 workload (N = 4,194,304, n_p 4096, ppn 16) and the
2^23-row banded random workload (N = 8,388,608, ~1.68e8 stored entries, n_p 8192,
ppn 32), where the packed plan keys reach their widest (about 1.5e8 standard
(t, j) pairs).

Plans: every exported list (Eqs. P, D, N, E, G, I, IL0-IL2 and the receive
layouts), the T/U assignment, the three-block split and every statistic bit for
bit, for the default mapping (Tables T, U), the majority mapping (the
alternative named after Eq. U) and the strided partition (Sec. 5).

Applies: the banded random workload with FP32-stored values, every element
within 1e-13 (|A32| |fl32(v)|)_i of the oracle's FP32-product / FP64-sum result
and within 1e-6 (|A| |v|)_i of the FP64 product."""
import threading

import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import abs_row_bound, assert_plans_equal, gpu_plan
from paper_1612_08060_gb300 import inputs as I
from paper_1612_08060_gb300 import napspmv as nap

pytestmark = pytest.mark.gpu

FLAGS = [(0, 0), (nap.MAP_MAJORITY, O.MAP_MAJORITY), (nap.PARTITION_STRIDED, O.STRIDED)]


def _oracle_plans(A, n_p, ppn):
    """The oracle's plan for every flag, built in parallel threads (the C
    builder runs without the interpreter lock)."""
    out = {}

    def one(gf, of):
        out[gf] = O.OraclePlan(A.row_ptr, A.col, n_p, ppn, flags=of)

    th = [threading.Thread(target=one, args=f) for f in FLAGS]
    for t in th:
        t.start()
    for t in th:
        t.join()
    return out


def _check_workload(cfg):
    w_ = I.workload(cfg)
    A = w_.build()
    ops = _oracle_plans(A, w_.n_p, w_.ppn)
    for gf, _ in FLAGS:
        gp = gpu_plan(A, w_.n_p, w_.ppn, nap.F32_VALUES | gf)
        assert_plans_equal(gp, ops[gf])
        del gp
        torch.cuda.synchronize()
    return A, w_, ops


def test_config3_plans_full_size():
    _, _, ops = _check_workload(3)
    st = ops[0].stats()
    # the stencil's closed counts (the oracle's own closed-form pins) hold too
    assert (st["std_msgs"], st["std_inter_msgs"], st["nap_inter_msgs"]) == (20472, 2040, 510)
    assert (st["std_inter_vals"], st["nap_inter_vals"]) == (1045500, 1044480)


def test_config4_plans_and_fp32_apply_full_size():
    A, w_, ops = _check_workload(4)
    st = ops[0].stats()
    assert st["std_msgs"] > 2 * 10**7 and st["nap_inter_msgs"] <= (w_.n_p // w_.ppn) ** 2
    # FP32-stored values on the default launch options
    v = I.vector(A.n, w_.seed)
    plan = gpu_plan(A, w_.n_p, w_.ppn)
    vd = torch.from_numpy(v).cuda()
    wd = torch.full_like(vd, float("nan"))
    nap.napspmv_apply_ex(plan, vd, wd, 1, 1.0, nap.make_opts(precision=nap.PREC_F32))
    assert nap.napspmv_status(plan) == nap.OK
    w = wd.cpu().numpy()
    a32 = A.val.astype(np.float32)
    ref32 = O.spmv_f32(A.row_ptr, A.col, a32, v)
    scale32 = O.spmv(A.row_ptr, A.col, np.abs(a32).astype(np.float64),
                     np.abs(v.astype(np.float32)).astype(np.float64))
    err = np.abs(w - ref32)
    assert np.all(err <= 1e-13 * scale32 + 1e-300), float(np.max(err / (scale32 + 1e-300)))
    ref = O.spmv(A.row_ptr, A.col, A.val, v)
    err = np.abs(w - ref)
    scale = abs_row_bound(A, v)
    assert np.all(err <= 1e-6 * scale), float(np.max(err / scale))
    assert np.linalg.norm(w - ref) <= 1e-6 * np.linalg.norm(ref)
