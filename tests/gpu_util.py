"""Helpers shared by the GPU tests: run the CUDA path through the C ABI and
compare it with the oracle."""
import numpy as np

import oracle as O
from paper_1612_08060_gb300 import napspmv as nap

LISTS = [(nap.LIST_STD, O.STD), (nap.LIST_NODE, O.NODE), (nap.LIST_INTER, O.INTER),
         (nap.LIST_J0, O.J0), (nap.LIST_J1, O.J1), (nap.LIST_J2, O.J2),
         (nap.LIST_BLL, O.BLL), (nap.LIST_BNL, O.BNL), (nap.LIST_LBUF, O.LBUF)]


def gpu_plan(A, n_p, ppn, flags=nap.F32_VALUES):
    return nap.napspmv_plan(A.row_ptr, A.col, A.val, n_p, ppn, flags)


def assert_plans_equal(gp, op):
    """Bit-exact comparison of every exported array and every statistic."""
    for gw, ow in LISTS:
        g = nap.export_list(gp, gw)
        o = op.list(ow)
        for name, a, b in zip(("src", "dst", "ptr", "idx"), g, o):
            assert np.array_equal(a, b), (O.LIST_NAMES[ow], name, a[:10], b[:10])
    tu = nap.napspmv_plan_export(gp, nap.LIST_TU)
    m = int(tu[0])
    sp, rp = op.tu()
    assert np.array_equal(tu[1:1 + m], sp) and np.array_equal(tu[1 + m:1 + 2 * m], rp)
    sp = nap.napspmv_plan_export(gp, nap.LIST_SPLIT)
    assert np.array_equal(sp[1:].reshape(-1, 3), op.split())
    gs = nap.napspmv_plan_stats(gp)
    for k, v in op.stats().items():
        assert gs[k] == v, (k, gs[k], v)


def abs_row_bound(A, v):
    """(|A| |v|)_i: the scale of each row's rounding error."""
    return O.spmv(A.row_ptr, A.col, np.abs(A.val), np.abs(v))


def assert_close_fp64(got, ref, scale, rtol=1e-13):
    """Elementwise |got - ref| <= rtol * (|A||v|)_i and normwise relative error
    <= rtol (the FP64 tolerance of the node-aware apply)."""
    err = np.abs(got - ref)
    assert np.all(err <= rtol * scale + 1e-300), float(np.max(err / (scale + 1e-300)))
    nr = np.linalg.norm(ref)
    if nr > 0:
        assert np.linalg.norm(got - ref) <= rtol * nr


def oracle_chain(A, v, reps, scale):
    x = v.copy()
    for _ in range(reps):
        x = O.spmv(A.row_ptr, A.col, A.val, x)
        if scale != 1.0:
            x = scale * x
    return x
