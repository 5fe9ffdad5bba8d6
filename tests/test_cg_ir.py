"""CG with iterative refinement (FP32-stored values inside, FP64 residual,
vectors and dots) reaches ||b - A x|| / ||b|| <= 1e-10, the residual recomputed
in FP64 by the oracle from the GPU's x; x agrees with the oracle's FP64 CG
within the condition-number bound."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import gpu_plan
from paper_1612_08060_gb300 import inputs as I
from paper_1612_08060_gb300 import napspmv as nap

pytestmark = pytest.mark.gpu


def _kappa(A):
    """2-norm condition number: closed form for the Dirichlet Laplacians
    (eigenvalues sum over axes of 2 - 2 cos(k pi / (n + 1))), dense otherwise."""
    d = int(round(A.val[A.row_ptr[A.n // 2]:A.row_ptr[A.n // 2 + 1]].max()))
    dim = {4: 2, 6: 3}.get(d)
    if dim is not None and np.all(np.abs(A.val[A.val < 0] + 1.0) == 0.0):
        n = int(round(A.n ** (1.0 / dim)))
        lo = dim * (2 - 2 * np.cos(np.pi / (n + 1)))
        hi = dim * (2 + 2 * np.cos(np.pi / (n + 1)))
        return hi / lo
    return np.linalg.cond(A.to_dense())


def _relres(A, x, b):
    return np.linalg.norm(b - O.spmv(A.row_ptr, A.col, A.val, x)) / np.linalg.norm(b)


@pytest.mark.parametrize("A,n_p,ppn", [(I.poisson2d(64), 16, 4), (I.poisson3d(24), 7, 3),
                                        (I.aniso_q1(48), 12, 4)])
def test_cg_ir_reaches_1e10(A, n_p, ppn):
    b = I.vector(A.n, 77)
    plan = gpu_plan(A, n_p, ppn)
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd)
    info = nap.napspmv_cg_ir(plan, bd, xd, rtol=1e-10, inner_rtol=1e-4)
    x = xd.cpu().numpy()
    assert info["converged"] == 1
    assert info["outer_iters"] >= 1
    rr = _relres(A, x, b)
    assert rr <= 1e-10, rr
    assert abs(rr - info["relres"]) <= 1e-12
    x_ref, _, rref = O.cg(A.row_ptr, A.col, A.val, b, rtol=1e-12)
    kappa = _kappa(A)
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) <= kappa * 2e-10


def test_cg_fp64_matches_oracle_iterations():
    A = I.poisson2d(40)
    b = I.vector(A.n, 5)
    plan = gpu_plan(A, 8, 2)
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd)
    info = nap.napspmv_cg(plan, bd, xd, rtol=1e-10)
    _, it_ref, _ = O.cg(A.row_ptr, A.col, A.val, b, rtol=1e-10)
    assert info["converged"] == 1
    assert _relres(A, xd.cpu().numpy(), b) <= 1e-10
    # polled every 8 iterations: the GPU may run up to 7 past the oracle's count
    assert it_ref <= info["inner_iters"] <= it_ref + 8


def test_cg_ir_larger_poisson():
    A = I.poisson2d(256)
    b = I.vector(A.n, 3)
    plan = gpu_plan(A, 32, 16)
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd)
    info = nap.napspmv_cg_ir(plan, bd, xd, rtol=1e-10, inner_rtol=1e-5)
    assert info["converged"] == 1
    assert _relres(A, xd.cpu().numpy(), b) <= 1e-10


def test_dot_is_deterministic_and_exact_enough():
    rng = np.random.default_rng(1)
    for n in (0, 1, 255, 256 * 1024 + 7, 3_000_001):
        x = rng.uniform(-1, 1, n)
        y = rng.uniform(-1, 1, n)
        xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
        r1 = torch.zeros(1, dtype=torch.float64, device="cuda")
        r2 = torch.zeros_like(r1)
        nap.napspmv_dot(xd, yd, n, r1)
        nap.napspmv_dot(xd, yd, n, r2)
        torch.cuda.synchronize()
        assert r1.item() == r2.item()
        ref = float(np.dot(x, y)) if n else 0.0
        assert abs(r1.item() - ref) <= 1e-13 * max(1.0, float(np.abs(x) @ np.abs(y)))
