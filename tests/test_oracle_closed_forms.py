"""The CPU oracle against closed forms: stencil row sums, discrete harmonic
functions, exact FP32-product emulation, CG on a known system, and message
counts of the stencil workloads derived from their geometry."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1612_08060_gb300 import inputs as I


def _deg_2d(n):
    g = np.zeros((n, n), int)
    g[1:, :] += 1
    g[:-1, :] += 1
    g[:, 1:] += 1
    g[:, :-1] += 1
    return g.ravel()


def test_poisson2d_row_sums_exact():
    A = I.poisson2d(23)
    w = O.spmv(A.row_ptr, A.col, A.val, np.ones(A.n))
    assert np.array_equal(w, 4.0 - _deg_2d(23))


def test_poisson3d_row_sums_exact():
    n = 9
    A = I.poisson3d(n)
    w = O.spmv(A.row_ptr, A.col, A.val, np.ones(A.n))
    z, y, x = np.indices((n, n, n)).reshape(3, -1)
    deg = sum(((c > 0).astype(int) + (c < n - 1).astype(int)) for c in (x, y, z))
    assert np.array_equal(w, 6.0 - deg)


@pytest.mark.parametrize("dim", [2, 3])
def test_linear_functions_are_harmonic(dim):
    n = 11
    A = I.poisson2d(n) if dim == 2 else I.poisson3d(n)
    c = np.indices((n,) * dim).reshape(dim, -1)  # slowest axis first
    x = sum((k + 2) * c[k] for k in range(dim)).astype(float)
    w = O.spmv(A.row_ptr, A.col, A.val, x)
    interior = np.all((c > 0) & (c < n - 1), axis=0)
    assert np.all(w[interior] == 0.0)
    assert np.any(w[~interior] != 0.0)


def test_q1_aniso_stencil_properties():
    n = 17
    A = I.aniso_q1(n, 0.001, math.pi / 8)
    d = A.to_dense()
    assert np.array_equal(d, d.T)
    w = O.spmv(A.row_ptr, A.col, A.val, np.ones(A.n))
    y, x = np.indices((n, n)).reshape(2, -1)
    interior = (x > 0) & (x < n - 1) & (y > 0) & (y < n - 1)
    assert np.max(np.abs(w[interior])) < 1e-15
    # eps = 1, theta = 0: the textbook Q1 Laplacian (1/3) [8 centre, -1 x 8]
    B = I.aniso_q1(n, 1.0, 0.0)
    mid = (n // 2) * n + n // 2
    row = B.val[B.row_ptr[mid]:B.row_ptr[mid + 1]]
    cols = B.col[B.row_ptr[mid]:B.row_ptr[mid + 1]]
    assert len(row) == 9
    np.testing.assert_allclose(row[cols == mid], [8.0 / 3.0], rtol=1e-15)
    np.testing.assert_allclose(row[cols != mid], [-1.0 / 3.0] * 8, rtol=1e-15)


def test_spmv_f32_exact_emulation():
    A = I.random_pattern(30, 0.2, 5)
    v = I.vector(30, 6)
    val32 = A.val.astype(np.float32)
    w = O.spmv_f32(A.row_ptr, A.col, val32, v)
    for i in range(A.n):
        s = 0.0
        for k in range(A.row_ptr[i], A.row_ptr[i + 1]):
            p = np.float32(val32[k]) * np.float32(v[A.col[k]])  # IEEE single product
            s += float(p)
        assert w[i] == s


def test_spmv_f32_error_bound():
    A = I.aniso_q1(64)
    v = I.vector(A.n, 7)
    w64 = O.spmv(A.row_ptr, A.col, A.val, v)
    w32 = O.spmv_f32(A.row_ptr, A.col, A.val.astype(np.float32), v)
    absAv = O.spmv(A.row_ptr, A.col, np.abs(A.val), np.abs(v))
    u32 = 2.0 ** -24
    assert np.all(np.abs(w32 - w64) <= 3.01 * u32 * absAv + 1e-300)
    rel = np.linalg.norm(w32 - w64) / np.linalg.norm(w64)
    assert rel <= 1e-6


def test_cg_solves_poisson():
    A = I.poisson2d(20)
    b = I.vector(A.n, 8)
    x, it, rr = O.cg(A.row_ptr, A.col, A.val, b, rtol=1e-12)
    assert rr <= 1e-12
    assert it < A.n
    x_ref = np.linalg.solve(A.to_dense(), b)
    kappa = np.linalg.cond(A.to_dense())
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) <= kappa * 1e-12


def test_cg_zero_iterations_from_solution():
    A = I.poisson2d(8)
    x_ref = I.vector(A.n, 9)
    b = A.to_dense() @ x_ref
    x, it, rr = O.cg(A.row_ptr, A.col, A.val, b, x0=np.linalg.solve(A.to_dense(), b),
                     rtol=1e-8)
    assert it == 0 and rr <= 1e-8


# ---------------------------------------------------------------- message counts
# Closed forms from the stencil geometry (natural ordering, contiguous rows):

def counts_2d5(n, n_p, ppn):
    """Ranks hold whole grid lines: rank r exchanges its boundary lines (n values)
    with r-1 and r+1 only."""
    nn = n_p // ppn
    std = 2 * (n_p - 1)
    inter = 2 * (nn - 1)
    return dict(std_msgs=std, std_inter_msgs=inter, std_intra_msgs=std - inter,
                std_inter_vals=inter * n, nap_inter_msgs=2 * (nn - 1),
                nap_inter_vals=2 * (nn - 1) * n)


def counts_3d7(n, f, g):
    """f ranks per z-plane (n/f lines each), g planes per node: y-neighbours in a
    plane exchange one line, z-neighbours a whole rank (n^2/f values)."""
    std = n * 2 * (f - 1) + 2 * (n - 1) * f
    inter = 2 * (n // g - 1) * f
    return dict(std_msgs=std, std_inter_msgs=inter, std_intra_msgs=std - inter,
                std_inter_vals=2 * (n // g - 1) * n * n, nap_inter_msgs=2 * (n // g - 1),
                nap_inter_vals=2 * (n // g - 1) * n * n)


def counts_q1(n, ppn):
    """Half a grid line per rank, ppn/2 lines per node, 9-point couplings: an
    interior rank talks to its other half and to both halves of the lines above
    and below (5 messages); across a node boundary each direction carries two
    half-lines (n/2 values each) and two single corner values."""
    nn = 2 * n // ppn
    inter = 8 * (nn - 1)
    return dict(std_msgs=10 * n - 8, std_inter_msgs=inter, std_intra_msgs=10 * n - 8 - inter,
                std_inter_vals=(nn - 1) * (2 * n + 4), nap_inter_msgs=2 * (nn - 1),
                nap_inter_vals=2 * (nn - 1) * n)


def _check(A, n_p, ppn, want):
    s = O.OraclePlan(A.row_ptr, A.col, n_p, ppn).stats()
    for k, v in want.items():
        assert s[k] == v, (k, s[k], v)
    return s


def test_counts_config1_full():
    """2D 5-point 64 x 64, n_p = 16, ppn = 4: 30 messages (24 intra / 6 inter),
    384 inter-node values; node-aware: 6 messages, 384 values."""
    want = counts_2d5(64, 16, 4)
    assert (want["std_msgs"], want["std_intra_msgs"], want["std_inter_msgs"]) == (30, 24, 6)
    assert (want["std_inter_vals"], want["nap_inter_msgs"], want["nap_inter_vals"]) == \
        (384, 6, 384)
    _check(I.poisson2d(64), 16, 4, want)


def test_counts_full_size_closed_forms():
    """The full stencil workloads' numbers from the same formulas."""
    c2 = counts_3d7(128, 8, 2)
    assert (c2["std_msgs"], c2["std_intra_msgs"], c2["std_inter_msgs"]) == (3824, 2816, 1008)
    assert (c2["std_inter_vals"], c2["nap_inter_msgs"], c2["nap_inter_vals"]) == \
        (2064384, 126, 2064384)
    c3 = counts_q1(2048, 16)
    assert (c3["std_msgs"], c3["std_intra_msgs"], c3["std_inter_msgs"]) == (20472, 18432, 2040)
    assert (c3["std_inter_vals"], c3["nap_inter_msgs"], c3["nap_inter_vals"]) == \
        (1045500, 510, 1044480)


@pytest.mark.parametrize("n,f,g", [(16, 4, 2), (24, 8, 2), (32, 8, 4), (20, 5, 1)])
def test_counts_3d7_scaled(n, f, g):
    _check(I.poisson3d(n), n * f, f * g, counts_3d7(n, f, g))


@pytest.mark.parametrize("n,ppn", [(32, 16), (64, 16), (48, 8), (40, 4)])
def test_counts_q1_scaled(n, ppn):
    _check(I.aniso_q1(n), 2 * n, ppn, counts_q1(n, ppn))


@pytest.mark.parametrize("n,n_p,ppn", [(40, 8, 2), (30, 10, 5), (64, 64, 8)])
def test_counts_2d5_scaled(n, n_p, ppn):
    _check(I.poisson2d(n), n_p, ppn, counts_2d5(n, n_p, ppn))


@pytest.mark.slow
def test_counts_config2_full():
    w = I.workload(2)
    _check(w.build(), w.n_p, w.ppn, counts_3d7(128, 8, 2))


@pytest.mark.parametrize("n,f,g", [(16, 2, 2), (24, 2, 4), (32, 4, 2), (21, 2, 3)])
def test_split_counts_3d7_closed_form(n, f, g):
    """Node splitting (reading R20) on a 3D 7-point stencil whose nodes hold g whole
    planes (f processes a plane, ppn = f g): an inner node has the two neighbouring
    nodes as partners, so each partner gets a group of ppn / 2 processes and an
    inner pair carries ppn / 2 pieces; the first and last node have one partner and
    a group of all ppn processes, so the 4 pairs touching them carry ppn pieces.
    Every piece is non-empty (a pair exchanges a whole plane), and splitting moves
    the same values."""
    A = I.poisson3d(n)
    n_p, ppn = n * f, f * g
    nodes = n_p // ppn
    plain = O.OraclePlan(A.row_ptr, A.col, n_p, ppn).stats()
    split = O.OraclePlan(A.row_ptr, A.col, n_p, ppn, flags=O.MAP_SPLIT).stats()
    pairs = 2 * (nodes - 1)
    assert plain["nap_inter_msgs"] == pairs
    assert split["nap_inter_vals"] == plain["nap_inter_vals"] == pairs * n * n
    assert split["nap_inter_msgs"] == (ppn // 2) * (pairs - 4) + ppn * 4
