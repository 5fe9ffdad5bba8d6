"""The seeded input generators follow their stated recipes: the stencil
matrices' sizes and symmetry, the banded random matrix's row-length law, band
fraction and diagonal dominance, the serving request stream, and the workload
table's sizes and partitions.  CPU only."""
import math

import numpy as np
import pytest

from paper_1612_08060_gb300 import inputs as I


def _rows_sorted_unique(A):
    for i in range(A.n):
        c = A.col[A.row_ptr[i]:A.row_ptr[i + 1]]
        assert np.all(np.diff(c) > 0), i


@pytest.mark.parametrize("n", [1, 2, 7, 30])
def test_stencil_sizes_and_symmetry(n):
    A2 = I.poisson2d(n)
    assert A2.n == n * n and A2.nnz == 5 * n * n - 4 * n
    A3 = I.poisson3d(n)
    assert A3.n == n ** 3 and A3.nnz == 7 * n ** 3 - 6 * n * n
    for A in (A2, A3):
        _rows_sorted_unique(A)
        D = A.to_dense()
        assert np.array_equal(D, D.T)


def test_aniso_q1_interior_rows():
    n = 12
    A = I.aniso_q1(n)
    D = A.to_dense()
    assert np.allclose(D, D.T, rtol=0, atol=1e-15)
    lens = np.diff(A.row_ptr).reshape(n, n)
    assert np.all(lens[1:-1, 1:-1] == 9)
    assert lens[0, 0] == 4
    # constants lie in the kernel of the interior stencil (a Q1 stiffness matrix)
    rs = D.sum(axis=1).reshape(n, n)
    assert np.allclose(rs[1:-1, 1:-1], 0.0, atol=1e-14)


def test_banded_random_recipe():
    N, seed = 20000, 77
    A = I.banded_random(N, seed)
    L = np.diff(A.row_ptr)
    assert L.min() >= 4 and L.max() <= 64
    # clip(Poisson(20), 4, 64): the mean sits within a few standard errors of 20
    assert abs(L.mean() - 20.0) < 5 * math.sqrt(20.0 / N)
    _rows_sorted_unique(A)
    rows = np.repeat(np.arange(N), L)
    diag = rows == A.col
    assert np.array_equal(np.bincount(rows[diag], minlength=N), np.ones(N, np.int64))
    off = ~diag
    absum = np.bincount(rows[off], weights=np.abs(A.val[off]), minlength=N)
    assert np.allclose(A.val[diag], 1.0 + absum, rtol=1e-15, atol=0)
    # 80% of the off-diagonal draws land in the band [i - W, i + W], plus the
    # uniform draws that happen to fall inside it (a fraction 2W / N of them)
    W = round(0.005 * N)
    inband = np.abs(A.col[off].astype(np.int64) - rows[off]) <= W
    expect = 0.8 + 0.2 * (2 * W + 1) / N
    assert abs(inband.mean() - expect) < 0.01
    # the same seed gives the same matrix
    B = I.banded_random(N, seed)
    assert np.array_equal(A.row_ptr, B.row_ptr) and np.array_equal(A.col, B.col)
    assert np.array_equal(A.val, B.val)


def test_vector_is_seeded_uniform():
    v = I.vector(10000, 3)
    assert np.array_equal(v, I.vector(10000, 3))
    assert not np.array_equal(v, I.vector(10000, 4))
    assert v.min() >= -1.0 and v.max() <= 1.0 and abs(v.mean()) < 0.05


def test_serving_request_stream():
    count, rate = 4000, 50.0
    R = I.serving_requests(count, rate, seed=11, n_lo=1e3, n_hi=2e6, p_spmv=0.7)
    t = np.array([r["arrival"] for r in R])
    assert np.all(np.diff(t) > 0)
    # Poisson arrivals: exponential gaps of mean 1 / rate
    assert abs(np.diff(t).mean() * rate - 1.0) < 0.1
    kinds = np.array([r["kind"] == "spmv" for r in R])
    assert abs(kinds.mean() - 0.7) < 4 * math.sqrt(0.21 / count)
    for r in R:
        assert r["n"] == r["side"] ** r["dim"] and r["dim"] in (2, 3)
        assert r["n_p"] == max(1, round(r["n"] / 2048)) and r["ppn"] == 16
        # N log-uniform in [1e3, 2e6] before rounding the side to an integer
        lo = max(2, round(1e3 ** (1 / r["dim"]))) ** r["dim"]
        hi = round(2e6 ** (1 / r["dim"])) ** r["dim"]
        assert lo <= r["n"] <= hi
    logn = np.log([r["n"] for r in R])
    assert abs(np.median(logn) - 0.5 * (math.log(1e3) + math.log(2e6))) < 0.2


def test_workload_table():
    w1, w2, w3, w4 = (I.workload(c) for c in (1, 2, 3, 4))
    assert (w1.n_p, w1.ppn) == (16, 4)
    assert (w2.n_p, w2.ppn) == (1024, 16) and w2.name.startswith("poisson3d_7pt_128^3")
    assert (w3.n_p, w3.ppn) == (4096, 16) and "2048^2" in w3.name
    assert (w4.n_p, w4.ppn) == (8192, 32) and "N8388608" in w4.name
    assert I.workload(1).build().n == 64 * 64
    small = I.workload(2, scale_down=8)
    assert small.build().n == 16 ** 3 and small.n_p == 2
    with pytest.raises(ValueError):
        I.workload(5)
