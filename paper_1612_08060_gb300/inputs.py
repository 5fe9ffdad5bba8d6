"""Seeded synthetic inputs shaped like the paper's workloads.

This module only builds inputs (CSR matrices, vectors, request streams).  It holds
none of the node-aware SpMV's arithmetic, so both the CUDA path and the CPU oracle
take their inputs from here.  Everything is numpy, seeded with PCG64
(``numpy.random.default_rng``).

Matrices are CSR with int64 row pointers, int32 columns (ascending within a row)
and float64 values:

* ``poisson2d(n)``   2D 5-point Laplacian on an n x n grid, natural (x-fastest)
  ordering, Dirichlet rows truncated: 4 on the diagonal, -1 per neighbour.
* ``poisson3d(n)``   3D 7-point Laplacian on n^3, natural ordering: 6 / -1.
* ``aniso_q1(n, eps, theta)``  rotated anisotropic diffusion, bilinear (Q1)
  9-point stencil with K = R(theta) diag(1, eps) R(theta)^T; the rotated
  anisotropic model problem of the paper's AMG experiments (Sec. 5).
* ``banded_random(N, ...)``  unstructured matrix with ~Poisson(20) entries per
  row: 80% of the off-diagonals near the diagonal, 20% uniform; the stand-in for
  the paper's random matrices (Sec. 5) and the absent SuiteSparse set.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class CSR:
    row_ptr: np.ndarray  # int64 [n+1]
    col: np.ndarray      # int32 [nnz]
    val: np.ndarray      # float64 [nnz]

    @property
    def n(self) -> int:
        return len(self.row_ptr) - 1

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        d[rows, self.col] = self.val
        return d


def _stencil(shape, offsets):
    """CSR of a constant-coefficient stencil on a grid of ``shape`` (slowest axis
    first), neighbours outside the grid dropped.  ``offsets`` is a list of
    (delta per axis, value); entries of a row come out in ascending column order."""
    shape = tuple(int(s) for s in shape)
    n = int(np.prod(shape))
    strides = [int(np.prod(shape[a + 1:])) for a in range(len(shape))]
    offsets = sorted(offsets, key=lambda o: sum(d * s for d, s in zip(o[0], strides)))
    coords = np.indices(shape).reshape(len(shape), n)
    ids = np.arange(n, dtype=np.int64)
    k = len(offsets)
    cols = np.empty((n, k), np.int64)
    vals = np.empty((n, k), np.float64)
    mask = np.ones((n, k), bool)
    for q, (delta, value) in enumerate(offsets):
        ok = np.ones(n, bool)
        lin = 0
        for a, d in enumerate(delta):
            c = coords[a] + d
            ok &= (c >= 0) & (c < shape[a])
            lin += d * strides[a]
        mask[:, q] = ok
        cols[:, q] = ids + lin
        vals[:, q] = value
    counts = mask.sum(axis=1)
    row_ptr = np.zeros(n + 1, np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return CSR(row_ptr, cols[mask].astype(np.int32), vals[mask])


def poisson2d(n: int) -> CSR:
    offs = [((0, 0), 4.0), ((0, -1), -1.0), ((0, 1), -1.0), ((-1, 0), -1.0), ((1, 0), -1.0)]
    return _stencil((n, n), offs)


def poisson3d(n: int) -> CSR:
    offs = [((0, 0, 0), 6.0)]
    for a in range(3):
        for d in (-1, 1):
            delta = [0, 0, 0]
            delta[a] = d
            offs.append((tuple(delta), -1.0))
    return _stencil((n, n, n), offs)


def q1_aniso_stencil(eps: float, theta: float) -> dict:
    """Q1 stencil of -div(K grad u), K = R diag(1, eps) R^T, keyed by (dx, dy).

    With a = cos^2 + eps sin^2, c = sin^2 + eps cos^2, b = (1 - eps) sin cos:
    the x-stiffness [-1, 2, -1] times the y-mass [1/6, 2/3, 1/6] scaled by a,
    the transposed pair scaled by c, and the mixed term +-b/2 on the diagonals.
    """
    s, co = math.sin(theta), math.cos(theta)
    a = co * co + eps * s * s
    c = s * s + eps * co * co
    b = (1.0 - eps) * s * co
    return {
        (0, 0): 4.0 * (a + c) / 3.0,
        (1, 0): -2.0 * a / 3.0 + c / 3.0, (-1, 0): -2.0 * a / 3.0 + c / 3.0,
        (0, 1): a / 3.0 - 2.0 * c / 3.0, (0, -1): a / 3.0 - 2.0 * c / 3.0,
        (1, 1): -(a + c) / 6.0 - b / 2.0, (-1, -1): -(a + c) / 6.0 - b / 2.0,
        (1, -1): -(a + c) / 6.0 + b / 2.0, (-1, 1): -(a + c) / 6.0 + b / 2.0,
    }


def aniso_q1(n: int, eps: float = 0.001, theta: float = math.pi / 8) -> CSR:
    st = q1_aniso_stencil(eps, theta)
    # grid axes (y, x): delta (dy, dx)
    offs = [((dy, dx), v) for (dx, dy), v in st.items()]
    return _stencil((n, n), offs)


def banded_random(N: int, seed: int, mean: float = 20.0, lo: int = 4, hi: int = 64,
                  band: float = 0.005, p_band: float = 0.8) -> CSR:
    """Row i stores its diagonal and L_i - 1 distinct off-diagonal columns, with
    L_i = clip(Poisson(mean), lo, hi).  Each off-diagonal column is, with
    probability p_band, uniform on [i - W, i + W] clipped to the matrix
    (W = round(band * N)), else uniform on [0, N).  Repeats and the diagonal are
    redrawn.  Off-diagonal values are N(0, 1); the diagonal is 1 + the row's sum
    of |off-diagonal|."""
    rng = np.random.default_rng(seed)
    W = max(1, int(round(band * N)))
    L = np.clip(rng.poisson(mean, N), lo, hi).astype(np.int64)
    L = np.minimum(L, N)
    m = L - 1
    rows = np.repeat(np.arange(N, dtype=np.int64), m)

    def draw(r):
        near = rng.random(len(r)) < p_band
        a = np.maximum(r - W, 0)
        b = np.minimum(r + W, N - 1)
        cb = a + np.floor(rng.random(len(r)) * (b - a + 1)).astype(np.int64)
        cu = rng.integers(0, N, len(r), dtype=np.int64)
        return np.where(near, cb, cu)

    cols = draw(rows)
    while True:
        key = rows * N + cols
        order = np.argsort(key, kind="stable")
        ks = key[order]
        bad = np.zeros(len(key), bool)
        bad[order[1:][ks[1:] == ks[:-1]]] = True
        bad |= cols == rows
        nb = int(bad.sum())
        if nb == 0:
            break
        cols[bad] = draw(rows[bad])
    # add the diagonal and sort every row by column
    rows_all = np.concatenate([rows, np.arange(N, dtype=np.int64)])
    cols_all = np.concatenate([cols, np.arange(N, dtype=np.int64)])
    order = np.argsort(rows_all * N + cols_all, kind="stable")
    rows_all = rows_all[order]
    cols_all = cols_all[order]
    off = rows_all != cols_all
    val = np.empty(len(cols_all))
    val[off] = rng.standard_normal(int(off.sum()))
    absum = np.bincount(rows_all[off], weights=np.abs(val[off]), minlength=N)
    val[~off] = 1.0 + absum
    row_ptr = np.zeros(N + 1, np.int64)
    np.cumsum(L, out=row_ptr[1:])
    return CSR(row_ptr, cols_all.astype(np.int32), val)


def random_pattern(n: int, density: float, seed: int, diag: bool = True) -> CSR:
    """Small random sparsity pattern (for brute-force checks): each (i, j) stored
    with probability ``density``, the diagonal always when ``diag``; values
    uniform on [-1, 1]."""
    rng = np.random.default_rng(seed)
    m = rng.random((n, n)) < density
    if diag:
        np.fill_diagonal(m, True)
    rows, cols = np.nonzero(m)
    row_ptr = np.zeros(n + 1, np.int64)
    np.cumsum(m.sum(axis=1), out=row_ptr[1:])
    val = rng.uniform(-1.0, 1.0, len(cols))
    return CSR(row_ptr, cols.astype(np.int32), val)


def vector(n: int, seed: int) -> np.ndarray:
    """v ~ U[-1, 1]."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, n)


# --------------------------------------------------------------------------
# The five workloads (sizes, partitions and runs of the benchmark and tests).

@dataclass
class Workload:
    name: str
    n_p: int
    ppn: int
    seed: int
    build: object  # () -> CSR


def workload(cfg: int, scale_down: int = 1) -> Workload:
    """Workload ``cfg`` (1..4).  ``scale_down`` > 1 shrinks the grid or N by that
    factor per axis (for quick structural tests) keeping rows per rank and ppn."""
    if cfg == 1:
        n = 64 // scale_down
        return Workload("poisson2d_5pt_64x64_np16_ppn4", 16, 4, 1235,
                        lambda: poisson2d(n))
    if cfg == 2:
        n = 128 // scale_down
        np_ = (n ** 3) // 2048 if scale_down == 1 else max(1, (n ** 3) // 2048)
        return Workload(f"poisson3d_7pt_{n}^3_np{np_}_ppn16", np_, 16, 1236,
                        lambda: poisson3d(n))
    if cfg == 3:
        n = 2048 // scale_down
        np_ = max(1, (n * n) // 1024)
        return Workload(f"aniso_q1_9pt_{n}^2_eps1e-3_theta_pi8_np{np_}_ppn16", np_, 16, 1237,
                        lambda: aniso_q1(n))
    if cfg == 4:
        N = (1 << 23) // scale_down
        np_ = max(1, N // 1024)
        return Workload(f"banded_random_N{N}_np{np_}_ppn32", np_, 32, 1238,
                        lambda: banded_random(N, 1238))
    raise ValueError(cfg)


def serving_requests(count: int, rate_hz: float, seed: int, n_lo: float = 1e3,
                     n_hi: float = 2e6, p_spmv: float = 0.7):
    """The serving mix: Poisson arrivals at ``rate_hz``; each request an SpMV
    (probability p_spmv) or a CG solve, on a 2D 5-point or 3D 7-point Laplacian
    (equal odds) with N log-uniform in [n_lo, n_hi]; n_p = max(1, round(N/2048)),
    ppn = 16.  Returns a list of dicts."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, count))
    out = []
    for q in range(count):
        N = math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))
        dim = 2 if rng.random() < 0.5 else 3
        side = max(2, int(round(N ** (1.0 / dim))))
        Nq = side ** dim
        kind = "spmv" if rng.random() < p_spmv else "cg"
        out.append(dict(id=q, arrival=float(t[q]), kind=kind, dim=dim, side=side, n=Nq,
                        n_p=max(1, int(round(Nq / 2048))), ppn=16,
                        seed=int(rng.integers(0, 2**31 - 1))))
    return out
