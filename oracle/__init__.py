"""ctypes wrapper of the CPU oracle (oracle.c) for node-aware parallel SpMV.

TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the benchmark's
CPU-baseline leg may import this package.  The CUDA library and its Python
binding never import it; the two implementations share no code.

Each function follows a definition of Bienz, Gropp, Olson, "Node aware sparse
matrix-vector multiplication" (arXiv 1612.08060); see the header of oracle.c for
the equation behind each one and the readings of the points the paper leaves
open.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

# message-list kinds, in the order oracle.c stores them
STD, NODE, INTER, J0, J1, J2, BLL, BNL, LBUF = range(9)
LIST_NAMES = ["STD", "NODE", "INTER", "J0", "J1", "J2", "BLL", "BNL", "LBUF"]
MAP_TEXT = 2
STRIDED = 4  # row i on rank i mod n_p (the strided partition of Sec. 5)
MAP_MAJORITY = 8  # node pairs mapped to the processes owning / using most of E(n,m)
MAP_SPLIT = 16  # a node with fewer partner nodes than processes is split over them

STAT_NAMES = [
    "std_msgs", "std_vals", "std_intra_msgs", "std_intra_vals", "std_inter_msgs",
    "std_inter_vals", "std_max_inter_msgs_proc", "std_max_inter_vals_proc",
    "std_max_intra_msgs_proc", "std_max_intra_vals_proc", "std_max_msg_vals",
    "nap_inter_msgs", "nap_inter_vals", "j0_msgs", "j0_vals", "j1_msgs", "j1_vals",
    "j2_msgs", "j2_vals", "nap_intra_msgs", "nap_intra_vals",
    "nap_max_inter_msgs_proc", "nap_max_inter_vals_proc", "nap_max_intra_msgs_proc",
    "nap_max_intra_vals_proc", "nap_max_inter_msg_vals", "node_pairs", "bll_total",
    "bnl_total", "lbuf_total", "nnz_on_process", "nnz_on_node", "nnz_off_node",
]


class _List(C.Structure):
    _fields_ = [("m", C.c_int64), ("total", C.c_int64),
                ("src", C.POINTER(C.c_int64)), ("dst", C.POINTER(C.c_int64)),
                ("ptr", C.POINTER(C.c_int64)), ("idx", C.POINTER(C.c_int64))]


_P64 = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_P32 = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_PF64 = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_PF32 = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")


def lib():
    global _lib
    if _lib is None:
        # NAPSPMV_ORACLE_LIB: a copy of the oracle with a planted mistake, loaded
        # by the test that checks the pins catch it (never set otherwise)
        l = C.CDLL(os.environ.get("NAPSPMV_ORACLE_LIB") or _build.build())
        l.orc_row_start.restype = C.c_int64
        l.orc_row_start.argtypes = [C.c_int64, C.c_int64, C.c_int64]
        l.orc_owner.restype = C.c_int64
        l.orc_owner.argtypes = [C.c_int64, C.c_int64, C.c_int64]
        l.orc_plan_build.restype = C.c_int
        l.orc_plan_build.argtypes = [C.c_int64, C.c_int64, _P64, _P32, C.c_int64, C.c_int64,
                                     C.c_int64, C.POINTER(C.c_void_p)]
        l.orc_plan_free.argtypes = [C.c_void_p]
        l.orc_plan_list.restype = C.POINTER(_List)
        l.orc_plan_list.argtypes = [C.c_void_p, C.c_int]
        for f in ("orc_plan_send_proc", "orc_plan_recv_proc", "orc_plan_split"):
            getattr(l, f).restype = C.POINTER(C.c_int64)
            getattr(l, f).argtypes = [C.c_void_p]
        l.orc_plan_stats.argtypes = [C.c_void_p, _P64]
        l.orc_spmv.argtypes = [C.c_int64, _P64, _P32, _PF64, _PF64, _PF64]
        l.orc_spmv_f32.argtypes = [C.c_int64, _P64, _P32, _PF32, _PF64, _PF64]
        l.orc_napspmv.restype = C.c_int
        l.orc_napspmv.argtypes = [C.c_void_p, _P64, _P32, _PF64, _PF64, _PF64]
        l.orc_cg.restype = C.c_int
        l.orc_cg.argtypes = [C.c_int64, _P64, _P32, _PF64, _PF64, _PF64, C.c_double,
                             C.c_int64, C.POINTER(C.c_int64), C.POINTER(C.c_double)]
        _lib = l
    return _lib


def _arr(ptr, n):
    if n == 0:
        return np.zeros(0, np.int64)
    return np.ctypeslib.as_array(ptr, shape=(n,)).copy()


class OraclePlan:
    """Standard and node-aware communication plans of one matrix and partition."""

    def __init__(self, row_ptr, col, n_p, ppn, flags=0):
        row_ptr = np.ascontiguousarray(row_ptr, np.int64)
        col = np.ascontiguousarray(col, np.int32)
        n = len(row_ptr) - 1
        h = C.c_void_p()
        rc = lib().orc_plan_build(n, int(row_ptr[-1]), row_ptr, col, int(n_p), int(ppn),
                                  int(flags), C.byref(h))
        if rc != 0:
            raise ValueError(f"oracle plan build failed: {rc}")
        self._h = h
        self.n, self.n_p, self.ppn = n, int(n_p), int(ppn)

    def __del__(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.orc_plan_free(self._h)
            self._h = None

    def list(self, which):
        """(src, dst, ptr, idx) int64 arrays of one message list."""
        L = lib().orc_plan_list(self._h, which).contents
        return (_arr(L.src, L.m), _arr(L.dst, L.m), _arr(L.ptr, L.m + 1), _arr(L.idx, L.total))

    def list_dict(self, which):
        """{(src, dst): tuple(idx)} view of a list (handy for small cases)."""
        s, d, p, i = self.list(which)
        return {(int(s[k]), int(d[k])): tuple(int(x) for x in i[p[k]:p[k + 1]])
                for k in range(len(s))}

    def tu(self):
        m = lib().orc_plan_list(self._h, NODE).contents.m
        return (_arr(lib().orc_plan_send_proc(self._h), m),
                _arr(lib().orc_plan_recv_proc(self._h), m))

    def split(self):
        return _arr(lib().orc_plan_split(self._h), 3 * self.n).reshape(self.n, 3)

    def stats(self):
        out = np.zeros(33, np.int64)
        lib().orc_plan_stats(self._h, out)
        return dict(zip(STAT_NAMES, (int(x) for x in out)))

    def napspmv(self, row_ptr, col, val, v):
        """Algorithm NAPSpMV simulated message by message (see oracle.c)."""
        w = np.empty(self.n, np.float64)
        rc = lib().orc_napspmv(self._h, np.ascontiguousarray(row_ptr, np.int64),
                               np.ascontiguousarray(col, np.int32),
                               np.ascontiguousarray(val, np.float64),
                               np.ascontiguousarray(v, np.float64), w)
        if rc != 0:
            raise ValueError(f"oracle NAPSpMV failed: {rc}")
        return w


def row_start(n, n_p, r):
    return lib().orc_row_start(n, n_p, r)


def owner(n, n_p, j):
    return lib().orc_owner(n, n_p, j)


def spmv(row_ptr, col, val, v):
    """w = A v in FP64, rows in order, stored column order."""
    n = len(row_ptr) - 1
    w = np.empty(n, np.float64)
    lib().orc_spmv(n, np.ascontiguousarray(row_ptr, np.int64), np.ascontiguousarray(col, np.int32),
                   np.ascontiguousarray(val, np.float64), np.ascontiguousarray(v, np.float64), w)
    return w


def spmv_f32(row_ptr, col, val32, v):
    """FP32-stored values, FP32 products, FP64 sums."""
    n = len(row_ptr) - 1
    w = np.empty(n, np.float64)
    lib().orc_spmv_f32(n, np.ascontiguousarray(row_ptr, np.int64),
                       np.ascontiguousarray(col, np.int32),
                       np.ascontiguousarray(val32, np.float32),
                       np.ascontiguousarray(v, np.float64), w)
    return w


def cg(row_ptr, col, val, b, x0=None, rtol=1e-10, max_it=100000):
    """FP64 CG; returns (x, iterations, true relative residual)."""
    n = len(row_ptr) - 1
    x = np.zeros(n) if x0 is None else np.array(x0, np.float64, copy=True)
    it = C.c_int64()
    rr = C.c_double()
    rc = lib().orc_cg(n, np.ascontiguousarray(row_ptr, np.int64),
                      np.ascontiguousarray(col, np.int32), np.ascontiguousarray(val, np.float64),
                      np.ascontiguousarray(b, np.float64), x, rtol, max_it, C.byref(it),
                      C.byref(rr))
    if rc != 0:
        raise ValueError(f"oracle CG failed: {rc}")
    return x, it.value, rr.value
