"""Thin ctypes binding of libnapspmv.so (include/napspmv.h), same names as the C ABI.

Only argument marshalling happens here: every step of the node-aware SpMV runs in
the library's CUDA kernels.  Vectors may be given as torch CUDA tensors (float64,
contiguous) or as raw device addresses (int).  If the library has not been built
the import fails loudly; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnapspmv.so")

OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_STATE, ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
HOST, DEVICE = 0, 1
F32_VALUES, MAP_TEXT, PARTITION_STRIDED, MAP_MAJORITY, COMPOSED_GATHERS, MAP_SPLIT = 1, 2, 4, 8, 16, 32
PREC_F64, PREC_F32 = 0, 1
ENGINE_DEFAULT, ENGINE_FUSED, ENGINE_PHASED, ENGINE_OVERLAP = 0, 1, 2, 3
PIPELINE_CTA, PIPELINE_WARP, PIPELINE_SELL = 1, 2, 3
HALO_ON, HALO_OFF = 1, 2
SOLO_NNZ = 1 << 19  # NAPSPMV_SOLO_NNZ
(LIST_STD, LIST_NODE, LIST_INTER, LIST_J0, LIST_J1, LIST_J2, LIST_BLL, LIST_BNL, LIST_LBUF,
 LIST_TU, LIST_SPLIT) = range(11)


class NapError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class napspmv_csr(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("row_ptr", C.c_void_p),
                ("col", C.c_void_p), ("val", C.c_void_p), ("mem", C.c_int32)]


class napspmv_opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("engine", C.c_int32), ("vec", C.c_int32),
                ("ctas_per_sm", C.c_int32), ("chunk", C.c_int32), ("tile_rows", C.c_int32),
                ("tile_nnz", C.c_int32), ("stages", C.c_int32), ("pipeline", C.c_int32),
                ("halo", C.c_int32), ("timeout_ms", C.c_int32), ("debug_stall", C.c_int32)]


STAT_FIELDS = [
    "std_msgs", "std_vals", "std_intra_msgs", "std_intra_vals", "std_inter_msgs",
    "std_inter_vals", "std_max_inter_msgs_proc", "std_max_inter_vals_proc",
    "std_max_intra_msgs_proc", "std_max_intra_vals_proc", "std_max_msg_vals",
    "nap_inter_msgs", "nap_inter_vals", "j0_msgs", "j0_vals", "j1_msgs", "j1_vals", "j2_msgs",
    "j2_vals", "nap_intra_msgs", "nap_intra_vals", "nap_max_inter_msgs_proc",
    "nap_max_inter_vals_proc", "nap_max_intra_msgs_proc", "nap_max_intra_vals_proc",
    "nap_max_inter_msg_vals", "node_pairs", "bll_total", "bnl_total", "lbuf_total",
    "nnz_on_process", "nnz_on_node", "nnz_off_node"]


class napspmv_stats(C.Structure):
    _fields_ = [(f, C.c_int64) for f in STAT_FIELDS] + [
        ("bytes_csr_f64", C.c_double), ("bytes_csr_f32", C.c_double), ("bytes_msg", C.c_double),
        ("plan_ms", C.c_double)]


class napspmv_cg_slot(C.Structure):
    _fields_ = [("plan", C.c_void_p), ("ws", C.c_void_p), ("b", C.c_void_p), ("x", C.c_void_p),
                ("r", C.c_void_p), ("p", C.c_void_p), ("q", C.c_void_p), ("scal", C.c_void_p)]


class napspmv_cg_info(C.Structure):
    _fields_ = [("outer_iters", C.c_int32), ("inner_iters", C.c_int32), ("relres", C.c_double),
                ("converged", C.c_int32)]


_lib = None
_VP = C.c_void_p


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it first "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        l = C.CDLL(LIB_PATH)
        sig = {
            "napspmv_plan": (C.c_int, [C.POINTER(napspmv_csr), C.c_int32, C.c_int32, C.c_uint32,
                                       C.POINTER(_VP)]),
            "napspmv_apply": (C.c_int, [_VP, _VP, _VP, _VP]),
            "napspmv_apply_n": (C.c_int, [_VP, _VP, _VP, C.c_int32, C.c_double, _VP]),
            "napspmv_apply_ex": (C.c_int, [_VP, _VP, _VP, _VP, C.c_int32, C.c_double,
                                           C.POINTER(napspmv_opts), _VP]),
            "napspmv_apply_host": (C.c_int, [_VP, _VP, _VP, C.c_int32, C.c_double, _VP]),
            "napspmv_apply_noalloc": (C.c_int, [_VP, _VP, _VP, C.c_int32, C.c_double, _VP]),
            "napspmv_spmv_step": (C.c_int, [_VP, _VP, _VP, _VP, C.c_double,
                                            C.POINTER(napspmv_opts), _VP]),
            "napspmv_apply_batch": (C.c_int, [C.c_int32, C.POINTER(_VP), C.POINTER(_VP),
                                              C.POINTER(_VP), C.POINTER(_VP),
                                              C.POINTER(C.c_int32), C.POINTER(C.c_double),
                                              C.POINTER(napspmv_opts), _VP]),
            "napspmv_status": (C.c_int, [_VP, _VP]),
            "napspmv_ws_status": (C.c_int, [_VP, _VP]),
            "napspmv_ws_create": (C.c_int, [_VP, C.POINTER(_VP)]),
            "napspmv_ws_destroy": (None, [_VP]),
            "napspmv_plan_stats": (C.c_int, [_VP, C.POINTER(napspmv_stats)]),
            "napspmv_plan_export": (C.c_int, [_VP, C.c_int32, _VP, C.POINTER(C.c_int64)]),
            "napspmv_get_default_opts": (C.c_int, [_VP, C.POINTER(napspmv_opts)]),
            "napspmv_set_default_opts": (C.c_int, [_VP, C.POINTER(napspmv_opts)]),
            "napspmv_cg_ir": (C.c_int, [_VP, _VP, _VP, C.c_double, C.c_double, C.c_int32,
                                        C.c_int32, C.POINTER(napspmv_cg_info), _VP]),
            "napspmv_cg": (C.c_int, [_VP, _VP, _VP, C.c_double, C.c_int32,
                                     C.POINTER(napspmv_cg_info), _VP]),
            "napspmv_dot": (C.c_int, [_VP, _VP, C.c_int64, _VP, _VP]),
            "napspmv_cg_batch_init": (C.c_int, [C.c_int32, C.POINTER(napspmv_cg_slot), C.c_int32,
                                                C.c_int32, _VP]),
            "napspmv_cg_batch_iterate": (C.c_int, [C.c_int32, C.POINTER(napspmv_cg_slot),
                                                   C.c_int32, C.c_int32, _VP]),
            "napspmv_batch_add": (C.c_int, [C.c_int32, C.POINTER(_VP), C.POINTER(_VP),
                                            C.POINTER(C.c_int64), _VP]),
            "napspmv_plan_destroy": (None, [_VP]),
            "napspmv_strerror": (C.c_char_p, [C.c_int]),
            "napspmv_last_error": (C.c_char_p, []),
            "napspmv_launch_count": (C.c_int64, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(l, name)
            f.restype = res
            f.argtypes = args
        _lib = l
    return _lib


def _check(rc):
    if rc != OK:
        raise NapError(rc, lib().napspmv_last_error().decode())
    return rc


def _dptr(x):
    """Device address of a torch CUDA tensor (float64, contiguous) or an int."""
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_cuda:
            raise ValueError("expected a CUDA tensor")
        if not x.is_contiguous():
            raise ValueError("expected a contiguous tensor")
        return x.data_ptr()
    raise TypeError(type(x))


def _stream(stream):
    if stream is None:
        try:
            import torch
            return torch.cuda.current_stream().cuda_stream
        except Exception:
            return 0
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Plan:
    """Owns a napspmv_plan_t*.  `keep` holds host/device arrays alive while used."""

    def __init__(self, handle, n, n_p, ppn, flags):
        self.handle = handle
        self.n, self.n_p, self.ppn, self.flags = n, n_p, ppn, flags

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            _lib.napspmv_plan_destroy(h)
            self.handle = None

    @property
    def _as_parameter_(self):
        return self.handle


class Workspace:
    def __init__(self, plan):
        h = _VP()
        _check(lib().napspmv_ws_create(plan.handle, C.byref(h)))
        self.handle, self.plan = h.value, plan

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            _lib.napspmv_ws_destroy(h)
            self.handle = None


def napspmv_plan(row_ptr, col, val, n_p, ppn, flags=0):
    """Plan for the CSR (numpy host arrays or torch CUDA tensors)."""
    dev = hasattr(row_ptr, "is_cuda") and row_ptr.is_cuda
    if dev:
        n = row_ptr.numel() - 1
        nnz = col.numel()
        rp, cl, vl = row_ptr.data_ptr(), col.data_ptr(), val.data_ptr()
        keep = (row_ptr, col, val)
    else:
        row_ptr = np.ascontiguousarray(row_ptr, np.int64)
        col = np.ascontiguousarray(col, np.int32)
        val = np.ascontiguousarray(val, np.float64)
        n, nnz = len(row_ptr) - 1, len(col)
        rp, cl, vl = row_ptr.ctypes.data, col.ctypes.data, val.ctypes.data
        keep = (row_ptr, col, val)
    csr = napspmv_csr(n, nnz, rp, cl if nnz else None, vl if nnz else None,
                      DEVICE if dev else HOST)
    h = _VP()
    _check(lib().napspmv_plan(C.byref(csr), int(n_p), int(ppn), int(flags), C.byref(h)))
    del keep
    return Plan(h.value, n, int(n_p), int(ppn), int(flags))


def make_opts(**kw):
    o = napspmv_opts()
    for k, v in kw.items():
        setattr(o, k, int(v))
    return o


def napspmv_apply(plan, v, w, stream=None):
    _check(lib().napspmv_apply(plan.handle, _dptr(v), _dptr(w), _stream(stream)))


def napspmv_apply_n(plan, v, w, reps, scale=1.0, stream=None):
    _check(lib().napspmv_apply_n(plan.handle, _dptr(v), _dptr(w), int(reps), float(scale),
                                 _stream(stream)))


def napspmv_apply_ex(plan, v, w, reps=1, scale=1.0, opts=None, ws=None, stream=None):
    _check(lib().napspmv_apply_ex(plan.handle, ws.handle if ws else None, _dptr(v), _dptr(w),
                                  int(reps), float(scale), C.byref(opts) if opts else None,
                                  _stream(stream)))


def napspmv_apply_noalloc(plan, v, w, reps=1, scale=1.0, stream=None):
    """As napspmv_apply_n, with no allocation (scratch in a fixed device array)."""
    _check(lib().napspmv_apply_noalloc(plan.handle, _dptr(v), _dptr(w), int(reps), float(scale),
                                       _stream(stream)))


def napspmv_spmv_step(plan, v, w, scale=1.0, opts=None, ws=None, stream=None):
    """The three-block SpMV step alone, on the workspace's current receive buffers."""
    _check(lib().napspmv_spmv_step(plan.handle, ws.handle if ws else None, _dptr(v), _dptr(w),
                                   float(scale), C.byref(opts) if opts else None,
                                   _stream(stream)))


def napspmv_apply_host(plan, v_host, w_host, reps=1, scale=1.0, stream=None):
    """v_host, w_host: numpy float64 arrays (or torch CPU tensors, pinned or not)."""
    def hp(a):
        if hasattr(a, "data_ptr"):
            return a.data_ptr()
        assert a.dtype == np.float64 and a.flags.c_contiguous
        return a.ctypes.data
    _check(lib().napspmv_apply_host(plan.handle, hp(v_host), hp(w_host), int(reps), float(scale),
                                    _stream(stream)))


def napspmv_apply_batch(plans, v, w, reps, scale=None, opts=None, ws=None, stream=None):
    n = len(plans)
    P = (_VP * n)(*[p.handle for p in plans])
    W = (_VP * n)(*[(x.handle if x else None) for x in ws]) if ws else None
    V = (_VP * n)(*[_dptr(x) for x in v])
    Wv = (_VP * n)(*[_dptr(x) for x in w])
    R = (C.c_int32 * n)(*[int(r) for r in reps])
    S = (C.c_double * n)(*[float(s) for s in scale]) if scale else None
    _check(lib().napspmv_apply_batch(n, P, W, V, Wv, R, S, C.byref(opts) if opts else None,
                                     _stream(stream)))


def napspmv_status(plan, stream=None):
    """Synchronises; returns the device-side status code (0 or ERR_TIMEOUT)."""
    return lib().napspmv_status(plan.handle, _stream(stream))


def napspmv_ws_status(ws, stream=None):
    return lib().napspmv_ws_status(ws.handle, _stream(stream))


def napspmv_plan_stats(plan):
    s = napspmv_stats()
    _check(lib().napspmv_plan_stats(plan.handle, C.byref(s)))
    return {f: getattr(s, f) for f, _ in napspmv_stats._fields_}


def napspmv_plan_export(plan, which):
    cnt = C.c_int64()
    _check(lib().napspmv_plan_export(plan.handle, int(which), None, C.byref(cnt)))
    buf = np.zeros(max(cnt.value, 1), np.int64)
    _check(lib().napspmv_plan_export(plan.handle, int(which), buf.ctypes.data, C.byref(cnt)))
    return buf[:cnt.value]


def export_list(plan, which):
    """(src, dst, ptr, idx) of a message list."""
    b = napspmv_plan_export(plan, which)
    m, total = int(b[0]), int(b[1])
    o = 2
    src = b[o:o + m]; o += m
    dst = b[o:o + m]; o += m
    ptr = b[o:o + m + 1]; o += m + 1
    idx = b[o:o + total]
    return src, dst, ptr, idx


def napspmv_get_default_opts(plan):
    o = napspmv_opts()
    _check(lib().napspmv_get_default_opts(plan.handle, C.byref(o)))
    return o


def napspmv_set_default_opts(plan, opts):
    _check(lib().napspmv_set_default_opts(plan.handle, C.byref(opts)))


def napspmv_cg_ir(plan, b, x, rtol=1e-10, inner_rtol=1e-5, max_outer=50, inner_max=100000,
                  stream=None):
    info = napspmv_cg_info()
    _check(lib().napspmv_cg_ir(plan.handle, _dptr(b), _dptr(x), float(rtol), float(inner_rtol),
                               int(max_outer), int(inner_max), C.byref(info), _stream(stream)))
    return {f: getattr(info, f) for f, _ in napspmv_cg_info._fields_}


def napspmv_cg(plan, b, x, rtol=1e-10, max_it=100000, stream=None):
    info = napspmv_cg_info()
    _check(lib().napspmv_cg(plan.handle, _dptr(b), _dptr(x), float(rtol), int(max_it),
                            C.byref(info), _stream(stream)))
    return {f: getattr(info, f) for f, _ in napspmv_cg_info._fields_}


def napspmv_dot(x, y, n, result, stream=None):
    _check(lib().napspmv_dot(_dptr(x), _dptr(y), int(n), _dptr(result), _stream(stream)))


def napspmv_strerror(code):
    return lib().napspmv_strerror(int(code)).decode()


def napspmv_launch_count():
    return int(lib().napspmv_launch_count())


def _slots(slots):
    arr = (napspmv_cg_slot * len(slots))()
    for i, d in enumerate(slots):
        arr[i] = napspmv_cg_slot(d["plan"].handle, d["ws"].handle if d.get("ws") else None,
                                 _dptr(d["b"]), _dptr(d["x"]), _dptr(d["r"]), _dptr(d["p"]),
                                 _dptr(d["q"]), _dptr(d["scal"]))
    return arr


def napspmv_cg_batch_init(slots, precision=PREC_F64, x_is_zero=False, stream=None):
    """slots: list of dicts with plan, ws, b, x, r, p, q, scal (tensors)."""
    arr = _slots(slots)
    _check(lib().napspmv_cg_batch_init(len(slots), arr, int(precision), int(bool(x_is_zero)),
                                       _stream(stream)))


def napspmv_cg_batch_iterate(slots, precision=PREC_F64, iters=1, stream=None):
    arr = _slots(slots)
    _check(lib().napspmv_cg_batch_iterate(len(slots), arr, int(precision), int(iters),
                                          _stream(stream)))


def napspmv_batch_add(ys, xs, stream=None):
    n = len(ys)
    Y = (_VP * n)(*[_dptr(y) for y in ys])
    X = (_VP * n)(*[_dptr(x) for x in xs])
    N = (C.c_int64 * n)(*[int(y.numel()) for y in ys])
    _check(lib().napspmv_batch_add(n, Y, X, N, _stream(stream)))
