"""The C-ABI library loads without a GPU and exports every function that
include/napspmv.h declares; host-only calls behave."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "napspmv.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(napspmv_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    import __graft_entry__ as g
    g.build()
    from paper_1612_08060_gb300 import napspmv
    return napspmv.LIB_PATH


def test_header_declares_the_plan_and_apply_calls():
    d = _declared()
    for name in ("napspmv_plan", "napspmv_apply", "napspmv_apply_n", "napspmv_plan_stats",
                 "napspmv_plan_export", "napspmv_cg_ir", "napspmv_plan_destroy",
                 "napspmv_strerror"):
        assert name in d


def test_every_declared_symbol_is_exported(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\bT (napspmv_\w+)", out))
    assert set(_declared()) <= exported


def test_strerror_and_argument_errors_without_gpu(libpath):
    from paper_1612_08060_gb300 import napspmv as nap
    assert nap.napspmv_strerror(0) == "ok"
    assert nap.napspmv_strerror(nap.ERR_TIMEOUT).startswith("device-side wait")
    # argument checks happen before any CUDA call
    h = ctypes.c_void_p()
    rc = nap.lib().napspmv_plan(None, 1, 1, 0, ctypes.byref(h))
    assert rc == nap.ERR_ARG
    assert b"invalid CSR" in nap.lib().napspmv_last_error()


def test_limits_and_flags_rejected_before_device_work(libpath):
    """Size limits, partition bounds and plan flags are checked on the host
    before the arrays are read: a descriptor claiming N = 2^30 over a tiny
    buffer is refused with ERR_UNSUPPORTED, never dereferenced."""
    import numpy as np
    from paper_1612_08060_gb300 import napspmv as nap
    rp = np.zeros(4, np.int64)
    col = np.zeros(1, np.int32)
    val = np.zeros(1, np.float64)

    def plan(n, nnz, n_p, ppn, flags=0):
        csr = nap.napspmv_csr(n, nnz, rp.ctypes.data, col.ctypes.data, val.ctypes.data, nap.HOST)
        h = ctypes.c_void_p()
        return nap.lib().napspmv_plan(ctypes.byref(csr), n_p, ppn, flags, ctypes.byref(h))

    assert plan(1 << 30, 0, 4, 2) == nap.ERR_UNSUPPORTED
    assert plan(3, (1 << 31) - 1, 1, 1) == nap.ERR_UNSUPPORTED
    assert plan(3, 0, 4, 2) == nap.ERR_ARG          # n_p > N
    assert plan(3, 0, 0, 2) == nap.ERR_ARG          # n_p < 1
    assert plan(3, 0, 2, 0) == nap.ERR_ARG          # ppn < 1
    assert plan(3, 0, 2, 1, 64) == nap.ERR_ARG      # unknown flag bit
    assert plan(3, 0, 2, 1, nap.MAP_TEXT | nap.MAP_MAJORITY) == nap.ERR_ARG
    assert b"excludes" in nap.lib().napspmv_last_error()
    assert plan(3, 0, 2, 1, nap.MAP_SPLIT | nap.MAP_MAJORITY) == nap.ERR_ARG


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_1612_08060_gb300 import napspmv as nap
    monkeypatch.setattr(nap, "_lib", None)
    monkeypatch.setattr(nap, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="missing"):
        nap.lib()


def test_binding_constants_match_the_header():
    """The Python names of the flag, engine and threshold values carry the
    header's numbers."""
    from paper_1612_08060_gb300 import napspmv as nap
    text = open(HEADER).read()
    defs = {}
    for name, val in re.findall(r"#define (NAPSPMV_\w+) \(?([0-9a-fx]+[ul]*(?: << \d+)?)\)?", text):
        val = re.sub(r"(?<=\d)[ul]+", "", val)
        defs[name] = eval(val)  # literal integers and shifts only
    pairs = {"F32_VALUES": "NAPSPMV_F32_VALUES", "MAP_TEXT": "NAPSPMV_MAP_TEXT",
             "PARTITION_STRIDED": "NAPSPMV_PARTITION_STRIDED",
             "MAP_MAJORITY": "NAPSPMV_MAP_MAJORITY", "COMPOSED_GATHERS": "NAPSPMV_COMPOSED_GATHERS",
             "MAP_SPLIT": "NAPSPMV_MAP_SPLIT", "PIPELINE_SELL": "NAPSPMV_PIPELINE_SELL",
             "ENGINE_FUSED": "NAPSPMV_ENGINE_FUSED", "ENGINE_PHASED": "NAPSPMV_ENGINE_PHASED",
             "ENGINE_OVERLAP": "NAPSPMV_ENGINE_OVERLAP", "PIPELINE_CTA": "NAPSPMV_PIPELINE_CTA",
             "PIPELINE_WARP": "NAPSPMV_PIPELINE_WARP", "HALO_ON": "NAPSPMV_HALO_ON",
             "HALO_OFF": "NAPSPMV_HALO_OFF", "SOLO_NNZ": "NAPSPMV_SOLO_NNZ"}
    for py, c in pairs.items():
        assert c in defs, c
        assert getattr(nap, py) == defs[c], (py, getattr(nap, py), defs[c])
