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


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_1612_08060_gb300 import napspmv as nap
    monkeypatch.setattr(nap, "_lib", None)
    monkeypatch.setattr(nap, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="missing"):
        nap.lib()
