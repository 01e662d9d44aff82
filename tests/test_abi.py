"""The C-ABI library: it loads, exports every entry point include/hx.h declares,
and rejects bad arguments on the host before touching the device."""

import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in os.listdir(os.path.join(ROOT, "include")) if h.endswith(".h")]


def _declared():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(hx_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for need in ("hx_create", "hx_destroy", "hx_last_error", "hx_map_reduce", "hx_stencil2d",
                 "hx_histogram"):
        assert need in names


@pytest.mark.parametrize("name", ["libhx.so", "libhx_debug.so"])
def test_library_exports_every_declared_symbol(name):
    import paper_2503_10855_b300 as hx

    path = os.path.join(os.path.dirname(hx.LIB_PATH), name)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = sorted(_declared() - exported)
    assert not missing, f"declared but not exported: {missing}"
    lib = ctypes.CDLL(path)
    for sym in _declared():
        getattr(lib, sym)


def test_debug_checks_report_build_and_reject_null():
    # release build: the kernels check nothing and the call says so; NULL
    # arguments fail on the host before any device call
    import paper_2503_10855_b300 as hx

    lib = hx.lib()
    I32, I64 = ctypes.c_int32, ctypes.c_int64
    assert lib.hx_debug_checks(None, None, None, None) == hx.HX_ERR_INVALID
    en = I32(-1)
    assert lib.hx_debug_checks(ctypes.byref(en), None, ctypes.byref(I64()), ctypes.byref(I64())) == hx.HX_ERR_INVALID
    if not hx.DEBUG:
        assert "libhx.so" in hx.LIB_PATH


def test_version_and_null_context_rejected_on_host():
    import paper_2503_10855_b300 as hx

    lib = hx.lib()
    assert hx.hx_version() >= 3
    P = ctypes.c_void_p
    assert lib.hx_map_reduce(None, P(0), P(0), P(0), ctypes.c_float(1.0), 4, P(16), P(0), P(0)) == hx.HX_ERR_INVALID
    assert b"ctx is NULL" in lib.hx_last_error()
    assert lib.hx_stencil2d(None, P(16), P(32), 4, 4, 1, P(64), None, P(0)) == hx.HX_ERR_INVALID
    assert lib.hx_histogram(None, P(16), 4, P(64), P(0), P(0)) == hx.HX_ERR_INVALID
    assert lib.hx_create(None, 0, 0) == hx.HX_ERR_INVALID
    lib.hx_destroy(None)


def test_python_binding_rejects_cpu_tensors():
    import torch

    import paper_2503_10855_b300 as hx

    class FakeCtx:
        handle = ctypes.c_void_p(0)

    with pytest.raises(TypeError):
        hx.hx_map_reduce(FakeCtx(), torch.zeros(4), torch.zeros(4), 1.0,
                         sum_out=torch.zeros(1))
