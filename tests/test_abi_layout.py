"""The binding's ctypes mirrors of the public structs have the layout of
include/hx.h: a small C program compiled against the header prints sizeof and
offsetof of every field the binding declares (nested unions and structs by
their member paths), and each must equal the ctypes size and offset.  Needs
only gcc, no GPU."""

import ctypes
import os
import shutil
import subprocess

import pytest

import paper_2503_10855_b300 as hx

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# C type name -> ctypes mirror in the binding
MIRRORS = {
    "hx_task": hx.HxTask,
    "hx_nest_op": hx.NestOp,
    "hx_nest": hx.Nest,
    "hx_tune_table": hx.TuneTable,
    "hx_server_config": hx.ServerConfig,
    "hx_server_stats": hx.ServerStats,
    "hx_server_step_record": hx.ServerStepRecord,
}


# binding field names that differ from the header's (a Python keyword)
C_NAMES = {"inputs": "in"}


def _leaves(cls, prefix="", base=0):
    """(C member path, offset) of every field of a ctypes struct, recursing
    into nested structs and unions."""
    out = []
    for name, typ in [(f[0], f[1]) for f in cls._fields_]:
        off = base + getattr(cls, name).offset
        path = prefix + C_NAMES.get(name, name)
        if isinstance(typ, type) and issubclass(typ, (ctypes.Structure, ctypes.Union)):
            out.append((path, off))
            out += _leaves(typ, path + ".", off)
        else:
            out.append((path, off))
    return out


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    d = tmp_path_factory.mktemp("abi")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "hx.h"', "int main(void) {"]
    for cname, cls in MIRRORS.items():
        lines.append(f'    printf("{cname} %zu\\n", sizeof({cname}));')
        for path, _ in _leaves(cls):
            lines.append(f'    printf("{cname}.{path} %zu\\n", offsetof({cname}, {path}));')
    lines += ["    return 0;", "}"]
    src = d / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = d / "layout"
    cc = subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                        capture_output=True, text=True)
    # a field the binding names but the header does not fails to compile
    assert cc.returncode == 0, cc.stderr[-3000:]
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {k: int(v) for k, v in (ln.rsplit(" ", 1) for ln in out.splitlines())}


@pytest.mark.parametrize("cname", sorted(MIRRORS))
def test_struct_layout_matches_header(c_layout, cname):
    cls = MIRRORS[cname]
    assert ctypes.sizeof(cls) == c_layout[cname], cname
    for path, off in _leaves(cls):
        assert off == c_layout[f"{cname}.{path}"], f"{cname}.{path}"
