"""The C-ABI library builds, loads and exports every entry point of include/hs3d.h.

No compute call is made here (this suite runs without a GPU); only argument
validation paths that return before touching the device are exercised.
"""
import ctypes as C
import os
import re
import shutil
import subprocess

import pytest

import paper_2206_09733_gb300 as hs
from paper_2206_09733_gb300 import build as hsbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(hs3d_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    hsbuild.build()
    return hs.lib()


def test_header_declares_the_boundary():
    d = _declared()
    for name in ("hs3d_mesh_create", "hs3d_residual", "hs3d_rk3_step", "hs3d_submit", "hs3d_poll"):
        assert name in d


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(hs.EXPORTS) == _declared()


def test_version_and_error_string(lib):
    assert "sm_103a" in hs.version()
    assert isinstance(lib.hs3d_last_error(), bytes)


@pytest.mark.parametrize("bad", [dict(N=0), dict(N=8), dict(ex=0), dict(amp=0.5), dict(periodic=0),
                                 dict(hi=-1.0)])
def test_invalid_mesh_descriptors_rejected_before_device_work(lib, bad):
    args = dict(ex=2, ey=2, ez=2, N=3, amp=0.0, periodic=1, hi=1.0)
    args.update(bad)
    d = hs.mesh_desc(args["ex"], args["ey"], args["ez"], args["N"], hi=(args["hi"],) * 3, amp=args["amp"])
    if args["periodic"] == 0:
        d.periodic[1] = 0
    h = C.c_void_p()
    st = lib.hs3d_mesh_create(C.byref(d), C.byref(h))
    assert st in (hs.ERR_INVALID, hs.ERR_UNSUPPORTED)
    assert not h.value
    assert lib.hs3d_last_error()


def test_null_arguments_rejected(lib):
    cfg = hs.solver_cfg()
    assert lib.hs3d_residual(None, C.byref(cfg), None, None, None) == hs.ERR_INVALID
    assert lib.hs3d_rk3_step(None, C.byref(cfg), None, None, 0.0, None) == hs.ERR_INVALID
    assert lib.hs3d_mesh_create(None, None) == hs.ERR_INVALID
    assert lib.hs3d_poll(None, 1, None) in (hs.ERR_INVALID, hs.ERR_UNSUPPORTED)


def test_structs_match_header_layout(tmp_path):
    """Size and field offsets of every public struct as the C compiler lays
    them out from include/hs3d.h, against the ctypes mirror."""
    structs = {"hs3d_mesh_desc": hs.MeshDesc, "hs3d_solver_cfg": hs.SolverCfg, "hs3d_ic": hs.IC,
               "hs3d_request": hs.Request, "hs3d_result": hs.Result}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "hs3d.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    gcc = shutil.which("gcc") or pytest.skip("no C compiler")
    subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    seen = 0
    for line in filter(None, out):
        cname, field, val = line.split()
        py = structs[cname]
        got = C.sizeof(py) if field == "size" else getattr(py, field).offset
        assert got == int(val), (cname, field, got, val)
        seen += 1
    assert seen == sum(1 + len(py._fields_) for py in structs.values())
