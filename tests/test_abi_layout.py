"""The Python binding marshals exactly what include/irp.h declares.

The binding describes the C ABI a second time, in ctypes: the struct layouts,
the enum values and every function's parameter list.  A field out of order,
a parameter missing or an int where the header has int64_t would pass
arguments to the wrong place without any error.  These checks compile the
header with the host C compiler and compare it with the binding, on the CPU.
"""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2008_11486_gb300 import _binding as B
from paper_2008_11486_gb300 import build as irp_build

HEADER = os.path.join(irp_build.INCLUDE, "irp.h")
STRUCTS = {"irp_clip_params": B.ClipParams, "irp_set": B.IrpSet,
           "irp_reduce_params": B.ReduceParams, "irp_host_io": B.IrpHostIo}


def _header_text():
    with open(HEADER) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    return re.sub(r"//[^\n]*", " ", src)


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    """sizeof and offsetof of every struct field, and the enum values, as the C
    compiler lays them out from the header."""
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "irp.h"', 'int main(void) {']
    for cname, cls in STRUCTS.items():
        lines.append(f'  printf("size {cname} %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("off {cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
    enums = re.findall(r"\b(IRP_[A-Z0-9_]+)\s*=\s*\d+", _header_text())
    for e in enums:
        lines.append(f'  printf("enum {e} %d\\n", (int){e});')
    lines += ['  printf("define IRP_MAX_FRAMES %d\\n", IRP_MAX_FRAMES);', '  return 0;', '}']
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run(["gcc", "-std=c11", "-I" + irp_build.INCLUDE, str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    table = {}
    for line in out.splitlines():
        kind, key, val = line.split()
        table[(kind, key)] = int(val)
    return table


def test_struct_layouts_match_the_header(c_layout):
    for cname, cls in STRUCTS.items():
        assert ctypes.sizeof(cls) == c_layout[("size", cname)], cname
        for fname, _ in cls._fields_:
            assert getattr(cls, fname).offset == c_layout[("off", f"{cname}.{fname}")], \
                f"{cname}.{fname}"


def test_enum_values_match_the_header(c_layout):
    enums = {k: v for (kind, k), v in c_layout.items() if kind == "enum"}
    status = {k: v for k, v in enums.items() if k == "IRP_OK" or k.startswith("IRP_ERR_")}
    assert {v: k for k, v in status.items()} == B.STATUS_NAMES
    assert enums["IRP_INTERP_NEAREST"] == B.INTERP["nearest"]
    assert enums["IRP_INTERP_BILINEAR"] == B.INTERP["bilinear"]
    assert enums["IRP_INTERP_SPLINE3"] == B.INTERP["spline3"]
    assert enums["IRP_INTERP_CUBIC"] == B.INTERP["cubic"]
    assert enums["IRP_F32"] == B.DTYPE["f32"] and enums["IRP_F16_SCALED"] == B.DTYPE["f16"]
    assert c_layout[("define", "IRP_MAX_FRAMES")] == B.MAX_FRAMES


def _param_class(decl):
    """The ctypes types that may marshal one C parameter declaration."""
    decl = decl.strip()
    if "*" in decl:
        return "pointer"
    words = decl.replace("const", " ").split()
    base = " ".join(words[:-1]) if len(words) > 1 else words[0]
    return {"int64_t": "int64", "size_t": "size", "double": "double", "float": "float",
            "uint32_t": "uint32", "int": "int", "irp_interp": "int", "irp_status": "int",
            "irp_stack_dtype": "int"}[base]


def _ctypes_class(t):
    if t in (ctypes.c_void_p, ctypes.c_char_p) or issubclass(t, ctypes._Pointer):
        return "pointer"
    for cls, name in ((ctypes.c_int64, "int64"), (ctypes.c_size_t, "size"),
                      (ctypes.c_double, "double"), (ctypes.c_float, "float"),
                      (ctypes.c_uint32, "uint32"), (ctypes.c_int, "int")):
        if t is cls:
            return name
    raise AssertionError(f"unexpected ctypes type {t}")


def test_every_prototype_matches_its_binding():
    protos = re.findall(r"\b(irp_status|size_t|const char\s*\*|int|void)\s+(irp_\w+)\s*\("
                        r"([^;{]*?)\)\s*;", _header_text(), flags=re.S)
    assert len(protos) >= 20
    L = B.lib()
    undeclared = []
    for ret, name, args in protos:
        f = getattr(L, name)
        if f.argtypes is None:
            undeclared.append(name)
            continue
        params = [] if args.strip() in ("", "void") else args.split(",")
        assert [_param_class(p) for p in params] == [_ctypes_class(t) for t in f.argtypes], name
        want_ret = {"irp_status": ctypes.c_int, "size_t": ctypes.c_size_t, "int": ctypes.c_int,
                    "void": None}.get(ret.strip(), ctypes.c_char_p)
        assert f.restype is want_ret, name
    # declared by its own test, which is the only caller
    assert set(undeclared) <= {"irp_reduce_set_noalloc"}
