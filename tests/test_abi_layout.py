"""The ctypes binding against the C header, on the CPU: every struct the
binding mirrors has the C layout (offsets and sizes from a C compiler), and
every entry point the header declares is bound with its parameter count and
the right kind (integer width or pointer) for every parameter."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "twopaco.h")

STRUCTS = {
    "twopaco_options": "_Options",
    "twopaco_stats": "_Stats",
    "twopaco_result": "_Result",
    "twopaco_edge": "_Edge",
    "twopaco_edge_list": "_EdgeList",
}


def _header_text() -> str:
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return re.sub(r"//[^\n]*", "", src)


def _c_layout(tmp_path):
    """{struct: (sizeof, {field: (offset, size)})} as a C compiler lays them out."""
    from paper_1602_05856_gb300 import twopaco as T
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "twopaco.h"', "int main(void) {"]
    for c_name, py_name in STRUCTS.items():
        lines.append(f'  printf("S {c_name} %zu\\n", sizeof({c_name}));')
        for f, _ in getattr(T, py_name)._fields_:
            lines.append(f'  printf("F {c_name} {f} %zu %zu\\n", offsetof({c_name}, {f}), '
                         f'sizeof((({c_name}*)0)->{f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        p = line.split()
        if p[0] == "S":
            layout[p[1]] = (int(p[2]), {})
        else:
            layout[p[1]][1][p[2]] = (int(p[3]), int(p[4]))
    return layout


def test_structs_match_the_c_layout(tmp_path):
    from paper_1602_05856_gb300 import twopaco as T
    layout = _c_layout(tmp_path)
    for c_name, py_name in STRUCTS.items():
        cls = getattr(T, py_name)
        size, fields = layout[c_name]
        assert ctypes.sizeof(cls) == size, c_name
        for f, _ in cls._fields_:
            d = getattr(cls, f)
            assert (d.offset, d.size) == fields[f], (c_name, f)
    # the header declares no field the binding leaves out
    hdr = _header_text()
    for c_name, py_name in STRUCTS.items():
        body = re.search(r"typedef struct " + c_name + r" \{(.*?)\} " + c_name + ";", hdr, re.S).group(1)
        declared = []
        for decl in (d.strip() for d in body.split(";") if d.strip()):
            first, *rest = [x.strip() for x in decl.split(",")]
            declared += [first.split()[-1].lstrip("*")] + [x.lstrip("*") for x in rest]
        assert declared == [f for f, _ in getattr(T, py_name)._fields_], c_name
    # the structured dtype the edges are read with
    size, fields = layout["twopaco_edge"]
    assert T.EDGE_DTYPE.itemsize == size
    for f in T.EDGE_DTYPE.names:
        assert T.EDGE_DTYPE.fields[f][1] == fields[f][0], f


def _prototypes():
    hdr = _header_text()
    out = {}
    for m in re.finditer(r"(?m)^([A-Za-z_][\w \*]*?)\b(twopaco_\w+)\s*\(([^;{)]*)\)\s*;", hdr):
        params = [p.strip() for p in m.group(3).split(",") if p.strip()]
        if params == ["void"]:
            params = []
        out[m.group(2)] = (m.group(1).strip(), params)
    return out


def _kind_of_c(param: str) -> str:
    if "*" in param:
        return "ptr"
    t = param.rsplit(None, 1)[0] if len(param.split()) > 1 else param
    if t in ("uint64_t", "unsigned long long"):
        return "u64"
    if t in ("int", "int32_t"):
        return "i32"
    if t in ("uint32_t", "unsigned int", "unsigned"):
        return "u32"
    raise AssertionError(f"unexpected parameter type {param!r}")


def _kind_of_ctypes(t) -> str:
    if t in (ctypes.c_void_p, ctypes.c_char_p) or isinstance(t, type(ctypes.POINTER(ctypes.c_int))):
        return "ptr"
    if ctypes.sizeof(t) == 8 and t in (ctypes.c_uint64, ctypes.c_ulonglong):
        return "u64"
    if t is ctypes.c_int:
        return "i32"
    if t is ctypes.c_uint32:
        return "u32"
    raise AssertionError(f"unexpected ctypes type {t!r}")


def test_every_declared_entry_point_is_bound_with_its_signature():
    from paper_1602_05856_gb300 import build, twopaco as T
    build.build()
    L = T.load()
    protos = _prototypes()
    assert set(protos) == set(re.findall(r"\b(twopaco_\w+)\s*\(", _header_text()))
    for name, (ret, params) in protos.items():
        fn = getattr(L, name)
        assert fn.argtypes is not None, f"{name} has no argtypes in the binding"
        assert len(fn.argtypes) == len(params), name
        for i, (p, t) in enumerate(zip(params, fn.argtypes)):
            assert _kind_of_c(p) == _kind_of_ctypes(t), (name, i, p, t)
        if ret == "void":
            assert fn.restype is None, name
        elif "*" in ret:
            assert fn.restype in (ctypes.c_char_p, ctypes.c_void_p), name
        elif ret == "int":
            assert fn.restype is ctypes.c_int, name
        else:
            assert ctypes.sizeof(fn.restype) == 8, name


def test_prototype_parser_reads_the_header():
    protos = _prototypes()
    assert protos["twopaco_strerror"] == ("const char*", ["int code"]) or \
        protos["twopaco_strerror"][1] == ["int code"]
    assert protos["twopaco_kernel_launches"][1] == []
    with pytest.raises(AssertionError):
        _kind_of_c("double x")
