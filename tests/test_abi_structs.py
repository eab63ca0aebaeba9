"""The binding's ctypes structures match the C structs of include/tnn.h:
the same field names and types in the same order (parsed from the header),
and the same size and field offsets as a C compiler lays them out."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tnn.h")

# C struct name -> binding class name
STRUCTS = {"tnn_shape": "Shape", "tnn_admm_params": "AdmmParams", "tnn_admm_report": "AdmmReport",
           "tnn_tsvt_item": "TsvtItem", "tnn_admm_item": "AdmmItem", "tnn_server_params": "ServerParams"}


def _header_structs():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef struct\s*\{(.*?)\}\s*(\w+)\s*;", text, flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            m = re.match(r"(?:const\s+)?(\w+)\s*(\*?)\s*(.*)", decl)
            ctype, ptr, names = m.group(1), m.group(2), m.group(3)
            for nm in names.split(","):
                nm = nm.strip()
                star = ptr or nm.startswith("*")
                fields.append((nm.lstrip("*").strip(), "ptr" if star else ctype))
        out[name] = fields
    return out


def _ctype_name(t, tnn):
    table = {ctypes.c_int64: "int64_t", ctypes.c_uint64: "uint64_t", ctypes.c_int32: "int32_t",
             ctypes.c_double: "double", ctypes.c_void_p: "ptr", tnn.Shape: "tnn_shape"}
    return table[t]


def test_binding_fields_match_header():
    from paper_1902_03070_gb300 import tnn
    hs = _header_structs()
    for cname, pyname in STRUCTS.items():
        assert cname in hs, cname
        py = [(f, _ctype_name(t, tnn)) for f, t in getattr(tnn, pyname)._fields_]
        assert py == hs[cname], (cname, py, hs[cname])


def test_binding_layout_matches_compiler(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_1902_03070_gb300 import tnn
    hs = _header_structs()
    lines = ["#include <stddef.h>", "#include <stdio.h>", "#include <stdint.h>",
             "typedef struct CUstream_st* cudaStream_t;", '#include "tnn.h"', "int main(void) {"]
    for cname in STRUCTS:
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in hs[cname]:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        a, b, v = line.split()
        got[(a, b)] = int(v)
    for cname, pyname in STRUCTS.items():
        cls = getattr(tnn, pyname)
        assert ctypes.sizeof(cls) == got[(cname, "size")], cname
        for f, _ in hs[cname]:
            assert getattr(cls, f).offset == got[(cname, f)], (cname, f)
