"""The C ABI without a GPU: libhp.so loads, exports every function include/hp.h declares,
the Python binding covers exactly those functions, its ctypes structures have the header's
members in the header's order with the C compiler's sizes and offsets, and every status
code has a message.  No call here touches the device."""
import ctypes as C
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hp.h")
STRUCTS = {"hp_problem_desc": "Desc", "hp_solve_stats": "SolveStats", "hp_newton_opts": "NewtonOpts",
           "hp_newton_stats": "NewtonStats", "hp_tuning": "Tuning"}


def _header_text():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    return re.sub(r"//[^\n]*", " ", text)


def _declared_functions():
    return set(re.findall(r"\b(hp_[A-Za-z0-9_]+)\s*\(", _header_text()))


def _struct_members():
    out = {}
    for body, name in re.findall(r"typedef\s+struct\s*\{(.*?)\}\s*(hp_\w+)\s*;", _header_text(), flags=re.S):
        members = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            parts = [p.strip() for p in decl.split(",")]
            first = re.findall(r"\*?\s*(\w+)\s*(?:\[\s*\d+\s*\])?\s*$", parts[0])[0]
            members.append(first)
            members += [re.sub(r"[\s*]|\[\s*\d+\s*\]", "", p) for p in parts[1:]]
        out[name] = members
    return out


@pytest.fixture(scope="module")
def hp():
    import paper_1909_03948_gb300.hp as hp_mod
    if not os.path.exists(hp_mod.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return hp_mod


def test_library_exports_every_declared_function(hp):
    declared = _declared_functions()
    assert len(declared) > 40
    L = C.CDLL(hp.LIB_PATH)
    missing = sorted(n for n in declared if not hasattr(L, n))
    assert not missing, missing
    bound = set(hp.EXPORTED)
    assert declared == bound, (sorted(declared - bound), sorted(bound - declared))
    hp.lib()  # the binding sets every restype / argtypes


def test_ctypes_structures_match_the_header(hp):
    members = _struct_members()
    for cname, pyname in STRUCTS.items():
        fields = [f for f, _ in getattr(hp, pyname)._fields_]
        assert members[cname] == fields, (cname, members[cname], fields)


@pytest.mark.skipif(shutil.which("gcc") is None, reason="no C compiler")
def test_ctypes_layout_equals_the_c_compilers(hp, tmp_path):
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "hp.h"', "int main(void) {"]
    for cname, pyname in STRUCTS.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in getattr(hp, pyname)._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        cname, key, val = line.split()
        got[(cname, key)] = int(val)
    for cname, pyname in STRUCTS.items():
        S = getattr(hp, pyname)
        assert got[(cname, "size")] == C.sizeof(S), cname
        for f, _ in S._fields_:
            assert got[(cname, f)] == getattr(S, f).offset, (cname, f)


def test_every_status_code_has_a_message(hp):
    L = hp.lib()
    for code in (hp.HP_OK, hp.HP_ERR_INVALID, hp.HP_ERR_NOT_CONVERGED, hp.HP_ERR_NONFINITE, hp.HP_ERR_CUDA,
                 hp.HP_ERR_NOMEM, hp.HP_ERR_STATE):
        assert L.hp_status_string(code).decode().strip()
