"""The C-ABI library loads and exports every entry point include/ptim.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "ptim.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pt_[a-zA-Z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2501_03061_gb300 import _lib, build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("pt_create", "pt_destroy", "pt_apply_exchange", "pt_build_ace", "pt_apply_ace",
                     "pt_ptim_step", "pt_apply_H", "pt_diag_occupations"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_prototypes_cover_the_header():
    from paper_2501_03061_gb300 import _lib
    assert set(declared_functions()) == set(_lib.PROTOTYPES)


def test_version_string(lib):
    from paper_2501_03061_gb300 import _lib
    l = _lib.load()
    assert b"sm_103a" in l.pt_version()


STRUCTS = ("pt_grid", "pt_kernel", "pt_exchange_item", "pt_ptim_params", "pt_ptim_stats")


def header_struct_fields():
    text = open(os.path.join(ROOT, "include", "ptim.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = {}
    for m in re.finditer(r"typedef struct \{(.*?)\}\s*(\w+);", text, flags=re.S):
        fields = []
        for decl in m.group(1).split(";"):
            decl = re.sub(r"\s+", " ", decl.strip())
            if not decl:
                continue
            parts = decl.split(",")
            fields.append(re.match(r"(.*?)(\w+)(\[\d+\])?$", parts[0].strip()).group(2))
            fields += [re.match(r"\s*\**\s*(\w+)", e).group(1) for e in parts[1:]]
        out[m.group(2)] = fields
    return out


def test_binding_structs_match_the_header_field_by_field():
    from paper_2501_03061_gb300 import _lib
    hdr = header_struct_fields()
    for name in STRUCTS:
        assert [f[0] for f in getattr(_lib, name)._fields_] == hdr[name], name


def test_binding_struct_layout_matches_the_c_compiler(tmp_path):
    """sizeof and every field offset as gcc lays the header's structs out, against ctypes."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    from paper_2501_03061_gb300 import _lib
    hdr = header_struct_fields()
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "ptim.h"', "int main(void) {"]
    for name in STRUCTS:
        offs = " ".join("%zu" for _ in hdr[name])
        args = ", ".join(f"offsetof({name}, {f})" for f in hdr[name])
        lines.append(f'  printf("{name} %zu {offs}\\n", sizeof({name}), {args});')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        name, *vals = line.split()
        got[name] = [int(v) for v in vals]
    for name in STRUCTS:
        cls = getattr(_lib, name)
        want = [ctypes.sizeof(cls)] + [getattr(cls, f[0]).offset for f in cls._fields_]
        assert got[name] == want, (name, got[name], want)
