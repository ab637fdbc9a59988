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


def test_header_bound_on_orbital_counts_matches_the_binding():
    from paper_2501_03061_gb300 import _lib
    text = open(os.path.join(ROOT, "include", "ptim.h")).read()
    m = re.search(r"#define\s+PT_MAX_ORBITALS\s+(\d+)", text)
    assert m and int(m.group(1)) == _lib.PT_MAX_ORBITALS
    # N x N matrices are indexed with 32-bit products inside the kernels
    assert _lib.PT_MAX_ORBITALS ** 2 < 2 ** 31


def test_context_free_entry_rejects_invalid_arguments_on_the_host():
    """pt_apply_exchange_noalloc takes no context, and every argument check it makes runs on the
    host before any CUDA call, so the C ABI's error contract is testable without a GPU: each
    invalid request returns PT_INVALID_ARG.  The pointers are 16-byte-aligned placeholders that
    these rejected calls never dereference."""
    from paper_2501_03061_gb300 import _lib
    from paper_2501_03061_gb300 import build
    lib = _lib.load(build.build())
    P = ctypes.c_void_p
    src, occ, out, tgt = P(0x10000), P(0x20000), P(0x30000), P(0x40000)

    def grid(n=(8, 8, 8), L=(5.0, 5.0, 5.0)):
        g = _lib.pt_grid()
        g.nx, g.ny, g.nz = n
        for a in range(3):
            g.L[a] = L[a]
        return g

    def kern(t=1, mu=0.106):
        k = _lib.pt_kernel()
        k.type, k.mu, k.g0 = t, mu, float("nan")
        return k

    def call(src=src, occ=occ, N=4, tgt=None, M=0, out=out, g=None, k=None, prec=0):
        g = grid() if g is None else g
        k = kern() if k is None else k
        return lib.pt_apply_exchange_noalloc(src, occ, N, tgt, M, out, ctypes.byref(g), ctypes.byref(k), prec, None)

    cases = {
        "N = 0": call(N=0),
        "N above PT_MAX_ORBITALS": call(N=_lib.PT_MAX_ORBITALS + 1),
        "N above the static scratch's 1024": call(N=1025),
        "M = 0 with separate targets": call(tgt=tgt, M=0),
        "M above PT_MAX_ORBITALS": call(tgt=tgt, M=_lib.PT_MAX_ORBITALS + 1),
        "NULL occupations": call(occ=None),
        "NULL source block": call(src=None),
        "source not on a 16-byte boundary": call(src=P(0x10008)),
        "output not on a 16-byte boundary": call(out=P(0x30004)),
        "targets not on a 16-byte boundary": call(tgt=P(0x40008), M=2),
        "output aliasing the sources": call(out=src),
        "output aliasing the targets": call(tgt=tgt, M=2, out=tgt),
        "unknown precision": call(prec=7),
        "negative precision": call(prec=-1),
        "unknown kernel type": call(k=kern(t=2)),
        "screened kernel with mu = 0": call(k=kern(mu=0.0)),
        "screened kernel with mu = NaN": call(k=kern(mu=float("nan"))),
        "grid side 14 (not 2,3,5-smooth)": call(g=grid((14, 8, 8))),
        "grid side 128 (above 64)": call(g=grid((8, 128, 8))),
        "grid side 1": call(g=grid((8, 8, 1))),
        "non-positive cell length": call(g=grid(L=(5.0, -1.0, 5.0))),
        "infinite cell length": call(g=grid(L=(5.0, 5.0, float("inf")))),
    }
    bad = {k: _lib.STATUS_NAMES.get(v, v) for k, v in cases.items() if v != _lib.PT_INVALID_ARG}
    assert not bad, bad
    # a NULL grid or kernel is rejected too
    k = kern()
    assert lib.pt_apply_exchange_noalloc(src, occ, 4, None, 0, out, None, ctypes.byref(k), 0, None) == _lib.PT_INVALID_ARG
    g = grid()
    assert lib.pt_apply_exchange_noalloc(src, occ, 4, None, 0, out, ctypes.byref(g), None, 0, None) == _lib.PT_INVALID_ARG


def test_selftest_wait_checks_its_arguments_on_the_host():
    """pt_selftest_wait rejects a NULL context before any CUDA call."""
    from paper_2501_03061_gb300 import _lib
    from paper_2501_03061_gb300 import build
    lib = _lib.load(build.build())
    assert lib.pt_selftest_wait(None, 0, 0.05, None) == _lib.PT_INVALID_ARG
