"""CPU-side checks of the C-ABI library: it builds, loads, and exports every
symbol the public header declares.  No compute call (no GPU here)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            names += re.findall(r"^\s*(?:int|const char \*)\s*(svdsc_\w+)\s*\(", text, re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2405_18966_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = _declared()
    for want in ("svdsc_create", "svdsc_solve", "svdsc_destroy", "svdsc_strerror"):
        assert want in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT\s+(svdsc_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_binding_loads_and_lists_exports(libpath):
    import paper_2405_18966_gb300 as pkg
    L = pkg.lib()
    assert set(pkg.EXPORTS) == set(_declared())
    for n in pkg.EXPORTS:
        assert hasattr(L, n)
    assert L.svdsc_strerror(pkg.ERR_CSR).decode().startswith("invalid CSR")
    assert L.svdsc_strerror(pkg.NOT_CONVERGED)


def test_bad_arguments_rejected_without_gpu(libpath):
    import ctypes as C
    import paper_2405_18966_gb300 as pkg
    L = pkg.lib()
    h = C.c_void_p()
    assert L.svdsc_create(C.byref(h), None, None, None) == pkg.ERR_ARG
    m = pkg.SvdscMatrix()
    m.format, m.m, m.n = 0, 0, 5
    assert L.svdsc_create(C.byref(h), C.byref(m), None, None) == pkg.ERR_ARG
    assert L.svdsc_solve(None, 1, 1, 1e-10, 1, None, 0, None, None, 1, None, 1, None, 0, None) == pkg.ERR_ARG
    assert L.svdsc_destroy(None) == pkg.OK


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    import paper_2405_18966_gb300 as pkg
    monkeypatch.setattr(pkg, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(pkg, "_lib", None)
    with pytest.raises(RuntimeError):
        pkg.lib()


def test_oracle_builds_independently():
    """The oracle and the CUDA sources share no file, header or include."""
    import oracle
    oracle.build()
    src = open(os.path.join(ROOT, "oracle", "svds_oracle.c")).read()
    assert "#include \"" not in src
    csrc = os.path.join(ROOT, "paper_2405_18966_gb300", "csrc")
    for f in os.listdir(csrc):
        text = open(os.path.join(csrc, f)).read()
        assert "oracle/" not in text and "svds_oracle" not in text and "orc_" not in text
    pkg_init = open(os.path.join(ROOT, "paper_2405_18966_gb300", "__init__.py")).read()
    assert "import oracle" not in pkg_init


def _c_layout(struct, fields, tmp_path):
    """sizeof / offsetof of a header struct, from a C program compiled against
    the public header alone (plain C, no CUDA)."""
    src = tmp_path / f"layout_{struct}.c"
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "svdsc.h"', "int main(void) {",
             f'  printf("size %zu\\n", sizeof({struct}));']
    lines += [f'  printf("{f} %zu\\n", offsetof({struct}, {f}));' for f in fields]
    lines += ["  return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / f"layout_{struct}"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    return {k: int(v) for k, v in (ln.split() for ln in out.splitlines())}


@pytest.mark.parametrize("struct,cls", [("svdsc_matrix", "SvdscMatrix"), ("svdsc_options", "SvdscOptions"),
                                        ("svdsc_info", "SvdscInfo")])
def test_binding_struct_layouts_match_the_header(struct, cls, tmp_path):
    """The ctypes mirrors in the Python binding have the header's size and
    field offsets (the header is the contract; the binding only marshals)."""
    import paper_2405_18966_gb300 as pkg
    C = getattr(pkg, cls)
    fields = [f for f, _ in C._fields_]
    lay = _c_layout(struct, fields, tmp_path)
    import ctypes
    assert ctypes.sizeof(C) == lay["size"], (ctypes.sizeof(C), lay["size"])
    for f in fields:
        assert getattr(C, f).offset == lay[f], (f, getattr(C, f).offset, lay[f])


def test_noalloc_address_table_is_keyed_by_context(tmp_path):
    """svdsc_cgs2_noalloc remembers its scratch array's device address per CUDA
    context ID (a device reset or a second context places the array anew);
    the table's keying is checked here in plain C++ without a GPU."""
    exe = tmp_path / "ctx_cache_test"
    subprocess.run(["g++", "-std=c++17", "-O1", "-Wall", "-Werror",
                    "-I", os.path.join(ROOT, "paper_2405_18966_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "c", "ctx_cache_test.cpp"), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and "OK (0 failures)" in r.stdout, r.stdout


def test_batched_options_rejected_without_gpu(libpath):
    """svdsc_batch_create checks its options before any CUDA call: each bad
    value returns SVDSC_ERR_ARG (and a good set would go on to the device)."""
    import ctypes as C
    import numpy as np
    import paper_2405_18966_gb300 as pkg
    L = pkg.lib()
    rp = np.array([0, 1, 2, 3], dtype=np.int64)
    ci = np.array([0, 1, 2], dtype=np.int32)
    val = np.ones(3, dtype=np.float32)
    m = pkg.SvdscMatrix()
    m.format, m.index_base, m.m, m.n, m.nnz = pkg.CSR_FORMAT, 0, 3, 3, 3
    m.row_ptr, m.col_idx, m.values = rp.ctypes.data, ci.ctypes.data, val.ctypes.data
    m.value_type = pkg.F32
    mats = (pkg.SvdscMatrix * 1)(m)
    k = np.array([1], dtype=np.int32)
    p = np.array([1], dtype=np.int32)
    h = C.c_void_p()
    bad = [dict(precision=pkg.FP64), dict(batch_cluster=3), dict(batch_handoff=-2), dict(batch_order=2),
           dict(batch_lead=-2), dict(block=4)]
    for b in bad:
        opt = pkg.SvdscOptions(pkg.MIXED, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0)
        for f, v in b.items():
            setattr(opt, f, v)
        rc = L.svdsc_batch_create(C.byref(h), 1, mats, k.ctypes.data_as(C.c_void_p),
                                  p.ctypes.data_as(C.c_void_p), C.byref(opt), None)
        assert rc == pkg.ERR_ARG, (b, rc)
