"""The C-ABI library loads and exports every symbol include/kr.h declares; host-side checks (CPU only).

No call here launches GPU work: only symbol lookup, kr_options_default, and
argument validation that the library performs on the host before any CUDA call.
"""
import ctypes
import os
import re
import shutil

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "kr.h")


def declared_symbols():
    with open(HEADER) as f:
        text = f.read()
    return sorted(set(re.findall(r"^KR_API\s+[\w\s\*]+?\b(kr_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available to build the library")
    from paper_1504_04395_gb300 import build
    return build.build()


def test_header_declares_the_interface():
    syms = declared_symbols()
    for name in ("kr_op_create_csr", "kr_solve", "kr_adjoint_solve", "kr_grad_values", "kr_last_error",
                 "kr_op_apply", "kr_thin_qr"):
        assert name in syms


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_binding_signatures_cover_the_header():
    import paper_1504_04395_gb300 as kr
    assert sorted(kr.SIGNATURES) == declared_symbols()


def test_missing_library_fails_loudly():
    import paper_1504_04395_gb300 as kr
    with pytest.raises(RuntimeError, match="not built"):
        kr.load_library("/nonexistent/libkrylov_gb300.so")


def test_options_default_and_struct_layout(libpath):
    import paper_1504_04395_gb300 as kr
    lib = kr.load_library(libpath)
    o = kr.KrOptions()
    lib.kr_options_default(ctypes.byref(o))
    assert o.tol == 1e-8 and o.maxit == 500 and o.precision == 0 and o.check_every == 8
    assert o.inner_tol == 1e-4 and o.max_outer == 30 and o.host_buffers == 0


def test_struct_layout_matches_c_compiler(tmp_path):
    """ctypes mirrors of kr_options / kr_info have the C compiler's sizes and offsets."""
    import subprocess
    import paper_1504_04395_gb300 as kr
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields_o = [f for f, _ in kr.KrOptions._fields_]
    fields_i = [f for f, _ in kr.KrInfo._fields_]
    src = ['#include <stdio.h>', '#include <stddef.h>', '#include "kr.h"', 'int main(void) {',
           'printf("%zu %zu\\n", sizeof(kr_options), sizeof(kr_info));']
    for f in fields_o:
        src.append('printf("o %s %%zu\\n", offsetof(kr_options, %s));' % (f, f))
    for f in fields_i:
        src.append('printf("i %s %%zu\\n", offsetof(kr_info, %s));' % (f, f))
    src.append("return 0; }")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(src))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    so, si = map(int, out[0].split())
    assert so == ctypes.sizeof(kr.KrOptions)
    assert si == ctypes.sizeof(kr.KrInfo)
    for line in out[1:]:
        if not line.strip():
            continue
        kind, name, off = line.split()
        cls = kr.KrOptions if kind == "o" else kr.KrInfo
        assert getattr(cls, name).offset == int(off), name


def _create(lib, n, rowptr, colidx, vals):
    h = ctypes.c_void_p()
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    ci = np.ascontiguousarray(colidx, dtype=np.int32)
    v = np.ascontiguousarray(vals, dtype=np.complex128)
    st = lib.kr_op_create_csr(n, len(ci), rp.ctypes.data, ci.ctypes.data, v.ctypes.data, 0, ctypes.byref(h))
    return st, h


def test_csr_validation_on_host(libpath):
    import paper_1504_04395_gb300 as kr
    lib = kr.load_library(libpath)
    # rowptr[0] != 0
    st, h = _create(lib, 2, [1, 2, 3], [0, 1], [1, 1])
    assert st == 6 and not h.value
    assert b"rowptr" in lib.kr_last_error()
    # non-monotone rowptr
    st, _ = _create(lib, 3, [0, 2, 1, 3], [0, 1, 2], [1, 1, 1])
    assert st == 6
    # column index out of range
    st, _ = _create(lib, 2, [0, 1, 2], [0, 5], [1, 1])
    assert st == 6 and b"column" in lib.kr_last_error()
    # rowptr[n] != nnz
    st, _ = _create(lib, 2, [0, 1, 1], [0, 1], [1, 1])
    assert st == 6


def test_lattice_operator_validation_on_host(libpath):
    """kr_op_create_lattice4d checks extents, coefficients and the gamma matrices on the host,
    before any device work (no GPU needed)."""
    import paper_1504_04395_gb300 as kr
    from workloads.lattice import GAMMA
    lib = kr.load_library(libpath)

    def create(dims, gamma, diag=(2.2, 0.0), hop=-0.5, links=None):
        dm = np.ascontiguousarray(dims, dtype=np.int64)
        sites = int(np.prod(dm))
        U = np.zeros((4, sites, 3, 3), dtype=np.complex128) if links is None else links
        U = np.ascontiguousarray(U)
        g = np.ascontiguousarray(np.asarray(gamma, dtype=np.complex128))
        d = np.array(diag, dtype=np.float64)
        h = ctypes.c_void_p()
        st = lib.kr_op_create_lattice4d(dm.ctypes.data, d.ctypes.data, float(hop), g.ctypes.data, U.ctypes.data, 0,
                                        ctypes.byref(h))
        return st, h

    st, h = create((3, 3, 2, 3), GAMMA)  # extent below 3
    assert st == 6 and not h.value and b"extent" in lib.kr_last_error()
    bad = GAMMA.copy()
    bad[1, 0, 1] = 0.5  # a second entry in a row
    st, _ = create((3, 3, 3, 3), bad)
    assert st == 6 and b"gamma" in lib.kr_last_error()
    bad = GAMMA.copy()
    bad[2] = np.diag([1, -1, 1, -1])  # entries on the diagonal
    st, _ = create((3, 3, 3, 3), bad)
    assert st == 6 and b"off-diagonal" in lib.kr_last_error()
    bad = GAMMA.copy()
    bad[0, 0, 3] = -bad[0, 0, 3]  # gamma[3][0] no longer the conjugate of gamma[0][3]
    st, _ = create((3, 3, 3, 3), bad)
    assert st == 6 and b"Hermitian" in lib.kr_last_error()
    st, _ = create((3, 3, 3, 3), GAMMA, hop=float("nan"))
    assert st == 6
    links = np.zeros((4, 81, 3, 3), dtype=np.complex128)
    links[1, 5, 2, 2] = np.inf
    st, _ = create((3, 3, 3, 3), GAMMA, links=links)
    assert st == 6 and b"link" in lib.kr_last_error()


def test_solve_argument_checks(libpath):
    import paper_1504_04395_gb300 as kr
    lib = kr.load_library(libpath)
    info = kr.KrInfo()
    # NULL operator
    assert lib.kr_solve(None, 0, 4, None, None, None, None, ctypes.byref(info)) == 6
    assert lib.kr_adjoint_solve(None, 0, 4, None, None, None, None, ctypes.byref(info)) == 6
    assert lib.kr_grad_values(None, 4, None, None, None, None) == 6
    assert lib.kr_op_apply(None, 0, 4, None, None, None) == 6
    assert lib.kr_block_reduce(0, 4, None, None, 1, None, None) == 6
    assert lib.kr_thin_qr(10, 0, None, None, None, None) == 6
    assert lib.kr_op_destroy(None) == 0
