"""CPU checks of the C-ABI library: it builds, loads without a GPU, and
exports every entry point include/tssvd.h declares.  No compute calls."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tssvd.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    # function-pointer types (the row-sharded calls' all-reduce) are not entry points
    src = re.sub(r"typedef\s+\w+\s*\(\s*\*\s*\w+\s*\)\s*\([^;]*\);", "", src)
    names = re.findall(r"^[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "defined")))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for n in ("ts_svd", "ts_svd_f32", "lowrank_svd", "ts_svd_backward", "tssvd_default_opts"):
        assert n in names, names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_1612_08709_gb300 import build as b
    path = b.build()
    L = ctypes.CDLL(path)
    for n in declared_functions():
        assert hasattr(L, n), "missing export: " + n
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True,
                         text=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if l.strip())
    for n in declared_functions():
        assert n in exported


def test_binding_names_match_the_header():
    import paper_1612_08709_gb300 as pkg
    names = declared_functions()
    for n in pkg.exported_symbols():
        assert n in names


def test_default_opts_and_status_strings_without_gpu():
    import paper_1612_08709_gb300 as pkg
    from paper_1612_08709_gb300._binding import _Opts
    L = pkg.lib()
    o = _Opts()
    L.tssvd_default_opts(ctypes.byref(o))
    assert o.passes == 2 and o.scale == 1 and o.max_sweeps == 50
    assert abs(o.drop_tol - 1e-11 ** 0.5) < 1e-20
    assert L.tssvd_status_string(0) == b"ok"
    assert b"invalid" in L.tssvd_status_string(-3)
    # the workspace query is host arithmetic only
    ws = L.ts_svd_workspace_size(20000, 50, 8, ctypes.byref(o))
    assert ws >= 20000 * 50 * 8


def test_invalid_arguments_are_rejected_before_any_device_work():
    import paper_1612_08709_gb300 as pkg
    from paper_1612_08709_gb300._binding import _Opts
    L = pkg.lib()
    o = _Opts()
    L.tssvd_default_opts(ctypes.byref(o))
    p = ctypes.c_void_p(16)
    assert L.ts_svd(None, 10, 3, 3, p, p, p, ctypes.byref(o)) == -1
    assert L.ts_svd(p, 2, 3, 3, p, p, p, ctypes.byref(o)) == -2
    assert L.ts_svd(p, 10, 0, 3, p, p, p, ctypes.byref(o)) == -3
    assert L.ts_svd(p, 10, 3, 2, p, p, p, ctypes.byref(o)) == -4
    assert L.ts_svd(p, 10, 3, 3, None, p, p, ctypes.byref(o)) == -5
    o.passes = 4
    assert L.ts_svd(p, 10, 3, 3, p, p, p, ctypes.byref(o)) == -8
    o.passes = 0
    assert L.ts_svd(p, 10, 3, 3, p, p, p, ctypes.byref(o)) == -8
    L.tssvd_default_opts(ctypes.byref(o))
    assert L.lowrank_svd(p, 10, 8, 8, 5, 4, 2, p, p, p, p, ctypes.byref(o)) == -5
    assert L.lowrank_svd(p, 10, 8, 8, 2, 9, 2, p, p, p, p, ctypes.byref(o)) == -6


def test_pca_argument_validation_without_gpu():
    """ts_pca rejects each invalid argument with its number before it
    touches the device (the pointers below are never dereferenced)."""
    import paper_1612_08709_gb300 as pkg
    from paper_1612_08709_gb300._binding import _Opts
    L = pkg.lib()
    o = _Opts()
    L.tssvd_default_opts(ctypes.byref(o))
    f = ctypes.c_void_p(256)
    assert L.ts_pca(None, 10, 2, 2, f, f, f, f, ctypes.byref(o)) == -1
    assert L.ts_pca(f, 1, 2, 2, f, f, f, f, ctypes.byref(o)) == -2
    assert L.ts_pca(f, 10, 0, 2, f, f, f, f, ctypes.byref(o)) == -3
    assert L.ts_pca(f, 10, 2, 1, f, f, f, f, ctypes.byref(o)) == -4
    assert L.ts_pca(f, 10, 2, 2, None, f, f, f, ctypes.byref(o)) == -5
    assert L.ts_pca(f, 10, 2, 2, f, None, f, f, ctypes.byref(o)) == -6
    assert L.ts_pca(f, 10, 2, 2, f, f, None, f, ctypes.byref(o)) == -7
    assert L.ts_pca(f, 10, 2, 2, f, f, f, None, ctypes.byref(o)) == -8
    assert L.ts_pca(f, 10, 2, 2, f, f, f, f, None) == -9
    o.passes = 4
    assert L.ts_pca(f, 10, 2, 2, f, f, f, f, ctypes.byref(o)) == -9
    # the workspace query is host arithmetic: the SVD's plus the centred copy
    L.tssvd_default_opts(ctypes.byref(o))
    assert (L.ts_pca_workspace_size(20000, 50, 8, ctypes.byref(o)) >=
            L.ts_svd_workspace_size(20000, 50, 8, ctypes.byref(o)) + 20000 * 50 * 8)


def test_tsqr_argument_validation_without_gpu():
    """ts_svd_tsqr rejects NULL or out-of-range arguments before touching
    the device (the pointers below are never dereferenced)."""
    import paper_1612_08709_gb300 as pkg
    from paper_1612_08709_gb300._binding import _Opts
    L = pkg.lib()
    o = _Opts()
    L.tssvd_default_opts(ctypes.byref(o))
    f = ctypes.c_void_p(256)
    assert L.ts_svd_tsqr(None, 10, 2, 2, f, f, f, f, f, ctypes.byref(o)) == -1
    assert L.ts_svd_tsqr(f, 1, 2, 2, f, f, f, f, f, ctypes.byref(o)) == -2
    assert L.ts_svd_tsqr(f, 10000, 5000, 5000, f, f, f, f, f, ctypes.byref(o)) == -3
    assert L.ts_svd_tsqr(f, 10, 2, 1, f, f, f, f, f, ctypes.byref(o)) == -4
    assert L.ts_svd_tsqr(f, 10, 2, 2, None, f, f, f, f, ctypes.byref(o)) == -5
    assert L.ts_svd_tsqr(f, 10, 2, 2, f, None, f, f, f, ctypes.byref(o)) == -6
    assert L.ts_svd_tsqr(f, 10, 2, 2, f, f, None, f, f, ctypes.byref(o)) == -7
    assert L.ts_svd_tsqr(f, 10, 2, 2, f, f, f, None, f, ctypes.byref(o)) == -8
    assert L.ts_svd_tsqr(f, 10, 2, 2, f, f, f, f, None, ctypes.byref(o)) == -9
    assert L.ts_svd_tsqr(f, 10, 2, 2, f, f, f, f, f, None) == -10
    o.passes = 3  # Algorithms 1 and 2 only: no third pass
    assert L.ts_svd_tsqr(f, 10, 2, 2, f, f, f, f, f, ctypes.byref(o)) == -10


def test_lowrank_tsqr_argument_validation_without_gpu():
    import paper_1612_08709_gb300 as pkg
    from paper_1612_08709_gb300._binding import _Opts
    L = pkg.lib()
    o = _Opts()
    L.tssvd_default_opts(ctypes.byref(o))
    f = ctypes.c_void_p(256)
    args = lambda **kw: [kw.get("A", f), kw.get("m", 100), kw.get("n", 50), kw.get("lda", 50),
                         kw.get("k", 5), kw.get("l", 8), kw.get("it", 1), kw.get("Om", f),
                         kw.get("th", f), kw.get("pm", f), kw.get("U", f), kw.get("S", f),
                         kw.get("V", f), kw.get("o", ctypes.byref(o))]
    assert L.lowrank_svd_tsqr(*args(A=None)) == -1
    assert L.lowrank_svd_tsqr(*args(k=9)) == -5
    assert L.lowrank_svd_tsqr(*args(l=51)) == -6
    assert L.lowrank_svd_tsqr(*args(th=None)) == -9
    assert L.lowrank_svd_tsqr(*args(pm=None)) == -10
    assert L.lowrank_svd_tsqr(*args(V=None)) == -13
    assert L.lowrank_svd_tsqr(*args(o=None)) == -14


def test_tsqr_workspace_query_without_gpu():
    """Algorithm 2's workspace holds B*, Q and Q2 (m x n' FP64 each) and the
    reduction tree; the query is host arithmetic (the tree plan) and grows
    with m."""
    import paper_1612_08709_gb300 as pkg
    from paper_1612_08709_gb300._binding import _Opts
    L = pkg.lib()
    o = _Opts()
    L.tssvd_default_opts(ctypes.byref(o))
    small = L.ts_svd_tsqr_workspace_size(20000, 50, ctypes.byref(o))
    big = L.ts_svd_tsqr_workspace_size(200000, 200, ctypes.byref(o))
    odd = L.ts_svd_tsqr_workspace_size(200000, 199, ctypes.byref(o))
    assert small >= 3 * 20000 * 50 * 8
    assert big >= 3 * 200000 * 200 * 8 and big > small
    assert odd >= 3 * 200000 * 200 * 8  # n odd is padded to n + 1
