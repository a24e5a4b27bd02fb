"""The C-ABI library loads and exports every entry point include/shiro.h declares (CPU only).

Also exercises the host-only entry points (workspace sizing, option and partition validation),
which make no CUDA call."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "shiro.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(shiro_[a-z_0-9]+)\s*\(", src)
    return sorted(set(n for n in names if n not in ("shiro_status",)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2512_20178_gb300 import shiro
    return shiro


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    L = lib.lib()
    for n in names:
        assert hasattr(L, n), f"{n} declared in shiro.h but not exported"
    bound = {s[0] for s in lib.SIGNATURES}
    assert set(names) == bound, set(names) ^ bound


def test_version_and_defaults(lib):
    assert lib.lib().shiro_version() >= 100
    o = lib.make_opts()
    d = o.as_dict()
    assert d["chunk_nnz"] >= 32 and d["long_row_nnz"] >= d["chunk_nnz"] and 1 <= d["group_rows"] <= 32


def _ws(lib, M, K, nnz, Pr, Pc, flags=0, vdt=0, **opts):
    A = lib.shiro_csr(M, K, nnz, None, None, None, vdt)
    part = lib.shiro_partition(Pr, Pc, None, None, flags)
    o = lib.make_opts(**opts)
    n = ctypes.c_size_t(0)
    st = lib.lib().shiro_plan_workspace(ctypes.byref(A), ctypes.byref(part), ctypes.byref(o),
                                        ctypes.byref(n))
    return st, n.value


def test_workspace_bounds_grow_with_inputs(lib):
    st, small = _ws(lib, 4096, 4096, 32768, 4, 4)
    assert st == 0 and small > 0
    st, big = _ws(lib, 1 << 20, 1 << 20, 16 << 20, 4, 4)
    assert st == 0 and big > 16 * (16 << 20) // 4
    st, tr = _ws(lib, 1 << 20, 1 << 20, 16 << 20, 4, 4, flags=lib.SHIRO_PLAN_TRANSPOSE)
    assert st == 0 and tr > big


def test_host_validation(lib):
    assert _ws(lib, 10, 10, 5, 0, 1)[0] == 4          # P_r < 1 -> UNSUPPORTED
    assert _ws(lib, 10, 10, 5, 2, 3, flags=lib.SHIRO_PLAN_LOCAL_DIAG)[0] == 1   # needs P_r == P_c
    assert _ws(lib, 10, 10, 5, 2, 2, flags=0x80)[0] == 1                         # unknown flag
    assert _ws(lib, 10, 10, 5, 2, 2, vdt=1)[0] == 4   # BF16 values unsupported
    assert _ws(lib, 10, 10, 5, 2, 2, chunk_nnz=8)[0] == 1
    assert _ws(lib, 10, 10, 5, 2, 2, group_rows=33)[0] == 1
    assert b"group_rows" in lib.lib().shiro_last_error()
    # Pipelines 0-6 and the listed ring / stage depths are accepted, others rejected.
    for pipe in range(7):
        assert _ws(lib, 10, 10, 5, 2, 2, pipeline=pipe)[0] == 0, pipe
    assert _ws(lib, 10, 10, 5, 2, 2, pipeline=8)[0] == 1
    assert _ws(lib, 10, 10, 5, 2, 2, pipeline=-1)[0] == 1
    for rows in (0, 4, 8, 12, 16, 32):
        assert _ws(lib, 10, 10, 5, 2, 2, pipeline=4, stage_rows=rows)[0] == 0, rows
    assert _ws(lib, 10, 10, 5, 2, 2, pipeline=4, stage_rows=5)[0] == 1
    assert b"stage_rows" in lib.lib().shiro_last_error()


def test_custom_bounds_validated(lib):
    A = lib.shiro_csr(10, 10, 0, None, None, None, 0)
    rb = (ctypes.c_int64 * 3)(0, 7, 9)   # does not end at M
    part = lib.shiro_partition(2, 1, ctypes.cast(rb, ctypes.c_void_p), None, 0)
    n = ctypes.c_size_t(0)
    st = lib.lib().shiro_plan_workspace(ctypes.byref(A), ctypes.byref(part), None, ctypes.byref(n))
    assert st == 1


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2512_20178_gb300 import shiro
    monkeypatch.setattr(shiro, "_lib", None)
    monkeypatch.setattr(shiro, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        shiro.lib()
