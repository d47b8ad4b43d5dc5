"""CPU-side checks of the C ABI: the library loads, exports every declared
symbol, sizes workspaces, and rejects bad arguments before touching the GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "llp.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(llp_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    import paper_2603_13147_b300 as llp
    llp.build()
    return llp.lib()


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert "llp_sssp" in names and "llp_bfs" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert missing == []


def test_version_and_status_strings(L):
    import paper_2603_13147_b300 as llp
    assert "sm_103a" in llp.version()
    assert llp.status_string(0) == "ok"
    assert "workspace" in llp.status_string(2)


def test_workspace_sizes_monotone(L):
    import paper_2603_13147_b300 as llp
    a = llp.sssp_workspace_size(1000, 5000)
    b = llp.sssp_workspace_size(2000, 5000)
    c = llp.sssp_workspace_size(2000, 50000)
    assert 4096 < a < b < c
    assert a % 256 == 0
    assert llp.sssp_workspace_size(0, 10) == 0


def test_invalid_arguments_rejected_on_host(L):
    import paper_2603_13147_b300 as llp
    c = llp.Csr()
    c.n, c.m = 10, 0
    c.offsets = 0x1000
    ws = ctypes.c_void_p(0x100000)
    out = ctypes.c_void_p(0x200000)
    # NULL graph / output / workspace
    assert L.llp_sssp(None, 0, out, None, ws, ctypes.c_size_t(1 << 30), None) == llp.LLP_ERR_INVALID_ARG
    assert L.llp_sssp(ctypes.byref(c), 0, None, None, ws, ctypes.c_size_t(1 << 30), None) == llp.LLP_ERR_INVALID_ARG
    # source out of range
    assert L.llp_sssp(ctypes.byref(c), 10, out, None, ws, ctypes.c_size_t(1 << 30), None) == llp.LLP_ERR_INVALID_ARG
    assert L.llp_bfs(ctypes.byref(c), -1, out, None, ws, ctypes.c_size_t(1 << 30), None) == llp.LLP_ERR_INVALID_ARG
    # misaligned workspace
    assert L.llp_bfs(ctypes.byref(c), 0, out, None, ctypes.c_void_p(0x100004), ctypes.c_size_t(1 << 30),
                     None) == llp.LLP_ERR_INVALID_ARG
    # workspace too small
    assert L.llp_bfs(ctypes.byref(c), 0, out, None, ws, ctypes.c_size_t(100), None) == llp.LLP_ERR_WORKSPACE_TOO_SMALL
    # m > 0 without indices
    c.m = 5
    assert L.llp_bfs(ctypes.byref(c), 0, out, None, ws, ctypes.c_size_t(1 << 30), None) == llp.LLP_ERR_INVALID_ARG


def test_pull_and_transpose_arguments_rejected_on_host(L):
    import paper_2603_13147_b300 as llp
    c = llp.Csr()
    c.n, c.m = 10, 0
    c.offsets = 0x1000
    t = llp.Csr()
    t.n, t.m = 10, 0
    t.offsets = 0x3000
    ws = ctypes.c_void_p(0x100000)
    out = ctypes.c_void_p(0x200000)
    big = ctypes.c_size_t(1 << 30)
    # missing transpose, or one that does not match the graph
    assert L.llp_bfs_pull(ctypes.byref(c), None, 0, out, None, ws, big, None) == llp.LLP_ERR_INVALID_ARG
    for field, val in (("n", 11), ("m", 3), ("offsets_64", 1), ("offsets", None)):
        bad = llp.Csr()
        ctypes.pointer(bad)[0] = t
        setattr(bad, field, val)
        assert L.llp_bfs_pull(ctypes.byref(c), ctypes.byref(bad), 0, out, None, ws, big, None) == \
            llp.LLP_ERR_INVALID_ARG, field
    assert L.llp_bfs_pull(ctypes.byref(c), ctypes.byref(t), 10, out, None, ws, big, None) == llp.LLP_ERR_INVALID_ARG
    # transpose: NULL outputs, misaligned or small workspace
    L.llp_csr_transpose_workspace_size.restype = ctypes.c_size_t
    assert L.llp_csr_transpose_workspace_size(ctypes.c_int32(10), ctypes.c_int64(0)) > 4096
    assert L.llp_csr_transpose(ctypes.byref(c), None, None, None, ws, big, None) == llp.LLP_ERR_INVALID_ARG
    assert L.llp_csr_transpose(ctypes.byref(c), out, None, None, ctypes.c_void_p(0x100004), big,
                               None) == llp.LLP_ERR_INVALID_ARG
    assert L.llp_csr_transpose(ctypes.byref(c), out, None, None, ws, ctypes.c_size_t(64),
                               None) == llp.LLP_ERR_WORKSPACE_TOO_SMALL
    c.m = 5  # arcs but no indices
    assert L.llp_csr_transpose(ctypes.byref(c), out, ctypes.c_void_p(0x300000), None, ws, big,
                               None) == llp.LLP_ERR_INVALID_ARG


def test_warm_arguments_rejected_on_host(L):
    import paper_2603_13147_b300 as llp
    c = llp.Csr()
    c.n, c.m = 10, 0
    c.offsets = 0x1000
    ws = ctypes.c_void_p(0x100000)
    out = ctypes.c_void_p(0x200000)
    big = ctypes.c_size_t(1 << 30)
    for f in (L.llp_sssp_warm, L.llp_bfs_warm):
        assert f(ctypes.byref(c), 0, out, None, -1, None, ws, big, None) == llp.LLP_ERR_INVALID_ARG
        assert f(ctypes.byref(c), 0, out, None, 3, None, ws, big, None) == llp.LLP_ERR_INVALID_ARG
        assert f(ctypes.byref(c), 10, out, None, 0, None, ws, big, None) == llp.LLP_ERR_INVALID_ARG
        assert f(ctypes.byref(c), 0, out, None, 0, None, ws, ctypes.c_size_t(64), None) == \
            llp.LLP_ERR_WORKSPACE_TOO_SMALL


def test_host_entry_arguments_rejected_on_host(L):
    import paper_2603_13147_b300 as llp
    c = llp.Csr()
    c.n, c.m = 10, 5
    c.offsets = 0x1000
    ws = ctypes.c_void_p(0x100000)
    out = ctypes.c_void_p(0x200000)
    big = ctypes.c_size_t(1 << 30)
    L.llp_sssp_host_workspace_size.restype = ctypes.c_size_t
    need = L.llp_sssp_host_workspace_size(ctypes.c_int32(10), ctypes.c_int64(5), ctypes.c_int32(0))
    L.llp_sssp_workspace_size.restype = ctypes.c_size_t
    assert need > L.llp_sssp_workspace_size(ctypes.c_int32(10), ctypes.c_int64(5))
    assert L.llp_sssp_host(ctypes.byref(c), 0, out, None, ws, big, None) == llp.LLP_ERR_INVALID_ARG  # no indices
    c.m = 0
    assert L.llp_sssp_host(None, 0, out, None, ws, big, None) == llp.LLP_ERR_INVALID_ARG
    assert L.llp_sssp_host(ctypes.byref(c), 0, None, None, ws, big, None) == llp.LLP_ERR_INVALID_ARG
    assert L.llp_sssp_host(ctypes.byref(c), 10, out, None, ws, big, None) == llp.LLP_ERR_INVALID_ARG
    assert L.llp_sssp_host(ctypes.byref(c), 0, out, None, ctypes.c_void_p(0x100010), big,
                           None) == llp.LLP_ERR_INVALID_ARG
    assert L.llp_sssp_host(ctypes.byref(c), 0, out, None, ws, ctypes.c_size_t(128),
                           None) == llp.LLP_ERR_WORKSPACE_TOO_SMALL
