"""The C-ABI library loads without a GPU and exports every function that
include/hashgraph.h declares; host-side argument checks need no device."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hashgraph.h")


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hg_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    path = __graft_entry__._builder().build()
    return ctypes.CDLL(path), path


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("hg_build", "hg_query_count", "hg_query_gather", "hg_join_count", "hg_free",
                     "hg_sync", "hg_table_view", "hg_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    L, path = lib
    for name in _declared_functions():
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (hg_[a-z_0-9]+)\b", out))
    assert set(_declared_functions()) <= exported


def test_invalid_arguments_are_rejected_without_a_gpu(lib):
    import paper_2104_00792_gb300 as hg
    out = ctypes.c_void_p()
    for kb, vb, B, n in [(3, 0, 16, 0), (4, 2, 16, 0), (4, 0, 0, 0), (4, 0, (1 << 31) + 1, 0), (8, 0, 16, 1 << 32)]:
        cfg = hg.hg_config(kb, vb, B, 0, 0)
        st = hg.lib.hg_build(ctypes.byref(cfg), None, None, n, None, ctypes.byref(out))
        assert st == hg.HG_ERR_INVALID_ARG
        assert out.value is None
        assert hg.lib.hg_last_error()
    cfg = hg.hg_config(4, 0, 16, 0, 0x80)
    assert hg.lib.hg_build(ctypes.byref(cfg), None, None, 0, None, ctypes.byref(out)) == hg.HG_ERR_INVALID_ARG
    cfg = hg.hg_config(4, 4, 16, 0, hg.HG_INDEX_VALUES)
    assert hg.lib.hg_build(ctypes.byref(cfg), None, None, 0, None, ctypes.byref(out)) == hg.HG_ERR_INVALID_ARG
    cfg = hg.hg_config(4, 0, 16, 0, 0)
    assert hg.lib.hg_build(ctypes.byref(cfg), None, None, 10, None, ctypes.byref(out)) == hg.HG_ERR_INVALID_ARG
    assert hg.lib.hg_query_count(None, None, 0, None, None, None) == hg.HG_ERR_INVALID_ARG
    assert hg.lib.hg_join_count(None, None, 0, None, None) == hg.HG_ERR_INVALID_ARG
    assert hg.lib.hg_free(None, None) == hg.HG_OK
    assert "sm_103a" in hg.hg_version()
    assert "probe" in hg.hg_prof_names()
