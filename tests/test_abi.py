"""The C-ABI library loads and exports every function declared in include/gcge.h (no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names.update(re.findall(r"\b(gcge_\w+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as ge
    ge.build()
    return ctypes.CDLL(os.path.join(ROOT, "paper_2111_06552_gb300", "libgcge.so"))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("gcge_create", "gcge_solve", "gcge_eigenpairs", "gcge_destroy",
                 "gcge_spmm_f64", "gcge_gram_f32", "gcge_syev", "gcge_block_cg_f64"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_header(lib):
    import paper_2111_06552_gb300 as g
    assert set(_declared()) <= set(g._SIGS)


def test_host_only_calls_without_gpu(lib):
    import paper_2111_06552_gb300 as g
    o = g.gcge_options_default()
    assert o.cg_max_iter == 30 and abs(o.cg_rtol - 1e-2) < 1e-15 and o.orth_leaf == 16
    assert g.lib().gcge_error_string(g.GCGE_EINVAL) == b"invalid argument"
    # invalid sizes are rejected on the host before any device work
    assert g.lib().gcge_create(None, None, 1, 1, 1e-8, None, None, None) == g.GCGE_EINVAL
    assert g.lib().gcge_gram_f64(10, 2, 2, 1.0, None, 1, None, 2, 0.0, None, 2, None) == g.GCGE_EINVAL
    assert g.lib().gcge_syev(4, None, 2, None, None, 4, None, None) == g.GCGE_EINVAL


def test_struct_layout_matches_header(lib):
    import paper_2111_06552_gb300 as g
    # gcge_options_default writes every field; a size mismatch would corrupt the sentinel
    buf = (ctypes.c_char * (ctypes.sizeof(g.gcge_options) + 64))()
    ctypes.memset(buf, 0x5A, len(buf))
    assert lib.gcge_options_default(buf) == 0
    assert bytes(buf[ctypes.sizeof(g.gcge_options):]) == b"\x5a" * 64
