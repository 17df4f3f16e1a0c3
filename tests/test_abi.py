"""The C ABI library builds, loads without a GPU, and exports every entry point include/gb.h
declares (no compute calls: this runs on the CPU)."""
from __future__ import annotations

import ctypes
import re

import paper_2601_06765_b300 as gb
from paper_2601_06765_b300 import build


def declared_entry_points() -> list[str]:
    src = open(gb.HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gb_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_hot_path_calls():
    names = declared_entry_points()
    for required in ("gb_symbolic_preprocess", "gb_reduce_macaulay", "gb_f4_step", "gb_groebner"):
        assert required in names


def test_library_exports_every_declared_symbol():
    build.build()
    L = ctypes.CDLL(gb.LIB_PATH)
    missing = [n for n in declared_entry_points() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_every_entry_point():
    L = gb.lib()
    for n in declared_entry_points():
        assert hasattr(L, n)
        if n not in ("gb_status_str", "gb_last_error", "gb_kernel_launches", "gb_graph_launches"):
            assert n in gb._SIGS, f"{n} has no binding signature"


def test_status_strings_without_gpu():
    L = gb.lib()
    assert L.gb_status_str(0) == b"GB_OK"
    assert L.gb_status_str(-7) == b"GB_EBUSY"


def test_null_arguments_are_rejected_without_gpu():
    L = gb.lib()
    assert L.gb_ctx_destroy(None) == -1
    assert L.gb_system_destroy(None) == -1
    assert L.gb_f4_step(None, None) == -1
    assert L.gb_macaulay_export(None, None) == -1


def test_binding_constants_match_the_header():
    """The enum and flag values the binding passes are the header's."""
    src = re.sub(r"/\*.*?\*/", "", open(gb.HEADER).read(), flags=re.S)
    vals = {k: int(v, 0) for k, v in re.findall(r"\b(GB_[A-Z0-9_]+)\s*=\s*(-?(?:0x[0-9a-fA-F]+|\d+))", src)}
    vals.update({k: int(v.rstrip("u"), 0) for k, v in re.findall(r"#define\s+(GB_[A-Z0-9_]+)\s+(\d+u?)", src)})
    for name in ("GB_OK", "GB_DONE", "GB_GREVLEX", "GB_DEGLEX", "GB_CTX_KEEP_STEP", "GB_CTX_REDUCE_SPARSE",
                 "GB_CTX_REDUCE_DENSE", "GB_CTX_NO_GRAPHS", "GB_CTX_SP_HASH", "GB_CTX_SKETCH", "GB_MODP_REDUCE64", "GB_MODP_REDUCE32",
                 "GB_MODP_MULADD", "GB_MODP_REDC", "GB_MODP_TO_MONT", "GB_MODP_MONT_MUL", "GB_MODP_INV",
                 "GB_MODP_INV_SMALL", "GB_MODP_LAZY32", "GB_MODP_LAZY_MONT", "GB_MODP_CHAIN_BARRETT", "GB_MODP_CHAIN_MONT", "GB_F5_NO_CRITERION"):
        assert name in vals, name
        assert getattr(gb, name) == vals[name], name
