"""B300-native F4 over F_p: the Python binding of include/gb.h.

Argument marshalling only: every step of the hot path runs in the CUDA kernels of libgb.so
(built in-tree by `paper_2601_06765_b300.build`).  PyTorch supplies device memory (the context's
arena is a torch tensor) and the stream.  There is no fallback: when libgb.so is missing or no
GPU is present, the calls raise.

Functions keep the C names (gb_ctx_create, gb_system_create, gb_symbolic_preprocess,
gb_reduce_macaulay, gb_f4_step, gb_groebner, ...).  `Context` and `System` wrap them for tests and
benchmarks.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgb.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "gb.h")

GB_OK, GB_DONE = 0, 1
STATUS = {0: "GB_OK", 1: "GB_DONE", -1: "GB_EINVAL", -2: "GB_ENOMEM", -3: "GB_EOVERFLOW",
          -4: "GB_ETIMEOUT", -5: "GB_EDEVICE", -6: "GB_EUNSUPPORTED", -7: "GB_EBUSY"}
GB_CTX_KEEP_STEP = 1
GB_CTX_REDUCE_SPARSE = 2
GB_CTX_REDUCE_DENSE = 4
GB_CTX_NO_GRAPHS = 8
GB_CTX_SP_HASH = 16
GB_CTX_SKETCH = 32
GB_F5_NO_CRITERION = 1
GB_GREVLEX, GB_DEGLEX = 0, 1  # gb_order
# gb_modp_op
(GB_MODP_REDUCE64, GB_MODP_REDUCE32, GB_MODP_MULADD, GB_MODP_REDC, GB_MODP_TO_MONT, GB_MODP_MONT_MUL,
 GB_MODP_INV, GB_MODP_INV_SMALL, GB_MODP_LAZY32, GB_MODP_LAZY_MONT, GB_MODP_CHAIN_BARRETT,
 GB_MODP_CHAIN_MONT) = range(12)
_ORDERS = {"grevlex": GB_GREVLEX, "deglex": GB_DEGLEX}

_u8p = ctypes.POINTER(ctypes.c_uint8)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_vp = ctypes.c_void_p


class gb_ctx_opts(ctypes.Structure):
    _fields_ = [("stream", _vp), ("arena", _vp), ("arena_bytes", ctypes.c_size_t),
                ("flags", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class gb_polys(ctypes.Structure):
    _fields_ = [("npolys", ctypes.c_uint32), ("poly_off", _u32p), ("exps", _u8p), ("coeffs", _u32p)]


class gb_polys_host(ctypes.Structure):
    _fields_ = [("npolys", ctypes.c_uint32), ("nterms", ctypes.c_uint64), ("poly_off", _u32p),
                ("exps", _u8p), ("coeffs", _u32p)]


class gb_macaulay_host(ctypes.Structure):
    _fields_ = [("nvars", ctypes.c_uint32), ("nrows", ctypes.c_uint32), ("ndict", ctypes.c_uint32),
                ("npivot", ctypes.c_uint32), ("nnz", ctypes.c_uint64), ("row_ptr", _u32p),
                ("col_ind", _u32p), ("val", _u32p), ("dict_exps", _u8p), ("row_t", _u8p),
                ("row_k", _u32p), ("row_flags", _u8p)]


class gb_echelon_host(ctypes.Structure):
    _fields_ = [("nC", ctypes.c_uint32), ("nb", ctypes.c_uint32), ("rank", ctypes.c_uint32),
                ("nonpiv", _u32p), ("dprime", _u32p), ("rref_piv", _u32p), ("rref", _u32p)]


class gb_step_stats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint32) for f in ("step", "degree", "npairs", "nrows", "ndict", "npivot",
                                                "nC", "nb", "rank", "nbasis", "closure_rounds",
                                                "sp_redo")] + \
               [("nnz", ctypes.c_uint64), ("axpy_rows", ctypes.c_uint64), ("axpy_fma", ctypes.c_uint64),
                ("ms_sp", ctypes.c_float), ("ms_reduce", ctypes.c_float),
                ("ms_rref", ctypes.c_float), ("ms_update", ctypes.c_float), ("ms_pairs", ctypes.c_float),
                ("ms_select", ctypes.c_float), ("ms_reduce_kernel", ctypes.c_float),
                ("ms_wall", ctypes.c_double), ("ms_mm", ctypes.c_double), ("mm_flops", ctypes.c_double),
                ("mm_launches", ctypes.c_uint64), ("rref_sketched", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class gb_run_stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_uint32), ("nbasis", ctypes.c_uint32), ("nnz_total", ctypes.c_uint64),
                ("axpy_rows", ctypes.c_uint64), ("axpy_fma", ctypes.c_uint64),
                ("ms_sp", ctypes.c_double), ("ms_reduce", ctypes.c_double), ("ms_rref", ctypes.c_double),
                ("ms_update", ctypes.c_double), ("ms_pairs", ctypes.c_double),
                ("ms_select", ctypes.c_double), ("ms_wall", ctypes.c_double),
                ("ms_reduce_kernel", ctypes.c_double), ("ms_finish", ctypes.c_double),
                ("nnz_steps", ctypes.c_uint64), ("ms_mm", ctypes.c_double), ("mm_flops", ctypes.c_double),
                ("mm_launches", ctypes.c_uint64)]


class gb_krylov_stats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint32) for f in ("b", "d", "nterms", "hankel_rank", "free_columns", "found",
                                                "verified", "reserved")] + \
               [("spmm_products", ctypes.c_uint64), ("ms_sequence", ctypes.c_double),
                ("ms_hankel", ctypes.c_double), ("ms_vectors", ctypes.c_double), ("ms_total", ctypes.c_double)]


class gb_macaulay_stats(ctypes.Structure):
    _fields_ = [("nrows", ctypes.c_uint32), ("ndict", ctypes.c_uint32), ("npivot", ctypes.c_uint32),
                ("closure_rounds", ctypes.c_uint32), ("nnz", ctypes.c_uint64), ("ms_sp", ctypes.c_float),
                ("ms_dict", ctypes.c_float), ("ms_assemble", ctypes.c_float), ("reserved", ctypes.c_uint32)]


class gb_f5_block(ctypes.Structure):
    _fields_ = [("degree", ctypes.c_uint32), ("index", ctypes.c_uint32), ("candidates", ctypes.c_uint32),
                ("admissible", ctypes.c_uint32), ("rows", ctypes.c_uint32), ("ndict", ctypes.c_uint32),
                ("npivot", ctypes.c_uint32), ("nC", ctypes.c_uint32), ("rank", ctypes.c_uint32),
                ("zero_reductions", ctypes.c_uint32), ("ms_filter", ctypes.c_float), ("ms_sp", ctypes.c_float),
                ("ms_reduce", ctypes.c_float), ("ms_rref", ctypes.c_float)]


class gb_f5_stats(ctypes.Structure):
    _fields_ = [("blocks", ctypes.c_uint32), ("nbasis", ctypes.c_uint32), ("candidates", ctypes.c_uint64),
                ("admissible", ctypes.c_uint64), ("zero_reductions", ctypes.c_uint64), ("nnz", ctypes.c_uint64),
                ("ms_wall", ctypes.c_double), ("ms_filter", ctypes.c_double), ("ms_sp", ctypes.c_double),
                ("ms_reduce", ctypes.c_double), ("ms_rref", ctypes.c_double), ("ms_finish", ctypes.c_double)]


class gb_server_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_uint64), ("system_steps", ctypes.c_uint64),
                ("admitted", ctypes.c_uint64), ("finished", ctypes.c_uint64), ("busy_ms", ctypes.c_double),
                ("max_running", ctypes.c_uint32), ("queued", ctypes.c_uint32),
                ("finish_passes", ctypes.c_uint64), ("finish_ms", ctypes.c_double)]


class gb_tune_report(ctypes.Structure):
    _fields_ = [("runs", ctypes.c_uint32), ("steps", ctypes.c_uint32), ("buckets_reduce", ctypes.c_uint32),
                ("buckets_rref", ctypes.c_uint32), ("dense_buckets", ctypes.c_uint32),
                ("buckets_scan", ctypes.c_uint32), ("ms_wall", ctypes.c_double)]


class gb_server_opts(ctypes.Structure):
    _fields_ = [("hbm_cap_bytes", ctypes.c_size_t), ("max_slots", ctypes.c_uint32),
                ("finish_min", ctypes.c_uint32), ("admit_min", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


def _struct_dict(s) -> dict:
    return {f: getattr(s, f) for f, _ in s._fields_ if f != "reserved"}


class GbError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {detail}")
        self.status = status


_lib = None

_SIGS = {
    "gb_ctx_create": [ctypes.c_int, ctypes.POINTER(gb_ctx_opts), ctypes.POINTER(_vp)],
    "gb_ctx_destroy": [_vp],
    "gb_ctx_memory": [_vp, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)],
    "gb_ctx_memory_peak": [_vp, ctypes.POINTER(ctypes.c_size_t), ctypes.c_int],
    "gb_system_create": [_vp, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int, ctypes.POINTER(gb_polys),
                         ctypes.POINTER(_vp)],
    "gb_system_destroy": [_vp],
    "gb_symbolic_preprocess": [_vp, ctypes.c_uint32, _u8p, _u32p, ctypes.c_int, ctypes.POINTER(_vp)],
    "gb_macaulay_export": [_vp, ctypes.POINTER(gb_macaulay_host)],
    "gb_macaulay_destroy": [_vp],
    "gb_macaulay_stats_get": [_vp, ctypes.POINTER(gb_macaulay_stats)],
    "gb_reduce_macaulay": [_vp, ctypes.POINTER(_vp)],
    "gb_echelon_export": [_vp, ctypes.POINTER(gb_echelon_host)],
    "gb_echelon_destroy": [_vp],
    "gb_f4_step": [_vp, ctypes.POINTER(gb_step_stats)],
    "gb_groebner": [_vp, ctypes.POINTER(gb_run_stats)],
    "gb_basis_export": [_vp, ctypes.c_int, ctypes.POINTER(gb_polys_host)],
    "gb_basis_redundant": [_vp, _u32p, _u8p],
    "gb_system_last_step": [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp)],
    "gb_batch_groebner": [_vp, ctypes.c_uint32, ctypes.POINTER(_vp), ctypes.POINTER(gb_run_stats)],
    "gb_autotune": [_vp, ctypes.c_uint32, ctypes.POINTER(_vp), ctypes.POINTER(gb_tune_report)],
    "gb_tune_save": [_vp, ctypes.c_char_p],
    "gb_tune_load": [_vp, ctypes.c_char_p],
    "gb_server_create": [_vp, ctypes.POINTER(gb_server_opts), ctypes.POINTER(_vp)],
    "gb_server_submit": [_vp, _vp, ctypes.POINTER(ctypes.c_uint64)],
    "gb_server_poll": [_vp, ctypes.c_uint64, ctypes.POINTER(_vp), ctypes.POINTER(ctypes.c_int)],
    "gb_server_destroy": [_vp],
    "gb_server_stats_get": [_vp, ctypes.POINTER(gb_server_stats)],
    "gb_reduce_rows_noalloc": [ctypes.c_uint32] * 5 + [_vp] * 7,
    "gb_modp_apply": [ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32] + [_vp] * 5,
    "gb_pair_update_replay": [ctypes.c_uint32, ctypes.c_uint32, _u8p, ctypes.c_uint32, _u32p, _u8p,
                              ctypes.c_uint32, _u32p, _u32p, _u8p],
    "gb_block_wiedemann": [_vp, ctypes.c_uint32, _u32p, _u32p, _u32p, _u32p, _u32p, ctypes.c_uint32,
                           ctypes.POINTER(gb_krylov_stats)],
    "gb_sig_filter": [_vp, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, _vp, _vp, _u32p],
    "gb_f5_groebner": [_vp, ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(gb_f5_block), ctypes.c_uint32, _u32p,
                       ctypes.POINTER(gb_f5_stats)],
    "gb_matmul_modp": [_vp] + [ctypes.c_uint32] * 4 + [_vp, ctypes.c_uint64, _vp, ctypes.c_uint64, _vp,
                                                       ctypes.c_uint64, ctypes.c_int],
}


def lib():
    """libgb.so, loaded once.  Raises when it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run python -m paper_2601_06765_b300.build")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.gb_status_str.argtypes = [ctypes.c_int]
        L.gb_status_str.restype = ctypes.c_char_p
        L.gb_last_error.argtypes = []
        L.gb_last_error.restype = ctypes.c_char_p
        L.gb_kernel_launches.argtypes = []
        L.gb_kernel_launches.restype = ctypes.c_uint64
        L.gb_graph_launches.argtypes = []
        L.gb_graph_launches.restype = ctypes.c_uint64
        _lib = L
    return _lib


def check(status: int, where: str) -> int:
    if status < 0:
        raise GbError(status, where, lib().gb_last_error().decode(errors="replace"))
    return status


def gb_kernel_launches() -> int:
    return int(lib().gb_kernel_launches())


def gb_graph_launches() -> int:
    return int(lib().gb_graph_launches())


def _p(a: np.ndarray | None, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct)) if a is not None else None


# ---- thin wrappers with the C names --------------------------------------------------------------

def gb_ctx_create(device: int = 0, stream: int | None = None, arena_ptr: int | None = None,
                  arena_bytes: int = 0, flags: int = 0) -> int:
    o = gb_ctx_opts(stream or None, arena_ptr or None, arena_bytes, flags, 0)
    h = _vp()
    check(lib().gb_ctx_create(device, ctypes.byref(o), ctypes.byref(h)), "gb_ctx_create")
    return h.value


def gb_ctx_destroy(ctx: int) -> None:
    check(lib().gb_ctx_destroy(ctx), "gb_ctx_destroy")


def _polys(system: dict):
    off = np.ascontiguousarray(system["poly_off"], dtype=np.uint32)
    ex = np.ascontiguousarray(system["exps"], dtype=np.uint8).reshape(-1)
    cf = np.ascontiguousarray(system["coeffs"], dtype=np.uint32)
    if ex.size == 0:
        ex = np.zeros(1, np.uint8)
        cf = np.zeros(1, np.uint32)
    keep = (off, ex, cf)
    return gb_polys(int(system["m"]), _p(off, ctypes.c_uint32), _p(ex, ctypes.c_uint8),
                    _p(cf, ctypes.c_uint32)), keep


def gb_system_create(ctx: int, system: dict) -> int:
    """A system from its dict; the optional key "order" is "grevlex" (the default) or "deglex"."""
    order = system.get("order", "grevlex")
    if order not in _ORDERS:
        raise ValueError(f"unknown term order {order!r}")
    F, keep = _polys(system)
    h = _vp()
    check(lib().gb_system_create(ctx, int(system["n"]), int(system["p"]), _ORDERS[order], ctypes.byref(F),
                                 ctypes.byref(h)), "gb_system_create")
    del keep
    return h.value


def gb_system_destroy(sys_h: int) -> None:
    check(lib().gb_system_destroy(sys_h), "gb_system_destroy")


def gb_symbolic_preprocess(sys_h: int, n: int, t_exps: np.ndarray, k: np.ndarray, closure: bool) -> int:
    t = np.ascontiguousarray(t_exps, dtype=np.uint8).reshape(-1, n)
    kk = np.ascontiguousarray(k, dtype=np.uint32)
    h = _vp()
    check(lib().gb_symbolic_preprocess(sys_h, len(kk), _p(t, ctypes.c_uint8), _p(kk, ctypes.c_uint32),
                                       int(bool(closure)), ctypes.byref(h)), "gb_symbolic_preprocess")
    return h.value


def gb_macaulay_export(mac: int) -> dict:
    L = lib()
    h = gb_macaulay_host()
    check(L.gb_macaulay_export(mac, ctypes.byref(h)), "gb_macaulay_export")
    n, r, N, M = h.nvars, h.nrows, h.ndict, h.nnz
    out = {"row_ptr": np.zeros(r + 1, np.uint32), "col": np.zeros(max(M, 1), np.uint32),
           "val": np.zeros(max(M, 1), np.uint32), "dict_exps": np.zeros((max(N, 1), n), np.uint8),
           "row_t": np.zeros((max(r, 1), n), np.uint8), "row_k": np.zeros(max(r, 1), np.uint32),
           "row_flags": np.zeros(max(r, 1), np.uint8)}
    h.row_ptr = _p(out["row_ptr"], ctypes.c_uint32)
    h.col_ind = _p(out["col"], ctypes.c_uint32)
    h.val = _p(out["val"], ctypes.c_uint32)
    h.dict_exps = _p(out["dict_exps"], ctypes.c_uint8)
    h.row_t = _p(out["row_t"], ctypes.c_uint8)
    h.row_k = _p(out["row_k"], ctypes.c_uint32)
    h.row_flags = _p(out["row_flags"], ctypes.c_uint8)
    check(L.gb_macaulay_export(mac, ctypes.byref(h)), "gb_macaulay_export")
    out["col"], out["val"] = out["col"][:M], out["val"][:M]
    out["dict_exps"], out["row_t"] = out["dict_exps"][:N], out["row_t"][:r]
    out["row_k"], out["row_flags"] = out["row_k"][:r], out["row_flags"][:r]
    out["npivot"] = h.npivot
    return out


def gb_macaulay_destroy(mac: int) -> None:
    check(lib().gb_macaulay_destroy(mac), "gb_macaulay_destroy")


def gb_reduce_macaulay(mac: int) -> int:
    h = _vp()
    check(lib().gb_reduce_macaulay(mac, ctypes.byref(h)), "gb_reduce_macaulay")
    return h.value


def gb_echelon_export(ech: int) -> dict:
    L = lib()
    h = gb_echelon_host()
    check(L.gb_echelon_export(ech, ctypes.byref(h)), "gb_echelon_export")
    nC, nb, rank = h.nC, h.nb, h.rank
    out = {"nonpiv": np.zeros(max(nb, 1), np.uint32), "dprime": np.zeros(max(nC * nb, 1), np.uint32),
           "rref_piv": np.zeros(max(rank, 1), np.uint32), "rref": np.zeros(max(rank * nb, 1), np.uint32)}
    h.nonpiv = _p(out["nonpiv"], ctypes.c_uint32)
    h.dprime = _p(out["dprime"], ctypes.c_uint32)
    h.rref_piv = _p(out["rref_piv"], ctypes.c_uint32)
    h.rref = _p(out["rref"], ctypes.c_uint32)
    check(L.gb_echelon_export(ech, ctypes.byref(h)), "gb_echelon_export")
    out["nonpiv"] = out["nonpiv"][:nb]
    out["dprime"] = out["dprime"][:nC * nb].reshape(nC, nb)
    out["rref_piv"] = out["rref_piv"][:rank]
    out["rref"] = out["rref"][:rank * nb].reshape(rank, nb)
    return out


def gb_echelon_destroy(ech: int) -> None:
    check(lib().gb_echelon_destroy(ech), "gb_echelon_destroy")


def gb_f4_step(sys_h: int) -> tuple[int, dict]:
    st = gb_step_stats()
    s = check(lib().gb_f4_step(sys_h, ctypes.byref(st)), "gb_f4_step")
    return s, _struct_dict(st)


def gb_groebner(sys_h: int) -> dict:
    st = gb_run_stats()
    check(lib().gb_groebner(sys_h, ctypes.byref(st)), "gb_groebner")
    return _struct_dict(st)


def gb_basis_export(sys_h: int, n: int, reduced: bool = True) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    L = lib()
    h = gb_polys_host()
    check(L.gb_basis_export(sys_h, int(reduced), ctypes.byref(h)), "gb_basis_export")
    off = np.zeros(h.npolys + 1, np.uint32)
    ex = np.zeros((max(h.nterms, 1), n), np.uint8)
    cf = np.zeros(max(h.nterms, 1), np.uint32)
    h.poly_off, h.exps, h.coeffs = _p(off, ctypes.c_uint32), _p(ex, ctypes.c_uint8), _p(cf, ctypes.c_uint32)
    check(L.gb_basis_export(sys_h, int(reduced), ctypes.byref(h)), "gb_basis_export")
    T = int(off[-1]) if off.size else 0
    return off, ex[:T], cf[:T]


def gb_basis_redundant(sys_h: int) -> np.ndarray:
    L = lib()
    c = ctypes.c_uint32()
    check(L.gb_basis_redundant(sys_h, ctypes.byref(c), None), "gb_basis_redundant")
    out = np.zeros(max(c.value, 1), np.uint8)
    check(L.gb_basis_redundant(sys_h, ctypes.byref(c), _p(out, ctypes.c_uint8)), "gb_basis_redundant")
    return out[:c.value]


def gb_system_last_step(sys_h: int) -> tuple[int, int]:
    m, e = _vp(), _vp()
    check(lib().gb_system_last_step(sys_h, ctypes.byref(m), ctypes.byref(e)), "gb_system_last_step")
    return m.value, e.value


def gb_batch_groebner(ctx: int, systems: list[int]) -> list[dict]:
    arr = (_vp * max(len(systems), 1))(*systems)
    st = (gb_run_stats * max(len(systems), 1))()
    check(lib().gb_batch_groebner(ctx, len(systems), arr, st), "gb_batch_groebner")
    return [_struct_dict(st[i]) for i in range(len(systems))]


def gb_autotune(ctx: int, systems: list[int]) -> dict:
    """Time the reduction schedules on copies of `systems` (fresh system handles of ctx) and keep
    the fastest per shape bucket in the context's table; returns the tuning report."""
    arr = (_vp * max(len(systems), 1))(*systems)
    rep = gb_tune_report()
    check(lib().gb_autotune(ctx, len(systems), arr, ctypes.byref(rep)), "gb_autotune")
    return _struct_dict(rep)


def gb_tune_save(ctx: int, path: str) -> None:
    check(lib().gb_tune_save(ctx, os.fsencode(path)), "gb_tune_save")


def gb_tune_load(ctx: int, path: str) -> None:
    check(lib().gb_tune_load(ctx, os.fsencode(path)), "gb_tune_load")


def gb_server_create(ctx: int, hbm_cap_bytes: int, max_slots: int = 0, finish_min: int = 0,
                     admit_min: int = 0) -> int:
    o = gb_server_opts(hbm_cap_bytes, max_slots, finish_min, admit_min, 0)
    h = _vp()
    check(lib().gb_server_create(ctx, ctypes.byref(o), ctypes.byref(h)), "gb_server_create")
    return h.value


def gb_server_submit(srv: int, sys_h: int) -> int:
    t = ctypes.c_uint64()
    check(lib().gb_server_submit(srv, sys_h, ctypes.byref(t)), "gb_server_submit")
    return t.value


def gb_server_poll(srv: int, ticket: int) -> tuple[int | None, int]:
    """(system handle, its status) when finished, else (None, GB_EBUSY)."""
    d = _vp()
    r = ctypes.c_int()
    s = lib().gb_server_poll(srv, ticket, ctypes.byref(d), ctypes.byref(r))
    if s == -7:
        return None, s
    check(s, "gb_server_poll")
    return d.value, r.value


def gb_server_stats_get(srv: int) -> dict:
    st = gb_server_stats()
    check(lib().gb_server_stats_get(srv, ctypes.byref(st)), "gb_server_stats_get")
    return _struct_dict(st)


def gb_server_destroy(srv: int) -> None:
    check(lib().gb_server_destroy(srv), "gb_server_destroy")


def gb_reduce_rows_noalloc(p: int, ndict: int, npivot: int, nnonpivot: int, nb: int, row_ptr: int,
                           col_ind: int, val: int, pivot_cols: int, nonpivot_cols: int, dprime: int,
                           stream: int | None = None) -> None:
    """The sparse reduction on caller-owned device buffers (integer device addresses); no device
    memory is allocated.  See include/gb.h for the layout and the limits."""
    check(lib().gb_reduce_rows_noalloc(p, ndict, npivot, nnonpivot, nb, row_ptr, col_ind, val,
                                       pivot_cols, nonpivot_cols, dprime, stream or None),
          "gb_reduce_rows_noalloc")


def gb_block_wiedemann(mac: int, b: int, X: np.ndarray, Z: np.ndarray, delta: np.ndarray,
                       want_seq: bool = True, wcap: int | None = None) -> dict:
    """Left kernel vectors of a Macaulay matrix handle by the block Wiedemann method (Sec. 9.3):
    X, Z (r x b) and delta (N) are the caller's random choices.  Returns the stats, the
    sequence (2d x b x b) and W (found x r).  See include/gb.h."""
    X = np.ascontiguousarray(X, dtype=np.uint32)
    Z = np.ascontiguousarray(Z, dtype=np.uint32)
    delta = np.ascontiguousarray(delta, dtype=np.uint32)
    r = X.shape[0]
    d = (r + max(b, 1) - 1) // max(b, 1) + 1  # b out of range is refused by the library
    seq = np.zeros((2 * d, b, b), np.uint32) if want_seq else None
    wcap = b if wcap is None else wcap
    W = np.zeros((max(wcap, 1), r), np.uint32)
    st = gb_krylov_stats()
    check(lib().gb_block_wiedemann(mac, b, _p(X, ctypes.c_uint32), _p(Z, ctypes.c_uint32),
                                   _p(delta, ctypes.c_uint32), _p(seq, ctypes.c_uint32) if want_seq else None,
                                   _p(W, ctypes.c_uint32), wcap, ctypes.byref(st)), "gb_block_wiedemann")
    out = _struct_dict(st)
    out["seq"] = seq
    out["W"] = W[:min(out["found"], wcap)]
    return out


def gb_macaulay_stats_get(mac: int) -> dict:
    """Sizes and DictBuild / RowAssemble device times of a matrix handle.  See include/gb.h."""
    st = gb_macaulay_stats()
    check(lib().gb_macaulay_stats_get(mac, ctypes.byref(st)), "gb_macaulay_stats_get")
    return _struct_dict(st)


def gb_sig_filter(ctx: int, index: int, e: int, ncand: int, forbidden: int | None, keys: int) -> int:
    """The F5 admissibility filter over one block of candidates (integer device addresses of the
    forbidden bitmap, or None, and of the key output); returns the number of admissible keys.
    See include/gb.h."""
    count = ctypes.c_uint32(0)
    check(lib().gb_sig_filter(ctx, index, e, ncand, forbidden or None, keys or None, ctypes.byref(count)),
          "gb_sig_filter")
    return count.value


def gb_f5_groebner(sysh: int, dmax: int, criterion: bool = True, max_blocks: int = 4096) -> tuple[list, dict]:
    """The signature-filtered (F5 criterion) Groebner basis of a homogeneous system up to degree
    dmax: (block records, run statistics).  See include/gb.h."""
    blocks = (gb_f5_block * max_blocks)()
    nb = ctypes.c_uint32(0)
    st = gb_f5_stats()
    check(lib().gb_f5_groebner(sysh, dmax, 0 if criterion else GB_F5_NO_CRITERION, blocks, max_blocks,
                               ctypes.byref(nb), ctypes.byref(st)), "gb_f5_groebner")
    return [_struct_dict(blocks[i]) for i in range(min(nb.value, max_blocks))], _struct_dict(st)


def gb_modp_apply(op: int, p: int, n: int, window: int, a: int, b: int | None, c: int | None, out: int,
                  stream: int | None = None) -> None:
    """One device F_p primitive applied elementwise (integer device addresses; b and c may be None
    where the operation does not read them).  See include/gb.h for the operations."""
    check(lib().gb_modp_apply(op, p, n, window, a, b or None, c or None, out, stream or None), "gb_modp_apply")


def gb_pair_update_replay(n: int, lms: np.ndarray, group_sizes, select_before=None):
    """The host pair bookkeeping replayed on leading monomials lms[nelem][n] (uint8), inserted in
    groups; returns (sorted list of pairs (i, j), in_basis flags).  See include/gb.h."""
    lms = np.ascontiguousarray(lms, dtype=np.uint8).reshape(-1, n)
    nelem = lms.shape[0]
    gs = np.ascontiguousarray(group_sizes, dtype=np.uint32)
    sel = None if select_before is None else np.ascontiguousarray(select_before, dtype=np.uint8)
    inb = np.zeros(max(nelem, 1), dtype=np.uint8)
    npairs = ctypes.c_uint32(0)
    cap = max(nelem * nelem, 1)
    out = np.zeros(2 * cap, dtype=np.uint32)
    u8 = lambda a: a.ctypes.data_as(_u8p)
    check(lib().gb_pair_update_replay(n, nelem, u8(lms) if nelem else None, len(gs),
                                      gs.ctypes.data_as(_u32p) if len(gs) else None,
                                      u8(sel) if sel is not None else None, cap, out.ctypes.data_as(_u32p),
                                      ctypes.byref(npairs), u8(inb)),
          "gb_pair_update_replay")
    k = npairs.value
    pairs = sorted((int(out[2 * q]), int(out[2 * q + 1])) for q in range(k))
    return pairs, [bool(x) for x in inb[:nelem]]


def gb_matmul_modp(ctx: int, p: int, m: int, n: int, k: int, A: int, lda: int, B: int, ldb: int, C: int,
                   ldc: int, subtract: bool = True) -> None:
    """C <- C -/+ A B mod p on the tensor cores; A, B, C are integer device addresses of row-major
    u32 matrices (m x k, k x n, m x n) with the given row pitches.  See include/gb.h."""
    check(lib().gb_matmul_modp(ctx, p, m, n, k, A, lda, B, ldb, C, ldc, 1 if subtract else 0),
          "gb_matmul_modp")


# ---- convenience wrappers -----------------------------------------------------------------------

def basis_terms(off: np.ndarray, ex: np.ndarray, cf: np.ndarray) -> list[list[tuple[tuple[int, ...], int]]]:
    return [[(tuple(int(x) for x in ex[j]), int(cf[j])) for j in range(off[i], off[i + 1])]
            for i in range(len(off) - 1)]


class Context:
    """A library context whose device arena is a torch tensor on `device`."""

    def __init__(self, device: int = 0, arena_bytes: int = 2 << 30, keep_step: bool = False,
                 reduce: str = "auto", stream=None, graphs: bool = True, sp: str = "ranks",
                 sketch: bool = False):
        """reduce: "auto" (per matrix by shape), "sparse" or "dense" (see GB_CTX_REDUCE_*).
        stream: a torch.cuda.Stream the context runs on (default: a stream of its own).
        graphs: False launches the echelon-form rounds one by one (GB_CTX_NO_GRAPHS).
        sp: "ranks" (every term ranked into a bitmap) or "hash" (the hash dictionary,
        GB_CTX_SP_HASH) for symbolic preprocessing.
        sketch: True echelonises tall D' through a random sketch first (GB_CTX_SKETCH)."""
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: this library has no CPU path")
        self.device = device
        self.arena = torch.empty(arena_bytes, dtype=torch.uint8, device=f"cuda:{device}")
        torch.cuda.synchronize(device)
        flags = (GB_CTX_KEEP_STEP if keep_step else 0) | {"auto": 0, "sparse": GB_CTX_REDUCE_SPARSE,
                                                            "dense": GB_CTX_REDUCE_DENSE}[reduce]
        if not graphs:
            flags |= GB_CTX_NO_GRAPHS
        if sketch:
            flags |= GB_CTX_SKETCH
        if sp == "hash":
            flags |= GB_CTX_SP_HASH
        elif sp != "ranks":
            raise ValueError("sp must be 'hash' or 'ranks'")
        self.stream = stream
        self.h = gb_ctx_create(device, stream.cuda_stream if stream is not None else None,
                               self.arena.data_ptr(), arena_bytes, flags)

    def memory(self) -> tuple[int, int]:
        u, c = ctypes.c_size_t(), ctypes.c_size_t()
        check(lib().gb_ctx_memory(self.h, ctypes.byref(u), ctypes.byref(c)), "gb_ctx_memory")
        return u.value, c.value

    def memory_peak(self, reset: bool = False) -> int:
        pk = ctypes.c_size_t()
        check(lib().gb_ctx_memory_peak(self.h, ctypes.byref(pk), int(reset)), "gb_ctx_memory_peak")
        return pk.value

    def close(self):
        if self.h:
            gb_ctx_destroy(self.h)
            self.h = 0

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class System:
    """One polynomial system (a dict from paper_2601_06765_b300.synth) on a Context."""

    def __init__(self, ctx: Context, system: dict):
        self.ctx = ctx
        self.n = int(system["n"])
        self.p = int(system["p"])
        self.h = gb_system_create(ctx.h, system)

    def step(self) -> tuple[int, dict]:
        return gb_f4_step(self.h)

    def groebner(self) -> dict:
        return gb_groebner(self.h)

    def f5(self, dmax: int, criterion: bool = True) -> tuple[list, dict]:
        return gb_f5_groebner(self.h, dmax, criterion)

    def basis(self, reduced: bool = True):
        return basis_terms(*gb_basis_export(self.h, self.n, reduced))

    def redundant(self) -> np.ndarray:
        return gb_basis_redundant(self.h)

    def last_step(self) -> tuple[dict, dict]:
        m, e = gb_system_last_step(self.h)
        return gb_macaulay_export(m), gb_echelon_export(e)

    def close(self):
        if self.h:
            gb_system_destroy(self.h)
            self.h = 0

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
