"""THE ORACLE -- test infrastructure only.

A plain CPU F4 over F_p (grevlex, or deglex with the DEGLEX flag; x1 > ... > xn) written in C (`f4_oracle.c`) and loaded here with
ctypes.  Only tests/, the package smoke check and bench.py's CPU-baseline leg may import it; the
product path never does.  It shares no code with the CUDA path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "f4_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

ONE_PAIR = 1
NEWEST_REDUCER = 2
DEGLEX = 4  # the deglex term order instead of grevlex (both x1 > ... > xn)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-Wextra", "-fPIC", "-shared",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load(path: str | None = None):
    """The oracle library (or, for mutation tests, a variant compiled from edited source)."""
    global _lib
    if path is None and _lib is not None:
        return _lib
    lib = ctypes.CDLL(path or build())
    P = ctypes.c_void_p
    u8p = ctypes.POINTER(ctypes.c_uint8)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    i64p = ctypes.POINTER(ctypes.c_int64)
    i32p = ctypes.POINTER(ctypes.c_int32)
    lib.or_new.restype = P
    lib.or_new.argtypes = [ctypes.c_int, ctypes.c_uint32, ctypes.c_int, u32p, u8p, u32p, ctypes.c_int]
    lib.or_free.argtypes = [P]
    lib.or_step.argtypes = [P]
    lib.or_run.argtypes = [P]
    lib.or_finish.argtypes = [P]
    lib.or_npairs.argtypes = [P]
    lib.or_stats.argtypes = [P, i64p]
    lib.or_dict.argtypes = [P, u8p]
    lib.or_rows.argtypes = [P, u8p, u32p, u8p, u8p]
    lib.or_csr.argtypes = [P, u32p, u32p, u32p]
    lib.or_nonpiv.argtypes = [P, u32p]
    lib.or_dprime.argtypes = [P, u32p]
    lib.or_rref.argtypes = [P, u32p, u32p]
    lib.or_snapshot.argtypes = [P, u8p]
    lib.or_ng.argtypes = [P]
    lib.or_poly_len.argtypes = [P, ctypes.c_int]
    lib.or_poly.argtypes = [P, ctypes.c_int, u8p, u32p]
    lib.or_redundant.argtypes = [P, u8p]
    lib.or_pairs.argtypes = [P, i32p]
    lib.or_final_size.argtypes = [P, i64p]
    lib.or_final.argtypes = [P, u32p, u8p, u32p]
    lib.or_reduce_row.argtypes = [ctypes.c_uint32, ctypes.c_int, ctypes.c_int, u32p, u32p, u32p, u32p, u32p,
                                  ctypes.c_uint32, ctypes.c_int, u32p, u32p]
    if path is None:
        _lib = lib
    return lib


def compile_variant(source: str, out_path: str):
    """Compile C source text (an edited copy of f4_oracle.c) and load it."""
    src = out_path + ".c"
    with open(src, "w") as f:
        f.write(source)
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-o", out_path, src])
    return _load(out_path)


def source() -> str:
    with open(_SRC) as f:
        return f.read()


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


@dataclass
class StepDump:
    """Everything the oracle computed in one F4 step (row order, dictionary order as fixed by the
    readings in f4_oracle.c)."""
    step: int
    degree: int
    npairs: int
    dict_exps: np.ndarray      # uint8[N, n], descending
    row_t: np.ndarray          # uint8[r, n]
    row_k: np.ndarray          # uint32[r]
    row_pivot: np.ndarray      # uint8[r]
    row_reducer: np.ndarray    # uint8[r]
    row_ptr: np.ndarray        # uint32[r+1]
    col: np.ndarray            # uint32[M]
    val: np.ndarray            # uint32[M]
    nonpiv: np.ndarray         # uint32[nb] dictionary columns of D'
    dprime: np.ndarray         # uint32[nC, nb]
    rref_piv: np.ndarray       # uint32[rank] positions in [0, nb)
    rref: np.ndarray           # uint32[rank, nb]
    redundant: np.ndarray      # uint8[ng] flags when the rows were chosen
    nA: int = 0
    nC: int = 0

    @property
    def N(self) -> int:
        return int(self.dict_exps.shape[0])

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])


@dataclass
class Oracle:
    """One F4 run of the oracle on one system (dict from paper_2601_06765_b300.synth)."""
    system: dict
    flags: int = 0
    lib: object = None
    _h: int = field(default=0, init=False)

    def __post_init__(self):
        lib = self.lib = self.lib or _load()
        s = self.system
        off = np.ascontiguousarray(s["poly_off"], dtype=np.uint32)
        ex = np.ascontiguousarray(s["exps"], dtype=np.uint8).reshape(-1)
        cf = np.ascontiguousarray(s["coeffs"], dtype=np.uint32)
        if ex.size == 0:
            ex = np.zeros(1, np.uint8)
            cf = np.zeros(1, np.uint32)
        self._h = lib.or_new(int(s["n"]), int(s["p"]), int(s["m"]), _ptr(off, ctypes.c_uint32),
                             _ptr(ex, ctypes.c_uint8), _ptr(cf, ctypes.c_uint32), int(self.flags))
        if not self._h:
            raise ValueError("oracle rejected the system")
        self.n = int(s["n"])
        self.p = int(s["p"])

    def __del__(self):
        if getattr(self, "_h", 0) and self.lib is not None:
            self.lib.or_free(self._h)
            self._h = 0

    # -- driving --------------------------------------------------------------------------
    def step(self) -> bool:
        return bool(self.lib.or_step(self._h))

    def run(self) -> list[list[tuple[tuple[int, ...], int]]]:
        self.lib.or_run(self._h)
        return self.final_basis()

    def finish(self):
        self.lib.or_finish(self._h)

    def npairs(self) -> int:
        return int(self.lib.or_npairs(self._h))

    # -- inspection -----------------------------------------------------------------------
    def stats(self) -> dict:
        o = np.zeros(16, np.int64)
        self.lib.or_stats(self._h, _ptr(o, ctypes.c_int64))
        keys = ["steps", "degree", "npairs", "rows", "N", "nnz", "nA", "nC", "nb", "rank", "ng"]
        return {k: int(v) for k, v in zip(keys, o)}

    def dump(self) -> StepDump:
        st = self.stats()
        n, r, N, M = self.n, st["rows"], st["N"], st["nnz"]
        nC, nb, rank = st["nC"], st["nb"], st["rank"]
        d = np.zeros((max(N, 1), n), np.uint8)
        self.lib.or_dict(self._h, _ptr(d, ctypes.c_uint8))
        t = np.zeros((max(r, 1), n), np.uint8)
        k = np.zeros(max(r, 1), np.uint32)
        pv = np.zeros(max(r, 1), np.uint8)
        rd = np.zeros(max(r, 1), np.uint8)
        self.lib.or_rows(self._h, _ptr(t, ctypes.c_uint8), _ptr(k, ctypes.c_uint32),
                     _ptr(pv, ctypes.c_uint8), _ptr(rd, ctypes.c_uint8))
        rp = np.zeros(r + 1, np.uint32)
        col = np.zeros(max(M, 1), np.uint32)
        val = np.zeros(max(M, 1), np.uint32)
        self.lib.or_csr(self._h, _ptr(rp, ctypes.c_uint32), _ptr(col, ctypes.c_uint32),
                    _ptr(val, ctypes.c_uint32))
        npv = np.zeros(max(nb, 1), np.uint32)
        self.lib.or_nonpiv(self._h, _ptr(npv, ctypes.c_uint32))
        dp = np.zeros(max(nC * nb, 1), np.uint32)
        self.lib.or_dprime(self._h, _ptr(dp, ctypes.c_uint32))
        rpv = np.zeros(max(rank, 1), np.uint32)
        rr = np.zeros(max(rank * nb, 1), np.uint32)
        self.lib.or_rref(self._h, _ptr(rpv, ctypes.c_uint32), _ptr(rr, ctypes.c_uint32))
        ng = self.lib.or_snapshot(self._h, None)
        red = np.zeros(max(ng, 1), np.uint8)
        self.lib.or_snapshot(self._h, _ptr(red, ctypes.c_uint8))
        return StepDump(step=st["steps"], degree=st["degree"], npairs=st["npairs"],
                        dict_exps=d[:N], row_t=t[:r], row_k=k[:r], row_pivot=pv[:r],
                        row_reducer=rd[:r], row_ptr=rp, col=col[:M], val=val[:M],
                        nonpiv=npv[:nb], dprime=dp[:nC * nb].reshape(nC, nb),
                        rref_piv=rpv[:rank], rref=rr[:rank * nb].reshape(rank, nb),
                        redundant=red[:ng], nA=st["nA"], nC=nC)

    def basis_poly(self, i: int) -> list[tuple[tuple[int, ...], int]]:
        """Element i of the running basis (monic, descending terms)."""
        ln = int(self.lib.or_poly_len(self._h, i))
        e = np.zeros((max(ln, 1), self.n), np.uint8)
        c = np.zeros(max(ln, 1), np.uint32)
        self.lib.or_poly(self._h, i, _ptr(e, ctypes.c_uint8), _ptr(c, ctypes.c_uint32))
        return [(tuple(int(x) for x in e[j]), int(c[j])) for j in range(ln)]

    def basis_size(self) -> int:
        return int(self.lib.or_ng(self._h))

    def redundant(self) -> np.ndarray:
        ng = self.basis_size()
        r = np.zeros(max(ng, 1), np.uint8)
        self.lib.or_redundant(self._h, _ptr(r, ctypes.c_uint8))
        return r[:ng]

    def pairs(self) -> np.ndarray:
        q = self.npairs()
        a = np.zeros(max(2 * q, 2), np.int32)
        self.lib.or_pairs(self._h, _ptr(a, ctypes.c_int32))
        return a[:2 * q].reshape(q, 2)

    def final_arrays(self) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
        """Final reduced basis as (poly_off uint32[s+1], exps uint8[T, n], coeffs uint32[T])."""
        t = np.zeros(1, np.int64)
        s = int(self.lib.or_final_size(self._h, _ptr(t, ctypes.c_int64)))
        T = int(t[0])
        off = np.zeros(s + 1, np.uint32)
        e = np.zeros((max(T, 1), self.n), np.uint8)
        c = np.zeros(max(T, 1), np.uint32)
        self.lib.or_final(self._h, _ptr(off, ctypes.c_uint32), _ptr(e, ctypes.c_uint8),
                      _ptr(c, ctypes.c_uint32))
        return off, e[:T], c[:T]

    def final_basis(self) -> list[list[tuple[tuple[int, ...], int]]]:
        off, e, c = self.final_arrays()
        out = []
        for i in range(len(off) - 1):
            out.append([(tuple(int(x) for x in e[j]), int(c[j])) for j in range(off[i], off[i + 1])])
        return out


def reduce_row(p: int, ndict: int, npivot: int, row_ptr: np.ndarray, col: np.ndarray, val: np.ndarray,
               rcol: np.ndarray, rval: np.ndarray, nonpiv: np.ndarray) -> np.ndarray:
    """D' of one row (Sec. 9.2): the row (rcol ascending, rval) reduced by the npivot monic pivot
    rows that open the CSR matrix (row_ptr, col, val over ndict columns), read at the non-pivot
    columns nonpiv -- the same loop the oracle's step runs for each of its non-pivot rows."""
    lib = _load()
    u32 = lambda a: np.ascontiguousarray(a, dtype=np.uint32)
    row_ptr, col, val, rcol, rval, nonpiv = map(u32, (row_ptr, col, val, rcol, rval, nonpiv))
    out = np.zeros(max(len(nonpiv), 1), dtype=np.uint32)
    P = ctypes.POINTER(ctypes.c_uint32)
    lib.or_reduce_row(p, ndict, npivot, _ptr(row_ptr, ctypes.c_uint32), _ptr(col, ctypes.c_uint32),
                      _ptr(val, ctypes.c_uint32), _ptr(rcol, ctypes.c_uint32), _ptr(rval, ctypes.c_uint32),
                      len(rcol), len(nonpiv), _ptr(nonpiv, ctypes.c_uint32), _ptr(out, ctypes.c_uint32))
    return out[:len(nonpiv)]


def groebner(system: dict, flags: int = 0, lib=None):
    """Reduced Groebner basis of the system, as a list of term lists."""
    return Oracle(system, flags, lib).run()
