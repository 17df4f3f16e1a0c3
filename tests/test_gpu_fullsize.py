"""Full-size checks of the n=13 sparse 31-bit workload (the large-matrix configuration), in the
launch configuration bench.py times, where the oracle cannot run the whole system.

- D' of a large step: each row of D' is the unique reduction of its non-pivot row by the monic
  pivot rows (Sec. 9.2), so the oracle computes sampled rows one at a time (oracle.reduce_row) from
  the step's own matrix; the matrix itself is the GPU's, checked bit-exact against the oracle for the
  first steps in test_gpu_parity.py.  Step 6 has more than 14000 pivots and 3000 non-pivot rows and
  takes the dense tensor-core reduction.
- RREF(D') of that step: identity on its pivot columns, zero left of each pivot, and every sampled row
  of D' is a combination of its rows.
- The reduced basis of the whole run (thousands of polynomials, millions of terms): monic, sorted by leading
  monomial descending (grevlex), minimal, and reduced on sampled terms (no term divisible by a
  leading monomial).  These hold for the reduced Groebner basis at any size."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2601_06765_b300 as gb
from paper_2601_06765_b300 import synth

pytestmark = pytest.mark.gpu

P31 = 2147483647


@pytest.fixture(scope="module")
def ctx():
    c = gb.Context(arena_bytes=48 << 30, keep_step=True)
    yield c
    c.close()


def test_sparse_n13_large_step_dprime_rows_and_rref(ctx):
    with gb.System(ctx, synth.sparse_n13(0)) as S:
        for _ in range(6):
            assert S.step()[0] == gb.GB_OK
        mac, ech = S.last_step()
    rp, col, val, nA = mac["row_ptr"], mac["col"], mac["val"], int(mac["npivot"])
    N = mac["dict_exps"].shape[0]
    nonpiv, D = ech["nonpiv"], ech["dprime"]
    # a large step: well past the oracle's reach, and on the dense path's shape rule for 31-bit primes
    assert nA >= 4096 and D.shape[0] >= 1024 and D.shape == (len(rp) - 1 - nA, len(nonpiv))
    rng = np.random.default_rng(6)
    sample = rng.choice(D.shape[0], 4, replace=False)
    for i in sample:
        a = nA + int(i)
        s, e = int(rp[a]), int(rp[a + 1])
        want = oracle.reduce_row(P31, N, nA, rp, col, val, col[s:e], val[s:e], nonpiv)
        assert np.array_equal(D[i], want), f"row {i} of D'"
    R = ech["rref"].astype(np.int64)
    piv = ech["rref_piv"].astype(np.int64)
    rank = len(piv)
    assert rank == R.shape[0] and 0 < rank <= min(D.shape)
    assert np.all(np.diff(piv) > 0)
    assert np.array_equal(R[:, piv], np.eye(rank, dtype=np.int64))
    for k in range(rank):
        assert not R[k, :piv[k]].any()
    for i in sample:
        res = D[i].astype(np.int64)
        coef = res[piv].copy()
        for k in range(rank):
            if coef[k]:
                res = (res - coef[k] * R[k]) % P31
        assert not res.any(), f"row {i} of D' outside the row space of RREF(D')"
    # every row at once: D = D[:, piv] R, tested on random vectors mod p.  With R in RREF, a row of D
    # equals its pivot-column entries times R exactly when it lies in the row space of R.
    Dl = D.astype(np.int64)
    for _ in range(3):
        x = rng.integers(0, P31, size=D.shape[1], dtype=np.int64)
        lhs = _matvec(Dl, x)
        rhs = _matvec(Dl[:, piv], _matvec(R, x))
        assert np.array_equal(lhs, rhs), "a row of D' outside the row space of RREF(D')"


def _matvec(M: np.ndarray, x: np.ndarray) -> np.ndarray:
    """(M x) mod p exactly in int64: x = x0 + 2^16 x1 with 16-bit halves, so every product is below
    2^47 and every row sum (at most 2^13 terms here) below 2^61."""
    assert M.shape[1] < (1 << 13)
    x0, x1 = x & 0xFFFF, x >> 16
    return ((M @ x0) % P31 + ((M @ x1) % P31) * 65536) % P31


def _grevlex_key(e: np.ndarray):
    # x^a > x^b: higher degree, then the last differing exponent smaller
    return (int(e.sum()),) + tuple(-int(x) for x in e[::-1])


def test_sparse_n13_reduced_basis_properties(ctx):
    h = gb.gb_system_create(ctx.h, synth.sparse_n13(0))
    gb.gb_groebner(h)
    off, ex, cf = gb.gb_basis_export(h, 13, True)
    gb.gb_system_destroy(h)
    ng = len(off) - 1
    assert ng > 0 and len(cf) == int(off[-1]) and ex.size == 13 * len(cf)
    ex = ex.reshape(-1, 13).astype(np.int16)
    lead = off[:-1].astype(np.int64)
    assert np.all(cf[lead] == 1), "monic"
    LM = ex[lead]
    keys = [_grevlex_key(m) for m in LM]
    assert all(keys[i] > keys[i + 1] for i in range(ng - 1)), "leading monomials descending"
    # minimal: no leading monomial divides another
    for c0 in range(0, ng, 256):
        blk = LM[c0:c0 + 256]
        div = (LM[None, :, :] <= blk[:, None, :]).all(axis=2)  # div[i, g]: LM[g] | blk[i]
        assert np.array_equal(div.sum(axis=1), np.ones(len(blk), dtype=np.int64)), "minimal"
    # reduced, on sampled non-leading terms
    is_lead = np.zeros(len(cf), dtype=bool)
    is_lead[lead] = True
    rng = np.random.default_rng(13)
    terms = rng.choice(np.flatnonzero(~is_lead), 20000, replace=False)
    for t0 in range(0, len(terms), 500):
        T = ex[terms[t0:t0 + 500]]
        hit = (LM[None, :, :] <= T[:, None, :]).all(axis=2).any(axis=1)
        assert not hit.any(), "a tail term is divisible by a leading monomial"
