"""Pins of the block Wiedemann oracle (oracle/wiedemann.py) against what the mathematics fixes,
independently of its own code: sympy's matrices over GF(p) (library routines) for the Krylov
sequence, the Hankel echelon form and the left nullspace of A; and Prop. 3.2 -- every vector
found is a polynomial identity among the step's shifted rows (plain-Python polynomial arithmetic
of tests/polyref.py)."""
from __future__ import annotations

import numpy as np
import pytest
from sympy import GF
from sympy.polys.matrices import DomainMatrix

import oracle
from oracle import wiedemann as W
from paper_2601_06765_b300 import synth
from tests import polyref as R


def _dm(rows, p):
    K = GF(p)
    rows = [[K(int(x)) for x in r] for r in rows]
    return DomainMatrix(rows, (len(rows), len(rows[0]) if rows else 0), K)


def _ints(M, p):
    return [[int(x) % p for x in row] for row in M.to_Matrix().tolist()]


def step_matrix(system, step):
    """(basis before the step, the step's dump) of the oracle."""
    o = oracle.Oracle(system)
    for _ in range(step - 1):
        assert o.step()
    basis = [R.terms_to_dict(o.basis_poly(i)) for i in range(o.basis_size())]
    assert o.step()
    return basis, o.dump()


def random_inputs(r, N, b, p, seed):
    rng = np.random.default_rng(seed)
    X = rng.integers(0, p, size=(r, b)).tolist()
    Z = rng.integers(0, p, size=(r, b)).tolist()
    delta = rng.integers(1, p, size=N).tolist()
    return X, Z, delta


# steps whose Macaulay matrix has dependent rows (zero reductions: nC > rank D')
CASES = [("n4_p65521_step3", synth.dense_system(4, 4, 65521, 17), 3),
         ("n3_p31_step3", synth.dense_system(3, 3, 2147483647, 18), 3),
         ("n6_step3", synth.dense_n6(0), 3)]


def _nullity(d):
    return d.nC - d.rref.shape[0]


@pytest.mark.parametrize("name,system,step", CASES, ids=[c[0] for c in CASES])
def test_cases_have_dependent_rows(name, system, step):
    _, d = step_matrix(system, step)
    assert _nullity(d) >= 1


@pytest.mark.parametrize("name,system,step", CASES[:2], ids=[c[0] for c in CASES[:2]])
def test_sequence_and_hankel_echelon_against_sympy(name, system, step):
    _, d = step_matrix(system, step)
    p = system["p"]
    r, N = len(d.row_k), d.N
    X, Z, delta = random_inputs(r, N, 4, p, 1)
    out = W.block_wiedemann(d.row_ptr, d.col, d.val, N, p, X, Z, delta)
    A = _dm(W.dense_matrix(d.row_ptr, d.col, d.val, N).tolist(), p)
    Dg = DomainMatrix.diag([GF(p)(int(x)) for x in delta], GF(p), (N, N))
    M = A * Dg * A.transpose()
    Xd, Zd = _dm(X, p), _dm(Z, p)
    for i in (0, 1, len(out["seq"]) - 1):
        want = _ints(Xd.transpose() * M ** (i + 1) * Zd, p)
        assert [[int(x) for x in row] for row in out["seq"][i]] == want
    Hd = _dm(W.hankel(out["seq"], out["d"], 4).tolist(), p)
    Rs, piv = Hd.rref()
    Rl = [row for row in _ints(Rs, p) if any(row)]
    assert [[int(x) for x in row] for row in out["H_rref"]] == Rl
    assert list(out["H_piv"]) == list(piv)


@pytest.mark.parametrize("b", [2, 4, 8])
@pytest.mark.parametrize("name,system,step", CASES, ids=[c[0] for c in CASES])
def test_found_vectors_are_syzygies(name, system, step, b):
    """Prop. 3.2: each row w of W gives sum_i w_i t_i g_{k_i} = 0 as a polynomial; W is in
    reduced echelon form; it spans at most the left nullspace of A, and all of it when b is at
    least its dimension (then W is the RREF basis of sympy's left nullspace)."""
    basis, d = step_matrix(system, step)
    p = system["p"]
    r, N = len(d.row_k), d.N
    X, Z, delta = random_inputs(r, N, b, p, 7 + b)
    out = W.block_wiedemann(d.row_ptr, d.col, d.val, N, p, X, Z, delta)
    Wm = out["W"]
    nul = _nullity(d)
    assert Wm.shape[0] == min(b, nul)  # with random blocks: the projection of Z onto ker A^T
    for w in Wm:
        acc: dict = {}
        for i in range(r):
            if w[i]:
                acc = R.axpy(acc, int(w[i]), tuple(int(x) for x in d.row_t[i]), basis[int(d.row_k[i])], p)
        assert acc == {}
    Wd = _dm(Wm.tolist(), p)
    Rw, _ = Wd.rref()
    assert _ints(Rw, p)[:Wm.shape[0]] == [[int(x) for x in row] for row in Wm]
    if b >= nul:
        A = _dm(W.dense_matrix(d.row_ptr, d.col, d.val, N).tolist(), p)
        ns = A.transpose().nullspace()
        Rn, _ = ns.rref()
        assert [[int(x) for x in row] for row in Wm] == [row for row in _ints(Rn, p) if any(row)]


def test_full_row_rank_gives_no_vectors():
    """With independent rows (ker A^T = 0) the symmetric operator is invertible and every y(c)
    vanishes: W is empty."""
    system = synth.dense_system(4, 4, 65521, 17)
    o = oracle.Oracle(system)
    assert o.step()
    d = o.dump()
    assert d.nC == d.rref.shape[0]  # the first step has no zero reduction
    r, N, p = len(d.row_k), d.N, system["p"]
    X, Z, delta = random_inputs(r, N, 4, p, 3)
    out = W.block_wiedemann(d.row_ptr, d.col, d.val, N, p, X, Z, delta)
    assert out["W"].shape[0] == 0
