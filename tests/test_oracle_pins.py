"""Pins of the CPU oracle against what the paper and the mathematics fix, independently of the
oracle's own code: a library Groebner basis (sympy), Buchberger's criterion, ideal membership of
the inputs, the variety by brute force, uniqueness of the reduced basis across oracle variants,
and, per F4 step, the dictionary / matrix / closure / echelon statements of Sec. 11."""
from __future__ import annotations

import numpy as np
import pytest
from sympy import GF
from sympy.polys.matrices import DomainMatrix
from sympy.polys.orderings import grevlex

import oracle
from paper_2601_06765_b300 import synth
from tests import polyref as R


def _final_dicts(system, flags=0):
    return [R.terms_to_dict(t) for t in oracle.groebner(system, flags)]


def _small_systems():
    out = []
    for n in (2, 3, 4):
        for p in (7, 11, 65521, 2147483647):
            out.append(synth.dense_system(n, n, p, 1000 + 10 * n + p % 97))
    for seed in range(3):
        out.append(synth.sparse_system(4, 4, 65521, 77 + seed, (3, 8)))
        out.append(synth.sparse_system(3, 3, 2147483647, 91 + seed, (2, 6), degree=3))
    # sparse systems over F_7 whose pair sets exercise every condition of the pair update
    for seed in (9007, 9011, 9111, 9116):
        out.append(synth.sparse_system(3, 3, 7, seed, (2, 4)))
    out.append(synth.dense_system(3, 2, 65521, 5))          # positive-dimensional ideal
    out.append(synth.dense_system(2, 4, 65521, 6))          # overdetermined: basis {1}
    return out


# ---- final reduced basis ------------------------------------------------------------------

@pytest.mark.parametrize("system", _small_systems(), ids=lambda s: f"n{s['n']}m{s['m']}p{s['p']}")
def test_reduced_basis_matches_sympy(system):
    """sympy's groebner(..., modulus=p, order='grevlex') is an independent implementation of the
    unique reduced Groebner basis (Sec. 1 problem statement)."""
    got = oracle.groebner(system)
    want = R.sympy_reduced_gb(system)
    assert got == want


def test_reduced_basis_matches_sympy_n5():
    s = synth.dense_system(5, 5, 65521, 4242)
    assert oracle.groebner(s) == R.sympy_reduced_gb(s)


@pytest.mark.parametrize("seed", range(3))
def test_buchberger_criterion_and_membership(seed):
    """Buchberger's criterion (Sec. 2.1): every S-polynomial of the output reduces to 0; each input
    reduces to 0 modulo the output; the output is reduced and monic."""
    s = synth.dense_system(4, 4, 65521, 300 + seed) if seed < 2 else synth.dense_n6(0)
    G = _final_dicts(s)
    p = s["p"]
    assert R.is_reduced(G, p)
    assert R.is_groebner(G, p)
    for f in R.system_polys(s):
        assert not R.remainder(f, G, p)


@pytest.mark.parametrize("n,p", [(2, 7), (3, 7), (3, 11), (4, 7), (3, 13)])
def test_variety_bruteforce(n, p):
    """The F_p-rational zeros of the output equal those of the input (brute force over F_p^n)."""
    for seed in range(3):
        s = synth.sparse_system(n, n, p, 500 + seed, (2, 5))
        F = R.system_polys(s)
        G = _final_dicts(s)
        assert R.zeros(G, n, p) == R.zeros(F, n, p)


@pytest.mark.parametrize("seed", range(6))
def test_variants_give_the_same_reduced_basis(seed):
    """The reduced basis is unique: one pair per step (Buchberger-like selection) and the newest
    instead of the oldest reducer change every intermediate matrix but not the result."""
    s = synth.dense_n6(seed) if seed < 3 else synth.sparse_system(5, 5, 2147483647, seed, (6, 12), 3)
    a = oracle.groebner(s)
    assert oracle.groebner(s, oracle.ONE_PAIR) == a
    assert oracle.groebner(s, oracle.NEWEST_REDUCER) == a
    assert oracle.groebner(s, oracle.ONE_PAIR | oracle.NEWEST_REDUCER) == a


def test_degenerate_inputs():
    """Zero polynomials are dropped; a constant gives the unit ideal; no input gives no basis."""
    p = 65521
    one = {"n": 2, "p": p, "m": 2, "poly_off": [0, 2, 3],
           "exps": [[1, 0], [0, 1], [0, 0]], "coeffs": [3, 4, 5]}
    assert oracle.groebner(synth._pack(2, p, [[((1, 0), 3), ((0, 1), 4)], [((0, 0), 5)]])) == [[((0, 0), 1)]]
    del one
    zero = synth._pack(3, p, [[((1, 0, 0), 7), ((1, 0, 0), p - 7)], [((0, 1, 1), 0)]])
    assert oracle.groebner(zero) == []
    # duplicate monomials merge mod p and the leading coefficient is normalised
    s = synth._pack(2, 11, [[((0, 1), 3), ((1, 0), 2), ((0, 1), 5), ((1, 0), 4)]])
    assert oracle.groebner(s) == [[((1, 0), 1), ((0, 1), (8 * pow(6, 9, 11)) % 11)]]


# ---- per-step matrix statements of Sec. 11 ------------------------------------------------

def _steps(system, flags=0, limit=100, lib=None):
    o = oracle.Oracle(system, flags, lib)
    out = []
    while len(out) < limit:
        basis = [R.terms_to_dict(o.basis_poly(i)) for i in range(o.basis_size())]
        if not o.step():
            break
        out.append((basis, o.dump()))
    return out


def _row_poly(basis, t, k):
    g = basis[int(k)]
    return {R.mono_mul(tuple(int(x) for x in t), e): c for e, c in g.items()}


STEP_SYSTEMS = [synth.dense_n6(0), synth.dense_system(4, 4, 2147483647, 31),
                synth.sparse_system(4, 4, 65521, 808, (5, 12), degree=3)]


@pytest.mark.parametrize("system", STEP_SYSTEMS, ids=["c1", "n4p31", "n4cubic"])
def test_dictionary_matrix_and_closure(system):
    check_dictionary_matrix_closure(system)


def check_dictionary_matrix_closure(system, lib=None, limit=100):
    """the dictionary-correctness theorem of Sec. 11: T is exactly the union of the row supports, in descending order (sympy's grevlex
    key).  the matrix-materialisation theorem of Sec. 11: row i of the CSR is t_i * g_{k_i}, nnz = M = sum |supp g_k|.  the race-freedom theorem of Sec. 11: the
    row segments partition [0, M).  the support-closure definition of Sec. 11 / Rem. 3.3: every dictionary monomial divisible by a
    non-redundant leading monomial is the leading monomial of a row, and reducer rows use the
    oldest such element."""
    for basis, d in _steps(system, limit=limit, lib=lib):
        n = system["n"]
        dict_monos = [tuple(int(x) for x in row) for row in d.dict_exps]
        union = set()
        rows = []
        for t, k in zip(d.row_t, d.row_k):
            f = _row_poly(basis, t, k)
            rows.append(f)
            union |= set(f)
        assert set(dict_monos) == union and len(dict_monos) == len(union)
        assert dict_monos == sorted(union, key=grevlex, reverse=True)
        col_of = {m: i for i, m in enumerate(dict_monos)}
        assert d.row_ptr[0] == 0 and int(d.row_ptr[-1]) == d.nnz
        assert d.nnz == sum(len(basis[int(k)]) for k in d.row_k)
        for i, f in enumerate(rows):
            a, b = int(d.row_ptr[i]), int(d.row_ptr[i + 1])
            assert b - a == len(f)
            cols = [int(c) for c in d.col[a:b]]
            assert cols == sorted(cols) and len(set(cols)) == len(cols)
            assert {dict_monos[c]: int(v) for c, v in zip(cols, d.val[a:b])} == f
        lms = [R.lm(f) for f in rows]
        nonred = [i for i, r in enumerate(d.redundant) if not r]
        lm_set = set(lms)
        for m in dict_monos:
            divs = [i for i in nonred if R.divides(R.lm(basis[i]), m)]
            if divs:
                assert m in lm_set
        for f, lmf, red, k in zip(rows, lms, d.row_reducer, d.row_k):
            if red:
                assert int(k) == min(i for i in nonred if R.divides(R.lm(basis[i]), lmf))
        # row order: pivots first by leading column, then non-pivot rows by (column, k)
        piv = [bool(x) for x in d.row_pivot]
        assert piv == sorted(piv, reverse=True)
        keyed = [(col_of[l], int(k)) for l, k in zip(lms, d.row_k)]
        npiv = sum(piv)
        assert keyed[:npiv] == sorted(keyed[:npiv]) and len({c for c, _ in keyed[:npiv]}) == npiv
        assert keyed[npiv:] == sorted(keyed[npiv:])
        pivcols = {c for c, _ in keyed[:npiv]}
        assert all(c in pivcols for c, _ in keyed[npiv:])
        # a pair-row leading column without a reducer row takes the pair row of smallest k
        for (c, k), red, pv in zip(keyed, d.row_reducer, piv):
            if not red and pv:
                assert all(k2 > k for (c2, k2), r2 in zip(keyed, d.row_reducer) if c2 == c and not r2
                           and (c2, k2) != (c, k))
        assert [c for c in range(len(dict_monos)) if c not in pivcols] == [int(c) for c in d.nonpiv]
        del n


def _dm(rows, ncols, p):
    K = GF(p)
    return DomainMatrix([[K(int(x)) for x in r] for r in rows], (len(rows), ncols), K)


def _ints(M, p):
    return [[int(x) % p for x in row] for row in M.to_Matrix().tolist()]


@pytest.mark.parametrize("system", [synth.dense_system(4, 4, 65521, 17),
                                    synth.dense_system(3, 3, 2147483647, 18),
                                    synth.sparse_system(4, 4, 65521, 19, (4, 9), degree=3)],
                         ids=["n4", "n3p31", "n4cubic"])
def test_reduction_and_echelon_against_library_rref(system):
    check_reduction_and_echelon(system)


def check_reduction_and_echelon(system, lib=None, limit=6):
    """Sec. 9.2 / the row-operations theorem of Sec. 11: D' spans, with the pivot rows, the row space of A and vanishes on the
    pivot columns (so it is the unique such reduction), and RREF(D') equals the rows of the full
    reduced echelon form of A whose leading column is a non-pivot column (sympy DomainMatrix over
    GF(p) as the library reference)."""
    p = system["p"]
    for basis, d in _steps(system, limit=limit, lib=lib):
        N = d.N
        if N > 160 or len(d.row_k) > 160:
            continue
        A = [[0] * N for _ in range(len(d.row_k))]
        for i in range(len(d.row_k)):
            for q in range(int(d.row_ptr[i]), int(d.row_ptr[i + 1])):
                A[i][int(d.col[q])] = int(d.val[q])
        nA = d.nA
        nonpiv = [int(c) for c in d.nonpiv]
        # D' padded to full width
        Dp = []
        for row in d.dprime.tolist():
            full = [0] * N
            for j, c in enumerate(nonpiv):
                full[c] = int(row[j])
            Dp.append(full)
        full_rank = _dm(A, N, p).rank() if A else 0
        assert _dm(A[:nA] + Dp, N, p).rank() == full_rank
        for r, orig in zip(Dp, A[nA:]):
            diff = [(a - b) % p for a, b in zip(r, orig)]
            assert _dm(A[:nA] + [diff], N, p).rank() == _dm(A[:nA], N, p).rank()
        Rm, pivots = _dm(A, N, p).rref()
        Rl = _ints(Rm, p)
        want = [[row[c] for c in nonpiv] for row, pc in zip(Rl, pivots) if pc in set(nonpiv)]
        assert d.rref.tolist() == want
        assert [nonpiv[int(j)] for j in d.rref_piv] == [pc for pc in pivots if pc in set(nonpiv)]


@pytest.mark.parametrize("system", [synth.dense_system(4, 4, 65521, 17),
                                    synth.dense_system(3, 3, 2147483647, 18),
                                    synth.sparse_system(5, 5, 65521, 19, (4, 12))],
                         ids=["n4", "n3p31", "n5sparse"])
def test_single_row_reduction_reproduces_dprime(system):
    """oracle.reduce_row (one non-pivot row reduced alone by the pivot rows, Sec. 9.2) gives the
    rows of D' that the step computes and the test above pins against the library RREF; the
    full-size GPU checks of D' rely on it."""
    for _, d in _steps(system, limit=6):
        for i in range(d.dprime.shape[0]):
            a = d.nA + i
            s, e = int(d.row_ptr[a]), int(d.row_ptr[a + 1])
            got = oracle.reduce_row(system["p"], d.N, d.nA, d.row_ptr, d.col, d.val, d.col[s:e], d.val[s:e], d.nonpiv)
            assert np.array_equal(got, d.dprime[i])


def test_kernel_vectors_are_syzygies():
    """Prop. 3.2: with a support-closed dictionary, v^T A = 0 iff sum v_i t_i g_{k_i} = 0; the
    left nullspace of A (sympy over GF(p)) gives polynomial identities among the shifted rows."""
    system = synth.dense_system(3, 3, 65521, 23)
    p = system["p"]
    checked = 0
    for basis, d in _steps(system, limit=4):
        N = d.N
        r = len(d.row_k)
        if r > 80 or N > 120:
            continue
        A = [[0] * N for _ in range(r)]
        for i in range(r):
            for q in range(int(d.row_ptr[i]), int(d.row_ptr[i + 1])):
                A[i][int(d.col[q])] = int(d.val[q])
        ns = _dm(A, N, p).transpose().nullspace()
        for v in _ints(ns, p):
            acc: dict = {}
            for i in range(r):
                if v[i]:
                    acc = R.axpy(acc, v[i], tuple(int(x) for x in d.row_t[i]), basis[int(d.row_k[i])], p)
            assert acc == {}
            checked += 1
    assert checked > 0  # this system's later steps have rank-deficient pair rows


# ---- pair selection, the Gebauer-Moeller update and the pair rows --------------------------

def check_pairs_replay(system, lib=None, limit=100):
    """The oracle's critical pairs against the textbook model of tests/polyref.py
    (Becker-Weispfenning's UPDATE, normal selection), fed only the leading monomials of the
    oracle's basis elements in insertion order.  Before every step the two pair sets and the
    set of elements still in G agree; the step's degree is the least lcm degree of that pair set
    and exactly the pairs of that degree leave it; the step's pair rows (those the closure did not
    add) are exactly the rows (lcm/LM(g_i), i), (lcm/LM(g_j), j) of the chosen pairs, each once;
    and no two rows of a step share (t, k)."""
    o = oracle.Oracle(system, 0, lib)
    model = R.PairModel()

    def lm_of(i):
        return R.lm(R.terms_to_dict(o.basis_poly(i)))

    def agree():
        got = {(int(a), int(b)) for a, b in o.pairs()}
        assert len(got) == o.npairs(), "the oracle holds a pair twice"
        assert got == model.B
        assert [not bool(x) for x in o.redundant()] == model.in_g

    for i in range(o.basis_size()):
        model.insert(lm_of(i))
    agree()
    steps = 0
    while steps < limit and model.B:
        ng = o.basis_size()
        degree, chosen = model.select()
        assert o.step()
        d = o.dump()
        assert d.degree == degree
        pair_rows = [(tuple(int(x) for x in t), int(k))
                     for t, k, red in zip(d.row_t, d.row_k, d.row_reducer) if not red]
        assert len(pair_rows) == len(set(pair_rows)), "equal pair rows were not collapsed"
        assert set(pair_rows) == model.pair_rows(chosen)
        all_rows = [(bytes(t), int(k)) for t, k in zip(d.row_t, d.row_k)]
        assert len(all_rows) == len(set(all_rows))
        for i in range(ng, o.basis_size()):
            model.insert(lm_of(i))
        agree()
        steps += 1
    if steps < limit:
        assert not o.step()
    return steps


def _coprime_shadow_system():
    """Leading monomials x2, x1*x2, x1 (grevlex) in that input order: when x1 arrives, its pair
    with x2 is coprime and has the same lcm x1*x2 as its pair with x1*x2, so UPDATE's first loop
    must keep the coprime pair long enough to shadow the other (Becker-Weispfenning), and the
    product criterion then drops it: no pair of the third input survives."""
    return synth._pack(3, 7, [[((0, 1, 0), 1), ((0, 0, 1), 3), ((0, 0, 0), 2)],
                              [((1, 1, 0), 1), ((0, 0, 2), 5), ((1, 0, 0), 4), ((0, 0, 0), 1)],
                              [((1, 0, 0), 1), ((0, 0, 1), 6), ((0, 0, 0), 3)],
                              [((0, 0, 2), 1), ((0, 1, 0), 2), ((0, 0, 1), 1)]])


PAIR_SYSTEMS = [_coprime_shadow_system(), synth.dense_n6(0), synth.dense_n6(1), synth.dense_system(4, 4, 7, 41),
                synth.dense_system(5, 5, 65521, 4242),
                synth.sparse_system(4, 4, 65521, 808, (5, 12), degree=3),
                synth.sparse_system(5, 5, 2147483647, 3, (6, 12), degree=3),
                synth.dense_system(3, 2, 65521, 5)] + \
    [synth.sparse_system(3, 3, 7, seed, (2, 4)) for seed in (9007, 9011, 9111, 9116)]


@pytest.mark.parametrize("system", PAIR_SYSTEMS, ids=lambda s: f"n{s['n']}m{s['m']}p{s['p']}")
def test_pairs_follow_the_textbook_update_and_normal_selection(system):
    assert check_pairs_replay(system) > 0
