"""Pins of the signature-filtered (F5 criterion) oracle against what the mathematics fixes.

- The Hilbert series of a regular sequence: the degree-d part of <f_1 .. f_i> has dimension
  C(n-1+d, n-1) minus the coefficient of t^d in prod_{j<=i} (1 - t^{d_j}) / (1 - t)^n.  The rank
  of every block's matrix must be that number (the criterion must not lose rows the ideal needs).
- Faugere's theorem for F5 on regular sequences: with the criterion no admissible row reduces to
  zero, i.e. every block's rank grows by its number of admissible rows.
- Soundness (the signature-sound compilation theorem): the criterion keeps the row space, so the
  leading-monomial sets equal those of the unfiltered matrices, which do reduce rows to zero.
- The reduced Groebner basis equals sympy's (a library routine) once dmax reaches its degree.
- Brute force on tiny systems: every filtered row lies in the span of the admissible rows of
  smaller signature.
- A non-regular sequence (f_2 a multiple of f_1) keeps all of the above except the zero count.
- Planted mistakes in the criterion or in the new-element rule fail one of the pins.
"""
from __future__ import annotations

from math import comb

import numpy as np
import pytest

from oracle import f5 as O
from paper_2601_06765_b300 import synth
from tests import polyref

P = 65521


def hilbert_ideal_dims(n: int, degrees: list[int], dmax: int) -> list[int]:
    """Closed form: dim of the degree-d part of an ideal generated by a regular sequence."""
    num = [1] + [0] * dmax
    for dj in degrees:
        nxt = num[:]
        for k in range(dj, dmax + 1):
            nxt[k] -= num[k - dj]
        num = nxt
    series = [comb(n - 1 + k, n - 1) for k in range(dmax + 1)]
    quotient = [sum(num[a] * series[d - a] for a in range(d + 1)) for d in range(dmax + 1)]
    return [series[d] - quotient[d] for d in range(dmax + 1)]


def _degrees(system):
    return [sum(next(iter(f))) for f in O.normalised_inputs(system)]


REGULAR = [
    ("hq_n3_m3", synth.homogeneous_system(3, 3, P, 11), 5),
    ("hq_n4_m3", synth.homogeneous_system(4, 3, P, 12), 6),
    ("hq_n4_m4", synth.homogeneous_system(4, 4, P, 13), 5),
    ("h23_n4_m3", synth.homogeneous_system(4, 3, P, 14, degree=[2, 3, 2]), 6),
    ("homogenised_dense_n3", synth.homogenize(synth.dense_system(3, 3, P, 15)), 5),
]


@pytest.fixture(scope="module")
def runs():
    return {name: (s, D, O.f5(s, D), O.f5(s, D, criterion=False)) for name, s, D in REGULAR}


@pytest.mark.parametrize("name", [r[0] for r in REGULAR])
def test_block_ranks_follow_the_hilbert_series(runs, name):
    s, D, got, _ = runs[name]
    degs = _degrees(s)
    for b in got["blocks"]:
        i, d = b["index"], b["degree"]
        assert len(got["L"][(i, d)]) == hilbert_ideal_dims(int(s["n"]), degs[:i], D)[d], (i, d)


@pytest.mark.parametrize("name", [r[0] for r in REGULAR])
def test_no_admissible_row_reduces_to_zero(runs, name):
    _, _, got, _ = runs[name]
    assert all(b["zero_reductions"] == 0 for b in got["blocks"])
    assert sum(b["candidates"] - b["admissible"] for b in got["blocks"]) > 0  # the criterion acts


@pytest.mark.parametrize("name", [r[0] for r in REGULAR])
def test_the_criterion_keeps_the_row_space(runs, name):
    _, _, got, plain = runs[name]
    assert got["L"] == plain["L"]
    assert sum(b["zero_reductions"] for b in plain["blocks"]) == \
        sum(b["candidates"] - b["admissible"] for b in got["blocks"])
    assert got["basis"] == plain["basis"]


@pytest.mark.parametrize("name", ["hq_n3_m3", "hq_n4_m4", "h23_n4_m3", "homogenised_dense_n3"])
def test_reduced_basis_equals_sympy(name):
    s = next(r[1] for r in REGULAR if r[0] == name)
    want = polyref.sympy_reduced_gb(s)
    D = max(sum(g[0][0]) for g in want)
    got = O.f5(s, D)["basis"]
    assert [[(tuple(e), c) for e, c in g] for g in got] == want


def _rank(rows, p):
    return len(O.rref(np.array(rows, dtype=np.int64), p)[1]) if len(rows) else 0


def test_filtered_rows_lie_in_the_span_of_smaller_signatures():
    s = synth.homogeneous_system(3, 3, P, 21)
    F = O.normalised_inputs(s)
    degs = _degrees(s)
    got = O.f5(s, 5)
    checked = 0
    for d in range(2, 6):
        cols = O.monomials_of_degree(3, d)
        col_of = {m: c for c, m in enumerate(cols)}
        adm_rows = []  # (index, candidate position, row) of the admissible rows at degree d
        for b in (b for b in got["blocks"] if b["degree"] == d):
            i = b["index"]
            cand = O.monomials_of_degree(3, d - degs[i - 1])
            kept = {k & 0xFFFFFFFF for k in b["keys"]}
            for j in kept:
                adm_rows.append((i, j, O.row_of(F[i - 1], cand[j], col_of, len(cols))))
            for j in range(len(cand)):
                if j in kept:
                    continue
                smaller = [r for (ii, jj, r) in adm_rows if ii < i or (ii == i and jj > j)]
                row = O.row_of(F[i - 1], cand[j], col_of, len(cols))
                assert _rank(smaller + [row], P) == _rank(smaller, P), (d, i, j)
                checked += 1
    assert checked > 0


def test_non_regular_sequence():
    """f_2 = x1 f_1 and f_3 random: the admissible row f_2 reduces to zero; everything else holds."""
    s = synth.homogeneous_system(3, 2, P, 31)
    f1 = O.normalised_inputs(s)[0]
    polys = [[(e, c) for e, c in f1.items()], [((e[0] + 1,) + e[1:], c) for e, c in f1.items()],
             list(zip(*[[tuple(int(x) for x in s["exps"][q]) for q in range(int(s["poly_off"][1]), int(s["poly_off"][2]))],
                        [int(c) for c in s["coeffs"][int(s["poly_off"][1]):int(s["poly_off"][2])]]]))]
    sys3 = synth._pack(3, P, polys)
    want = polyref.sympy_reduced_gb(sys3)
    D = max(sum(g[0][0]) for g in want)
    got, plain = O.f5(sys3, D), O.f5(sys3, D, criterion=False)
    assert sum(b["zero_reductions"] for b in got["blocks"]) >= 1
    assert got["L"] == plain["L"]
    assert [[(tuple(e), c) for e, c in g] for g in got["basis"]] == want


def _monic(f: dict, p: int) -> dict:
    inv = pow(f[polyref.lm(f)], p - 2, p)
    return {e: c * inv % p for e, c in f.items()}


def _reduce_at(f: dict, piv: dict, p: int) -> dict:
    """f with every monomial that is a pivot's leading monomial eliminated, largest first."""
    from sympy.polys.orderings import grevlex
    f = dict(f)
    while True:
        hit = [e for e in f if e in piv]
        if not hit:
            return f
        m = max(hit, key=grevlex)
        f = polyref.axpy(f, (p - f[m]) % p, (0,) * len(m), piv[m], p)


def _echelon(rows: list, p: int) -> list:
    """The reduced echelon basis of the span of the rows (dict polynomials), by leading monomial
    descending."""
    from sympy.polys.orderings import grevlex
    done: list = []
    rows = [r for r in rows if r]
    while rows:
        r = max(rows, key=lambda f: grevlex(polyref.lm(f)))
        rows.remove(r)
        r = _monic(r, p)
        t = polyref.lm(r)
        rows = [x for x in (polyref.axpy(x, (p - x.get(t, 0)) % p, (0,) * len(t), r, p) if t in x else x
                            for x in rows) if x]
        done = [polyref.axpy(x, (p - x.get(t, 0)) % p, (0,) * len(t), r, p) if t in x else x for x in done]
        done.append(r)
    return sorted(done, key=lambda f: grevlex(polyref.lm(f)), reverse=True)


def _new_elements_by_reduction(s, D, got) -> list:
    """Every block's new elements recomputed as an F4 step would: the block's rows are a basis of
    the previous blocks' span at this degree (distinct leading monomials) and the admissible
    candidates; the first row of each leading monomial is a pivot; the other rows are reduced at
    the pivots' leading monomials, and the remainders brought to reduced echelon form."""
    p, n = int(s["p"]), int(s["n"])
    F = [_monic(f, p) for f in polyref.system_polys(s) if f]
    degs = [sum(next(iter(f))) for f in F]
    out = []
    for d in sorted({b["degree"] for b in got["blocks"]}):
        E: list = []  # dict polynomials with distinct leading monomials spanning the previous blocks
        for b in (b for b in got["blocks"] if b["degree"] == d):
            i = b["index"]
            cand = O.monomials_of_degree(n, d - degs[i - 1])
            rows = list(E) + [{polyref.mono_mul(cand[k & 0xFFFFFFFF], e): c for e, c in F[i - 1].items()}
                              for k in b["keys"]]
            piv: dict = {}
            rest = []
            for r in rows:
                t = polyref.lm(r)
                if t in piv:
                    rest.append(r)
                else:
                    piv[t] = _monic(r, p)
            new = _echelon([_reduce_at(r, piv, p) for r in rest], p)
            out.extend(sorted(((e, c) for e, c in g.items()), key=lambda x: O.grevlex_key(x[0]), reverse=True)
                       for g in new)
            E = list(piv.values()) + new
    return out


def test_new_elements_equal_the_reduced_non_pivot_rows():
    for name in ("hq_n3_m3", "h23_n4_m3"):
        s, D = next((r[1], r[2]) for r in REGULAR if r[0] == name)
        got = O.f5(s, D)
        assert _new_elements_by_reduction(s, D, got) == [[(tuple(e), c) for e, c in g] for g in got["elements"]]


def _pins_pass(monkeypatch_target=None) -> bool:
    try:
        s, D = REGULAR[1][1], REGULAR[1][2]
        got, plain = O.f5(s, D), O.f5(s, D, criterion=False)
        degs = _degrees(s)
        for b in got["blocks"]:
            i, d = b["index"], b["degree"]
            if len(got["L"][(i, d)]) != hilbert_ideal_dims(int(s["n"]), degs[:i], D)[d]:
                return False
            if b["zero_reductions"] != 0:
                return False
        if got["L"] != plain["L"] or got["basis"] != plain["basis"]:
            return False
        if sum(b["new"] for b in got["blocks"]) != len(got["elements"]):
            return False
        return _new_elements_by_reduction(s, D, got) == [[(tuple(e), c) for e, c in g] for g in got["elements"]]
    except Exception:  # noqa: BLE001 -- a crash is a caught mutant too
        return False


def test_pins_pass_on_the_oracle():
    assert _pins_pass()


MUTANTS = {
    # the criterion read at the block's own index: removes rows the ideal needs
    "criterion_own_index": ("forbidden_set", lambda L, i, e: L.get((i, e), set())),
    # the criterion read one degree too high
    "criterion_degree_plus_one": ("forbidden_set", lambda L, i, e: L.get((i - 1, e + 1), set())),
    # the criterion two generators back: sound but weaker, so rows reduce to zero
    "criterion_two_back": ("forbidden_set", lambda L, i, e: L.get((i - 2, e), set())),
    # the criterion one degree too low
    "criterion_degree_minus_one": ("forbidden_set", lambda L, i, e: L.get((i - 1, e - 1), set())),
    # new elements: the candidates' own leading monomials not counted as the block's
    "new_includes_candidate_leads": ("block_leading_monomials", lambda prev, cand, adm, lead_f: set(prev)),
    # new elements: the earlier echelon rows' leading monomials not counted
    "new_includes_old_leads": ("block_leading_monomials",
                               lambda prev, cand, adm, lead_f: {O.mono_mul(cand[j], lead_f) for j in adm}),
}


@pytest.mark.parametrize("name", list(MUTANTS))
def test_planted_mistakes_are_caught(monkeypatch, name):
    attr, fn = MUTANTS[name]
    monkeypatch.setattr(O, attr, fn)
    assert not _pins_pass(), name
