"""Pins of the oracle's deglex order (the other graded order of Sec. 7.3: degree first, ties broken
lexicographically, x1 > ... > xn), independently of the oracle's own code:

- sympy's groebner(..., modulus=p, order='grlex') gives the unique reduced basis in the same order;
- the comparator, seen through the oracle's sorted dictionary, agrees with sympy's grlex key
  on every monomial of a step;
- the zeros over F_p of the output equal those of the input (brute force);
- the two orders give different reduced bases where they must (a tie that grevlex and deglex break
  differently), and the same where the ideal is generated by linear forms;
- planted mistakes in the deglex comparator fail these pins."""
from __future__ import annotations

import os
import subprocess
import sys
import tempfile

import pytest
from sympy.polys.orderings import grlex

import oracle
from paper_2601_06765_b300 import synth
from tests import polyref as R


def sympy_reduced_gb_grlex(system: dict) -> list[list[tuple[tuple[int, ...], int]]]:
    """sympy's reduced Groebner basis over GF(p) in grlex, term lists sorted descending, polynomials
    by leading monomial descending."""
    from sympy import Poly, groebner, symbols
    n, p = system["n"], system["p"]
    X = symbols(f"x1:{n + 1}")
    F = [Poly.from_dict(f, *X, modulus=p).as_expr() for f in R.system_polys(system) if f]
    if not F:
        return []
    G = groebner(F, *X, modulus=p, order="grlex")
    out = [[(tuple(int(x) for x in m), int(c) % p) for m, c in g.terms(order="grlex")] for g in G.polys]
    out.sort(key=lambda t: grlex(t[0][0]), reverse=True)
    return out


def _systems():
    out = []
    for n in (2, 3, 4):
        for p in (7, 65521, 2147483647):
            out.append(synth.dense_system(n, n, p, 2000 + 10 * n + p % 89))
    for seed in range(3):
        out.append(synth.sparse_system(4, 4, 65521, 170 + seed, (3, 8)))
        out.append(synth.sparse_system(3, 3, 2147483647, 190 + seed, (2, 6), degree=3))
    for seed in (9007, 9011):
        out.append(synth.sparse_system(3, 3, 7, seed, (2, 4)))
    out.append(synth.dense_system(3, 2, 65521, 5))  # positive-dimensional
    out.append(synth.dense_system(2, 4, 65521, 6))  # overdetermined: basis {1}
    return out


@pytest.mark.parametrize("system", _systems(), ids=lambda s: f"n{s['n']}m{s['m']}p{s['p']}")
def test_deglex_reduced_basis_matches_sympy(system):
    assert oracle.groebner(system, oracle.DEGLEX) == sympy_reduced_gb_grlex(system)


def test_deglex_dictionary_order_matches_sympy_key():
    """Every step's dictionary is strictly descending in sympy's grlex key."""
    s = synth.dense_system(4, 4, 65521, 31)
    o = oracle.Oracle(s, oracle.DEGLEX)
    steps = 0
    while o.step():
        d = o.dump()
        keys = [grlex(tuple(int(x) for x in e)) for e in d.dict_exps]
        assert all(keys[i] > keys[i + 1] for i in range(len(keys) - 1))
        steps += 1
    assert steps >= 3


@pytest.mark.parametrize("n,p", [(2, 7), (3, 7), (3, 11)])
def test_deglex_variety_bruteforce(n, p):
    for seed in range(3):
        s = synth.sparse_system(n, n, p, 700 + seed, (2, 5))
        G = [R.terms_to_dict(t) for t in oracle.groebner(s, oracle.DEGLEX)]
        assert R.zeros(G, n, p) == R.zeros(R.system_polys(s), n, p)


def test_orders_differ_on_a_tie_and_agree_on_linear_forms():
    p = 65521
    # x1 x3 - x2^2 and x2 x3 - x1^2: grevlex leads with x2^2 and x1^2, deglex with x1 x3 and x1^2
    s = synth._pack(3, p, [[((1, 0, 1), 1), ((0, 2, 0), p - 1)], [((0, 1, 1), 1), ((2, 0, 0), p - 1)]])
    a, b = oracle.groebner(s), oracle.groebner(s, oracle.DEGLEX)
    assert a != b
    assert a == R.sympy_reduced_gb(s) and b == sympy_reduced_gb_grlex(s)
    # linear forms: both orders compare degree-1 monomials as x1 > x2 > ... > xn
    lin = synth._pack(3, p, [[((1, 0, 0), 2), ((0, 1, 0), 3), ((0, 0, 1), 5), ((0, 0, 0), 7)],
                             [((0, 1, 0), 1), ((0, 0, 1), 4), ((0, 0, 0), 1)]])
    assert oracle.groebner(lin) == oracle.groebner(lin, oracle.DEGLEX)


MUTANTS = {
    "deglex_tiebreak": ("            if (a->e[i] != b->e[i]) return a->e[i] > b->e[i] ? 1 : -1;",
                        "            if (a->e[i] != b->e[i]) return a->e[i] < b->e[i] ? 1 : -1;"),
    "deglex_scan_direction": ("        for (int i = 0; i < n; ++i)\n            if (a->e[i] != b->e[i]) return a->e[i] > b->e[i]",
                              "        for (int i = n - 1; i >= 0; --i)\n            if (a->e[i] != b->e[i]) return a->e[i] > b->e[i]"),
    "deglex_flag_ignored_in_step": ("    uint32_t p = S->p;\n    g_deglex = (S->flags & OR_DEGLEX) != 0;\n",
                                    "    uint32_t p = S->p;\n    g_deglex = 0;\n"),
}

PIN_SYSTEMS = [synth.dense_system(3, 3, 65521, 2013), synth.sparse_system(3, 3, 7, 9007, (2, 4)),
               synth.dense_system(4, 4, 7, 2041)]


def _deglex_pins_pass(lib) -> bool:
    try:
        return all(oracle.groebner(s, oracle.DEGLEX, lib) == sympy_reduced_gb_grlex(s) for s in PIN_SYSTEMS)
    except (AssertionError, KeyError, ValueError, IndexError, ZeroDivisionError):
        return False


def _pins_pass_in_child(source: str, tag: str) -> bool:
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with tempfile.TemporaryDirectory() as d:
        so = os.path.join(d, f"{tag}.so")
        code = ("import sys, oracle\n"
                "from tests.test_oracle_deglex import _deglex_pins_pass\n"
                f"lib = oracle.compile_variant(open({so!r} + '.src').read(), {so!r})\n"
                "sys.exit(0 if _deglex_pins_pass(lib) else 3)\n")
        with open(so + ".src", "w") as f:
            f.write(source)
        try:
            r = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, timeout=60)
        except subprocess.TimeoutExpired:
            return False
        return r.returncode == 0


def test_unmutated_source_passes_the_deglex_pins():
    assert _pins_pass_in_child(oracle.source(), "plain")


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_deglex_mutant_is_caught(name):
    old, new = MUTANTS[name]
    src = oracle.source()
    assert src.count(old) == 1, "mutation site must exist exactly once"
    assert not _pins_pass_in_child(src.replace(old, new), name)
