"""Planted mistakes: each mutant is the oracle's C source with one plausible error (a wrong sign,
a dropped term, a transposed operand, an off-by-one, a missing condition), compiled on the CPU.
Every mutant must fail at least one of the pins, which shows that the pins would catch that kind
of mistake in the oracle itself."""
from __future__ import annotations

import os
import subprocess
import sys
import tempfile

import pytest

import oracle
from paper_2601_06765_b300 import synth
from tests import polyref as R
from tests.test_oracle_pins import (PAIR_SYSTEMS, check_dictionary_matrix_closure,
                                    check_pairs_replay, check_reduction_and_echelon)

MUTANTS = {
    "axpy_sign": ("uint32_t mf = p - f; /* v <- v - f * pivot row */",
                  "uint32_t mf = f; /* v <- v - f * pivot row */"),
    "grevlex_tiebreak": ("if (a->e[i] != b->e[i]) return a->e[i] < b->e[i] ? 1 : -1;",
                         "if (a->e[i] != b->e[i]) return a->e[i] > b->e[i] ? 1 : -1;"),
    "grevlex_scan_direction": ("for (int i = n - 1; i >= 0; --i)\n        if (a->e[i] != b->e[i])",
                               "for (int i = 0; i < n; ++i)\n        if (a->e[i] != b->e[i])"),
    "dropped_term_in_expansion": ("        for (int j = 0; j < f->len; ++j) {\n            omono m = m_mul(&rows[a].t, &f->mon[j], n);\n            if (set_insert",
                                  "        for (int j = 0; j < f->len - 1; ++j) {\n            omono m = m_mul(&rows[a].t, &f->mon[j], n);\n            if (set_insert"),
    "csr_value_index_shift": ("            val[row_ptr[a] + j] = f->cf[j];",
                              "            val[row_ptr[a] + j] = f->cf[j ? j - 1 : 0];"),
    "rref_not_reduced": ("        for (int i = 0; i < nC; ++i) {\n            if (i == rank) continue;",
                         "        for (int i = rank + 1; i < nC; ++i) {\n            if (i == rank) continue;"),
    "lcm_is_gcd": ("r.e[i] = a->e[i] > b->e[i] ? a->e[i] : b->e[i];",
                   "r.e[i] = a->e[i] < b->e[i] ? a->e[i] : b->e[i];"),
    "inverse_sign_fix_dropped": ("    if (s0 < 0) s0 += p;\n", "\n"),
    "pair_filter_too_eager": ("int drop = m_divides(lh, &l12, n) && !m_eq(&l1h, &l12, n) && !m_eq(&l2h, &l12, n);",
                              "int drop = m_divides(lh, &l12, n) && !m_eq(&l1h, &l12, n);"),
    "reducer_ignores_redundancy": ("        for (int g = 0; g < S->ng; ++g)\n            if (!S->redundant[g] && m_divides(&S->g[g].mon[0], m, S->n)) return g;",
                                   "        for (int g = 0; g < S->ng; ++g)\n            if (m_divides(&S->g[g].mon[0], m, S->n)) return g;"),
    "pivot_pair_row_largest_k": ("if (best[c] < 0 || rows[a].k < rows[best[c]].k) best[c] = a;",
                                 "if (best[c] < 0 || rows[a].k > rows[best[c]].k) best[c] = a;"),
    "reduction_starts_one_column_late": ("    for (int c = start; c < N; ++c) {",
                                         "    for (int c = start + 1; c < N; ++c) {"),
    "tail_not_reduced": ("        opoly r = full_reduce(S, &tail, B, nB);",
                         "        opoly r = full_reduce(S, &tail, B, 0);"),
    # pair selection (normal strategy) and the Gebauer-Moeller update: these change every
    # intermediate matrix but not the reduced basis, so only the pair replay catches them
    "selection_takes_largest_degree": ("        if (d < dmin) dmin = d;",
                                       "        if (d > dmin || dmin == 1 << 30) dmin = d;"),
    "product_criterion_dropped": ("if (keepD[a] && !m_coprime(lh, &S->g[C[a]].mon[0], n)) add_pair(S, C[a], hidx);",
                                  "if (keepD[a]) add_pair(S, C[a], hidx);"),
    "chain_criterion_on_old_pairs_dropped": ("        if (!drop) S->pairs[w++] = S->pairs[q];",
                                             "        (void)drop; S->pairs[w++] = S->pairs[q];"),
    "equal_pair_rows_not_collapsed": ("if (u == 0 || rows[u - 1].k != rows[a].k || !m_eq(&rows[u - 1].t, &rows[a].t, n)) rows[u++] = rows[a];",
                                      "rows[u++] = rows[a];"),
    "first_loop_checks_rejected_pairs": ("                if (keepD[b] && m_divides(&L[b], &L[a], n)) keep = 0;",
                                         "                if (m_divides(&L[b], &L[a], n)) keep = 0;"),
    "first_loop_no_coprime_exemption": ("        if (!m_coprime(lh, &S->g[C[a]].mon[0], n)) {",
                                        "        if (1) {"),
}

SMALL = [synth.sparse_system(3, 3, 7, 9007, (2, 4)), synth.sparse_system(3, 3, 7, 9011, (2, 4)),
         synth.dense_system(3, 3, 65521, 1), synth.dense_system(4, 4, 7, 2),
         synth.sparse_system(3, 3, 2147483647, 3, (3, 6), degree=3)]


def _pins_pass(lib) -> bool:
    try:
        for s in SMALL:
            if oracle.groebner(s, lib=lib) != R.sympy_reduced_gb(s):
                return False
        check_dictionary_matrix_closure(synth.dense_system(4, 4, 65521, 9), lib=lib, limit=4)
        check_reduction_and_echelon(synth.dense_system(3, 3, 65521, 10), lib=lib, limit=3)
        for s in PAIR_SYSTEMS:
            check_pairs_replay(s, lib=lib)
    except (AssertionError, KeyError, ValueError, IndexError, ZeroDivisionError):
        return False
    return True


def _pins_pass_in_child(source: str, tag: str) -> bool:
    """Compile `source` and run the pins in a child process: a mutant may also crash (the oracle
    aborts when a row monomial is missing from its dictionary) or stop terminating, which both
    count as caught."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with tempfile.TemporaryDirectory() as d:
        so = os.path.join(d, f"{tag}.so")
        code = ("import sys, oracle\n"
                "from tests.test_oracle_mutants import _pins_pass\n"
                f"lib = oracle.compile_variant(open({so!r} + '.src').read(), {so!r})\n"
                "sys.exit(0 if _pins_pass(lib) else 3)\n")
        with open(so + ".src", "w") as f:
            f.write(source)
        try:
            r = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True,
                               timeout=30)
        except subprocess.TimeoutExpired:  # a mutant whose F4 loop no longer terminates
            return False
        return r.returncode == 0


def test_unmutated_source_passes():
    assert _pins_pass_in_child(oracle.source(), "plain")


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name):
    old, new = MUTANTS[name]
    src = oracle.source()
    assert src.count(old) == 1, "mutation site must exist exactly once"
    assert not _pins_pass_in_child(src.replace(old, new), name)
