"""The seeded input generators against the recipe they state (shapes, ranges, structure), on the
CPU: the workloads of every test and of bench.py come from here, for both the oracle and the
CUDA path."""
from __future__ import annotations

from math import comb

import numpy as np
import pytest
import sympy

from paper_2601_06765_b300 import synth


def _polys(s):
    off = np.asarray(s["poly_off"])
    ex = np.asarray(s["exps"]).reshape(-1, s["n"])
    cf = np.asarray(s["coeffs"])
    return [(ex[off[i]:off[i + 1]], cf[off[i]:off[i + 1]]) for i in range(s["m"])]


def test_deterministic_per_seed():
    a, b, c = synth.dense_n10(0), synth.dense_n10(0), synth.dense_n10(1)
    for k in ("poly_off", "exps", "coeffs"):
        assert np.array_equal(np.asarray(a[k]), np.asarray(b[k]))
    assert not np.array_equal(np.asarray(a["coeffs"]), np.asarray(c["coeffs"]))


@pytest.mark.parametrize("make,n,p", [(synth.dense_n6, 6, 65521), (synth.dense_n10, 10, 65521)])
def test_dense_workloads_hold_every_quadratic_monomial(make, n, p):
    s = make(0)
    assert s["n"] == n and s["m"] == n and s["p"] == p
    want = sorted(synth.monomials_upto(n, 2))
    assert len(want) == comb(n + 2, 2)
    for ex, cf in _polys(s):
        assert sorted(tuple(int(x) for x in e) for e in ex) == want
        assert cf.min() >= 1 and cf.max() <= p - 1


def test_sparse_n13_recipe():
    s = synth.sparse_n13(0)
    assert s["n"] == 13 and s["m"] == 13 and s["p"] == 2 ** 31 - 1
    for ex, cf in _polys(s):
        mons = [tuple(int(x) for x in e) for e in ex]
        assert len(mons) == 30 == len(set(mons))
        degs = [sum(m) for m in mons]
        assert max(degs) == 2 and min(degs) >= 0
        assert cf.min() >= 1 and cf.max() <= s["p"] - 1


def test_mixed_batch_recipe():
    for s in synth.mixed_batch(24):
        n = s["n"]
        assert 5 <= n <= 9 and s["m"] == n and s["p"] == 65521
        tops = set()
        for ex, _ in _polys(s):
            mons = [tuple(int(x) for x in e) for e in ex]
            avail = len(synth.monomials_upto(n, max(sum(m) for m in mons)))
            assert len(mons) == len(set(mons))
            assert min(10, avail) <= len(mons) <= min(40, avail)
            tops.add(max(sum(m) for m in mons))
        assert len(tops) == 1 and tops <= {2, 3}


def test_largest_primes_below_2_31():
    ps = synth.largest_primes_below(2 ** 31, 128)
    assert len(ps) == 128 and ps[0] == 2 ** 31 - 1
    assert all(sympy.isprime(q) for q in ps)
    assert all(sympy.prevprime(ps[i]) == ps[i + 1] for i in range(len(ps) - 1))  # none skipped


def test_multi_prime_system_is_one_integer_system():
    """The coefficients modulo three primes come from one integer in [1, 2^31 - 2] (CRT)."""
    ps = synth.largest_primes_below(2 ** 31, 128)
    trio = [ps[0], ps[63], ps[127]]
    systems = synth.multi_prime_system(trio)
    cfs = [np.asarray(s["coeffs"], dtype=object) for s in systems]
    assert all(s["n"] == 8 and len(_polys(s)) == 8 for s in systems)
    for j in range(0, len(cfs[0]), 37):
        x = int(sympy.ntheory.modular.crt(trio[:2], [int(cfs[0][j]), int(cfs[1][j])])[0])
        assert 1 <= x <= 2 ** 31 - 2
        assert x % trio[2] == int(cfs[2][j])


def test_served_requests_and_arrivals():
    for i in range(40):
        s = synth.served_request(i)
        assert 5 <= s["n"] <= 11 and s["m"] == s["n"] and s["p"] in (65521, 2 ** 31 - 1)
    t = synth.poisson_arrivals(20000, 50.0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    assert abs(gaps.mean() - 1 / 50.0) < 0.05 / 50.0  # mean gap 1/rate within 5%
