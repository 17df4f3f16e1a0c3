"""The library's critical-pair bookkeeping (the host side of the F4 loop, csrc/f4.cpp) against the
textbook model of tests/polyref.py, on the CPU (no device is used).

The library inserts the new elements of one F4 step together: for each element it finds the least
newer element of the step whose leading monomial divides its own, forms every new element's pairs
against the elements still in the basis at its turn, and prunes them by the Gebauer-Moeller
criteria in a closed form of the sequential rule.  The model inserts one element at a time by the
procedure UPDATE of Becker-Weispfenning.  Between steps both remove the pairs of the least lcm
degree (the normal selection).  After every replay the pair sets and the basis membership must be
equal, for random leading monomials (small exponents, so that divisibility, equal lcms and coprime
pairs are frequent) in random step sizes.
"""
from __future__ import annotations

import numpy as np
import pytest

import paper_2601_06765_b300 as gb
from tests.polyref import PairModel


def model_replay(lms, group_sizes, select_before):
    M = PairModel()
    e = 0
    for g, size in enumerate(group_sizes):
        if select_before[g] and M.B:
            M.select()
        for _ in range(size):
            M.insert(tuple(int(x) for x in lms[e]))
            e += 1
    return sorted(M.B), M.in_g


def random_case(rng, n, nelem, emax):
    lms = rng.integers(0, emax + 1, size=(nelem, n)).astype(np.uint8)
    sizes = []
    left = nelem
    while left:
        s = int(min(left, rng.integers(1, 9)))
        sizes.append(s)
        left -= s
    select = [0] + [int(rng.random() < 0.8) for _ in sizes[1:]]
    return lms, sizes, select


@pytest.mark.parametrize("seed", range(40))
def test_replay_equals_the_textbook_update(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 7))
    lms, sizes, select = random_case(rng, n, int(rng.integers(5, 60)), int(rng.integers(1, 4)))
    got = gb.gb_pair_update_replay(n, lms, sizes, select)
    assert got == model_replay(lms, sizes, select), (n, sizes)


@pytest.mark.parametrize("seed", range(6))
def test_one_step_and_one_at_a_time_agree(seed):
    """All elements in one group gives what inserting them one group each gives (no selection in
    between): the library's step-level update is the sequential one."""
    rng = np.random.default_rng(100 + seed)
    n = 4
    lms = rng.integers(0, 3, size=(40, n)).astype(np.uint8)
    together = gb.gb_pair_update_replay(n, lms, [40])
    single = gb.gb_pair_update_replay(n, lms, [1] * 40)
    assert together == single == model_replay(lms, [40], [0])


def test_special_cases():
    # equal leading monomials: the later one divides the earlier, which leaves the basis
    lms = np.array([[1, 1], [1, 1], [2, 0]], dtype=np.uint8)
    got = gb.gb_pair_update_replay(2, lms, [3])
    assert got == model_replay(lms, [3], [0])
    assert got[1][0] is False
    # coprime leading monomials only: the product criterion leaves no pair
    lms = np.array([[3, 0, 0], [0, 2, 0], [0, 0, 5]], dtype=np.uint8)
    assert gb.gb_pair_update_replay(3, lms, [1, 1, 1]) == ([], [True, True, True])
    # a constant: it divides every other leading monomial
    lms = np.array([[1, 2], [2, 1], [0, 0]], dtype=np.uint8)
    got = gb.gb_pair_update_replay(2, lms, [2, 1], [0, 1])
    assert got == model_replay(lms, [2, 1], [0, 1]) and got[1] == [False, False, True]
    # nothing at all
    assert gb.gb_pair_update_replay(3, np.zeros((0, 3), dtype=np.uint8), []) == ([], [])


def test_rejected_arguments():
    with pytest.raises(gb.GbError):
        gb.gb_pair_update_replay(17, np.zeros((1, 17), dtype=np.uint8), [1])
    with pytest.raises(gb.GbError):
        gb.gb_pair_update_replay(2, np.zeros((3, 2), dtype=np.uint8), [2])
