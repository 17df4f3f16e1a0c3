"""The deglex term order on the CUDA path (the other graded order of Sec. 7.3), bit for bit against
the oracle run in deglex, whose own pins (sympy's grlex bases and keys) are in
test_oracle_deglex.py.  Every step is compared: dictionary, rows, CSR, D', RREF(D'), redundancy,
new basis elements and the reduced basis, with each reduction schedule forced."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2601_06765_b300 as gb
from paper_2601_06765_b300 import synth
from tests.test_gpu_parity import compare_step

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=["sparse", "dense"])
def ctx(request):
    c = gb.Context(arena_bytes=6 << 30, keep_step=True, reduce=request.param)
    yield c
    c.close()


def _deglex(system: dict) -> dict:
    return {**system, "order": "deglex"}


def run_parity_deglex(ctx, system, max_steps: int | None = None):
    o = oracle.Oracle(system, oracle.DEGLEX)
    with gb.System(ctx, _deglex(system)) as S:
        steps = 0
        while max_steps is None or steps < max_steps:
            st, stats = S.step()
            ran = o.step()
            assert (st == gb.GB_OK) == ran, f"step {steps + 1}: one side finished early"
            if not ran:
                break
            steps += 1
            d = o.dump()
            mac, ech = S.last_step()
            compare_step(d, mac, ech, f"deglex step {steps}")
            assert np.array_equal(S.redundant(), o.redundant()), f"step {steps}: redundancy"
            ng = o.basis_size()
            gpu_basis = S.basis(reduced=False)
            assert len(gpu_basis) == ng
            for i in range(ng - d.rref.shape[0], ng):
                assert gpu_basis[i] == o.basis_poly(i), f"step {steps}: element {i}"
        if max_steps is None or steps < max_steps:
            S.groebner()
            assert S.basis() == o.run(), "reduced basis"
        return steps


SMALL = [
    ("dense_n3_p16", synth.dense_system(3, 3, 65521, 11)),
    ("dense_n4_p31", synth.dense_system(4, 4, 2147483647, 12)),
    ("dense_n4_p7", synth.dense_system(4, 4, 7, 13)),
    ("sparse_n5_p16", synth.sparse_system(5, 5, 65521, 14, (4, 12))),
    ("sparse_n4_cubic_p31", synth.sparse_system(4, 4, 2147483629, 15, (5, 15), degree=3)),
    ("positive_dim_n4", synth.dense_system(4, 2, 65521, 18)),
    ("F7_pairs", synth.sparse_system(3, 3, 7, 9007, (2, 4))),
]


@pytest.mark.parametrize("name,system", SMALL, ids=[s[0] for s in SMALL])
def test_small_systems_deglex(ctx, name, system):
    run_parity_deglex(ctx, system)


def test_dense_n6_deglex(ctx):
    """n=6 dense quadratics mod 65521: every step and the reduced basis, in deglex."""
    assert run_parity_deglex(ctx, synth.dense_n6(0)) >= 5


def test_dictionary_order_is_deglex_exhaustive(ctx):
    """The device keys in deglex: one polynomial holding every monomial of degree <= 6 in 4
    variables; its dictionary lists all C(10, 4) = 210 monomials in sympy's grlex order."""
    from sympy.polys.orderings import grlex
    n, D = 4, 6
    mons = synth.monomials_upto(n, D)
    system = _deglex(synth._pack(n, 65521, [[(e, 1 + i) for i, e in enumerate(mons)]]))
    with gb.System(ctx, system) as S:
        mac = gb.gb_macaulay_export(gb.gb_symbolic_preprocess(S.h, n, np.zeros((1, n), np.uint8),
                                                              np.zeros(1, np.uint32), False))
    got = [tuple(int(x) for x in r) for r in mac["dict_exps"]]
    assert len(got) == 210
    assert got == sorted(mons, key=grlex, reverse=True)


def test_unknown_order_is_rejected(ctx):
    with pytest.raises(ValueError):
        gb.gb_system_create(ctx.h, {**synth.dense_system(2, 2, 7, 1), "order": "lex"})
