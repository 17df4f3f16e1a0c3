"""Parity of the CUDA path with the CPU oracle, bit for bit (integer work: no tolerance).

Every F4 step is compared: the dictionary T (the dictionary-correctness theorem of Sec. 11), the
row metadata and the CSR plan Pi (the matrix-materialisation theorem of Sec. 11), the reduced
non-pivot block D' and RREF(D') (Sec. 9.2), the redundancy flags, the new basis elements, and
finally the reduced Groebner basis.  All calls go through the C ABI."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2601_06765_b300 as gb
from paper_2601_06765_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=["sparse", "dense", "sparse-hash"])
def ctx(request):
    """Every case runs with each reduction schedule forced: the sparse row-by-row reduction and
    the dense blocked elimination on the tensor cores must both reproduce the unique D'.  The
    symbolic preprocessing ranks every term into a bitmap, and once more (sparse-hash) goes
    through the hash dictionary: both must build the same T and Pi."""
    reduce, _, sp = request.param.partition("-")
    c = gb.Context(arena_bytes=6 << 30, keep_step=True, reduce=reduce, sp=sp or "ranks")
    yield c
    c.close()


def compare_step(d: oracle.StepDump, mac: dict, ech: dict, where: str):
    assert np.array_equal(mac["dict_exps"], d.dict_exps), f"{where}: dictionary"
    assert np.array_equal(mac["row_t"], d.row_t), f"{where}: row shifts"
    assert np.array_equal(mac["row_k"], d.row_k), f"{where}: row basis indices"
    assert np.array_equal(mac["row_flags"] & 1, d.row_pivot), f"{where}: pivot flags"
    assert np.array_equal((mac["row_flags"] >> 1) & 1, d.row_reducer), f"{where}: reducer flags"
    assert np.array_equal(mac["row_ptr"], d.row_ptr), f"{where}: row_ptr"
    assert np.array_equal(mac["col"], d.col), f"{where}: col_ind"
    assert np.array_equal(mac["val"], d.val), f"{where}: val"
    assert mac["npivot"] == d.nA
    assert np.array_equal(ech["nonpiv"], d.nonpiv), f"{where}: non-pivot columns"
    assert np.array_equal(ech["dprime"], d.dprime), f"{where}: D'"
    assert np.array_equal(ech["rref_piv"], d.rref_piv), f"{where}: RREF pivots"
    assert np.array_equal(ech["rref"], d.rref), f"{where}: RREF(D')"


def run_parity(ctx, system, max_steps: int | None = None, final: bool = True):
    o = oracle.Oracle(system)
    with gb.System(ctx, system) as S:
        assert np.array_equal(S.redundant(), o.redundant())
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
            compare_step(d, mac, ech, f"step {steps}")
            assert stats["nnz"] == d.nnz and stats["rank"] == d.rref.shape[0]
            assert np.array_equal(S.redundant(), o.redundant()), f"step {steps}: redundancy"
            # the new basis elements
            ng = o.basis_size()
            gpu_basis = S.basis(reduced=False)
            assert len(gpu_basis) == ng
            for i in range(ng - d.rref.shape[0], ng):
                assert gpu_basis[i] == o.basis_poly(i), f"step {steps}: element {i}"
        if final and (max_steps is None or steps < max_steps):
            S.groebner()
            assert S.basis() == o.run(), "reduced basis"
        return steps


SMALL = [
    ("dense_n3_p16", synth.dense_system(3, 3, 65521, 11)),
    ("dense_n4_p31", synth.dense_system(4, 4, 2147483647, 12)),
    ("dense_n4_p7", synth.dense_system(4, 4, 7, 13)),
    ("sparse_n5_p16", synth.sparse_system(5, 5, 65521, 14, (4, 12))),
    ("sparse_n4_cubic_p31", synth.sparse_system(4, 4, 2147483629, 15, (5, 15), degree=3)),
    ("sparse_n6_p16", synth.sparse_system(6, 6, 65521, 16, (8, 20))),
    ("overdetermined_n3", synth.dense_system(3, 5, 65521, 17)),
    ("positive_dim_n4", synth.dense_system(4, 2, 65521, 18)),
    ("unit_ideal_n2", synth.dense_system(2, 4, 65521, 19)),
    ("F7_pairs", synth.sparse_system(3, 3, 7, 9007, (2, 4))),
]


@pytest.mark.parametrize("name,system", SMALL, ids=[s[0] for s in SMALL])
def test_small_systems(ctx, name, system):
    run_parity(ctx, system)


@pytest.mark.parametrize("seed", range(3))
def test_dense_n6(ctx, seed):
    """n=6 dense quadratics mod 65521: every step and the reduced basis."""
    assert run_parity(ctx, synth.dense_n6(seed)) >= 5


def test_dense_n10_full(ctx):
    """The benchmark workload (n=10 dense quadratics mod 65521), every step bit-exact."""
    assert run_parity(ctx, synth.dense_n10(0)) == 11


def test_sparse_n13_p31_first_steps(ctx):
    """n=13 sparse quadratics mod 2^31-1 (31-bit Montgomery path): the first steps the oracle
    finishes in seconds."""
    run_parity(ctx, synth.sparse_n13(0), max_steps=4, final=False)


def test_mixed_batch_members(ctx):
    """A few members of the mixed batch (quadratic and cubic, n in 5..9), whole runs."""
    batch = synth.mixed_batch(256)
    for i in (1, 0, 3, 5):
        run_parity(ctx, batch[i])


def test_multi_prime_members(ctx):
    """The n=8 dense system modulo several of the 128 largest primes below 2^31 (first steps)."""
    primes = synth.largest_primes_below(2 ** 31, 128)
    systems = synth.multi_prime_system([primes[0], primes[63], primes[127]])
    for s in systems:
        run_parity(ctx, s, max_steps=4, final=False)


def test_standalone_sp_and_reduce_match_oracle_steps(ctx):
    """gb_symbolic_preprocess + gb_reduce_macaulay called directly with the oracle's pair rows of
    step k (after k-1 F4 steps on the device) reproduce the oracle's step-k matrices."""
    system = synth.dense_n6(1)
    o = oracle.Oracle(system)
    with gb.System(ctx, system) as S:
        for k in range(1, 6):
            assert o.step()
            d = o.dump()
            pair = d.row_reducer == 0
            mac = gb.gb_symbolic_preprocess(S.h, S.n, d.row_t[pair], d.row_k[pair], True)
            ech = gb.gb_reduce_macaulay(mac)
            mh = gb.gb_macaulay_export(mac)
            compare_step(d, mh, gb.gb_echelon_export(ech), f"standalone {k}")
            ms = gb.gb_macaulay_stats_get(mac)  # the per-run record: N, M = nnz, the stage split
            assert (ms["nnz"], ms["ndict"], ms["nrows"]) == (len(mh["col"]), mh["dict_exps"].shape[0], len(mh["row_ptr"]) - 1)
            assert 0 < ms["ms_dict"] <= ms["ms_sp"] and ms["ms_assemble"] >= 0
            gb.gb_echelon_destroy(ech)
            gb.gb_macaulay_destroy(mac)
            assert S.step()[0] == gb.GB_OK


def test_sp_without_closure(ctx):
    """closure = 0: T is exactly the union of the given rows' supports (the support-closure
    definition of Sec. 11), no reducer rows."""
    system = synth.dense_system(4, 4, 65521, 77)
    with gb.System(ctx, system) as S:
        t = np.zeros((4, 4), np.uint8)
        t[1, 0] = 1
        t[2, 3] = 2
        k = np.array([0, 1, 2, 3], np.uint32)
        mac = gb.gb_macaulay_export(gb.gb_symbolic_preprocess(S.h, 4, t, k, False))
        basis = S.basis(reduced=False)
        union = set()
        for ti, ki in zip(t, k):
            for e, _ in basis[ki]:
                union.add(tuple(int(a + b) for a, b in zip(e, ti)))
        assert {tuple(int(x) for x in r) for r in mac["dict_exps"]} == union
        assert not ((mac["row_flags"] >> 1) & 1).any()


def test_dictionary_order_is_grevlex_exhaustive(ctx):
    """The key assumption of Sec. 11 (injective, order-refining keys) on the device keys: one
    polynomial holding every monomial of degree <= 6 in 4 variables; its dictionary must list all C(10, 4) = 210 monomials in sympy's grevlex order."""
    from sympy.polys.orderings import grevlex
    n, D = 4, 6
    mons = synth.monomials_upto(n, D)
    system = synth._pack(n, 65521, [[(e, 1 + i) for i, e in enumerate(mons)]])
    with gb.System(ctx, system) as S:
        mac = gb.gb_macaulay_export(gb.gb_symbolic_preprocess(S.h, n, np.zeros((1, n), np.uint8),
                                                              np.zeros(1, np.uint32), False))
    got = [tuple(int(x) for x in r) for r in mac["dict_exps"]]
    assert len(got) == 210
    assert got == sorted(mons, key=grevlex, reverse=True)


def test_determinism(ctx):
    """the determinism theorem of Sec. 11: the same batch gives byte-identical plans on repeated runs."""
    system = synth.dense_n6(2)
    dumps = []
    for _ in range(2):
        with gb.System(ctx, system) as S:
            out = []
            while S.step()[0] == gb.GB_OK:
                out.append(S.last_step())
            dumps.append(out)
    for (m1, e1), (m2, e2) in zip(*dumps):
        for key in m1:
            assert np.array_equal(np.asarray(m1[key]), np.asarray(m2[key]))
        for key in e1:
            assert np.array_equal(e1[key], e2[key])


def test_errors_are_reported(ctx):
    with pytest.raises(gb.GbError) as ei:
        gb.gb_system_create(ctx.h, {**synth.dense_system(2, 2, 7, 1), "p": 65535})
    assert ei.value.status == -1
    with pytest.raises(gb.GbError):
        gb.gb_system_create(ctx.h, {**synth.dense_system(2, 2, 7, 1), "n": 17})
    empty = synth._pack(3, 65521, [])
    with gb.System(ctx, empty) as S:
        assert S.step()[0] == gb.GB_DONE
        S.groebner()
        assert S.basis() == []
    zero = synth._pack(3, 65521, [[((1, 0, 0), 5), ((1, 0, 0), 65516)]])
    with gb.System(ctx, zero) as S:
        S.groebner()
        assert S.basis() == []
