"""The sketched echelon form of a tall D' (RREF(R D') for a random R, checked exactly against D';
GB_CTX_SKETCH) against the oracle and against the full echelon form, bit for bit.

RREF(D') is the unique reduced basis of the row space of D' (Sec. 9.2), so a sketch that spans the
same space gives the same bits, and the exact check (D' - D'[:, piv] RREF = 0) sends any other
sketch back to the full echelon form.  The library sketches only D' with at least 2048 rows;
GB_SKETCH_MIN_ROWS lowers that bound here so that the small oracle-checked steps take the path,
and GB_SKETCH_RANK1 makes every sketch of rank one, whose check must fail on any D' of larger
rank (a D' of rank one is spanned by it, and is sketched correctly)."""
from __future__ import annotations

import numpy as np
import pytest

import paper_2601_06765_b300 as gb
from paper_2601_06765_b300 import synth
from tests.test_gpu_parity import run_parity

pytestmark = pytest.mark.gpu

SYSTEMS = [("dense_n6", synth.dense_n6(0)), ("dense_n10", synth.dense_n10(0)),
           ("sparse_n5_cubic_p31", synth.sparse_system(5, 5, 2147483647, 71, (6, 14), degree=3))]


def _sketched_steps(system, **kw):
    with gb.Context(arena_bytes=4 << 30, sketch=True, **kw) as ctx, gb.System(ctx, system) as S:
        out = []
        while True:
            st, stats = S.step()
            if st != gb.GB_OK:
                break
            out.append((stats["nC"], stats["rank"], stats["rref_sketched"]))
        return out


@pytest.mark.parametrize("name,system", SYSTEMS, ids=[n for n, _ in SYSTEMS])
def test_sketched_steps_equal_the_oracle(monkeypatch, name, system):
    monkeypatch.setenv("GB_SKETCH_MIN_ROWS", "16")
    assert any(sk for _, _, sk in _sketched_steps(system))  # some step's echelon form came from the sketch
    with gb.Context(arena_bytes=4 << 30, keep_step=True, sketch=True) as ctx:
        assert run_parity(ctx, system) > 0


@pytest.mark.parametrize("name,system", SYSTEMS[:2], ids=[n for n, _ in SYSTEMS[:2]])
def test_a_bad_sketch_is_caught_by_the_check(monkeypatch, name, system):
    monkeypatch.setenv("GB_SKETCH_MIN_ROWS", "16")
    monkeypatch.setenv("GB_SKETCH_RANK1", "1")
    steps = _sketched_steps(system)
    # a rank-one sketch spans D' only when D' has rank at most one; every other D' falls back
    assert all(rank <= 1 for _, rank, sk in steps if sk)
    assert any(nc >= 16 and rank > 1 and not sk for nc, rank, sk in steps)
    with gb.Context(arena_bytes=4 << 30, keep_step=True, sketch=True) as ctx:
        assert run_parity(ctx, system) > 0


def test_large_steps_sketched_equal_the_full_echelon_form():
    """The n=13 run's large steps (up to 6864 rows of D') with and without the sketch: the same
    RREF(D') bit for bit, and the sketch taken where D' is tall."""
    system = synth.sparse_n13(0)
    got = {}
    for sketch in (True, False):
        with gb.Context(arena_bytes=48 << 30, keep_step=True, sketch=sketch) as ctx, gb.System(ctx, system) as S:
            rows = []
            for _ in range(10):
                st, stats = S.step()
                assert st == gb.GB_OK
                _, eh = gb.gb_system_last_step(S.h)
                ech = gb.gb_echelon_export(eh)
                rows.append((stats["nC"], stats["rank"], stats["rref_sketched"], ech["rref_piv"].copy(),
                             ech["rref"].copy()))
            got[sketch] = rows
    assert any(r[2] for r in got[True]) and not any(r[2] for r in got[False])
    for (nc, rank, sk, piv_a, rr_a), (_, _, _, piv_b, rr_b) in zip(got[True], got[False]):
        assert np.array_equal(piv_a, piv_b) and np.array_equal(rr_a, rr_b)
        if nc >= 2048 and rank + 32 <= 512:  # tall, and the 512-row sketch has room for the rank
            assert sk
