"""The autotuner of the reduction schedules (gb_autotune, gb_tune_save / gb_tune_load).

The schedules it picks between give the same D' and RREF(D') (Sec. 9.2), so a tuned context must
reproduce every step of an untuned one bit for bit, and the oracle's reduced basis.  A table loaded
from a file must steer the reduction: a bucket set to the dense schedule reduces like a context
with the dense schedule forced (same work count), and an RREF bucket set to a graph schedule
launches graphs."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2601_06765_b300 as gb
from paper_2601_06765_b300 import synth

pytestmark = pytest.mark.gpu

SYSTEMS = [synth.dense_n6(0), synth.sparse_system(7, 7, 2147483647, 31, (10, 30))]


def _steps(ctx, system):
    """(stats, D', RREF) of every step, and the reduced basis."""
    out = []
    with gb.System(ctx, system) as S:
        while True:
            st, stats = S.step()
            if st != gb.GB_OK:
                break
            _, ech = S.last_step()
            out.append((stats, ech["dprime"].copy(), ech["rref"].copy()))
        S.groebner()
        return out, S.basis()


def _lg(x: int) -> int:
    return (x + 1).bit_length() - 1


def test_autotune_keeps_results_and_round_trips(tmp_path):
    with gb.Context(arena_bytes=2 << 30, keep_step=True) as plain, \
            gb.Context(arena_bytes=2 << 30, keep_step=True) as tuned:
        hs = [gb.gb_system_create(tuned.h, s) for s in SYSTEMS]
        rep = gb.gb_autotune(tuned.h, hs)
        for h in hs:
            gb.gb_system_destroy(h)
        assert rep["runs"] == 3 and rep["steps"] > 0
        assert rep["buckets_reduce"] > 0 and rep["buckets_rref"] > 0
        assert rep["buckets_scan"] == 17  # n = 2^8 .. 2^24
        for system in SYSTEMS:
            a, basis_a = _steps(plain, system)
            b, basis_b = _steps(tuned, system)
            assert len(a) == len(b)
            for i, (x, y) in enumerate(zip(a, b)):
                assert np.array_equal(x[1], y[1]), f"step {i + 1}: D'"
                assert np.array_equal(x[2], y[2]), f"step {i + 1}: RREF"
            assert basis_a == basis_b == oracle.Oracle(system).run()
        # save, load into a fresh context, save again: the same table
        f1, f2 = tmp_path / "t1.txt", tmp_path / "t2.txt"
        gb.gb_tune_save(tuned.h, str(f1))
        with gb.Context(arena_bytes=1 << 30) as other:
            gb.gb_tune_load(other.h, str(f1))
            gb.gb_tune_save(other.h, str(f2))
        rows = [ln for ln in f1.read_text().splitlines() if not ln.startswith("#")]
        assert rows and rows == [ln for ln in f2.read_text().splitlines() if not ln.startswith("#")]
        assert len(rows) == rep["buckets_reduce"] + rep["buckets_rref"] + rep["buckets_scan"]
        assert sum(ln.startswith("scan ") for ln in rows) == 17


def test_loaded_table_steers_the_schedules(tmp_path):
    system = SYSTEMS[1]
    with gb.Context(arena_bytes=2 << 30, keep_step=True, reduce="dense") as dense:
        want, basis_want = _steps(dense, system)
    cls = 1  # p = 2^31 - 1
    lines = set()
    for stats, _, _ in want:
        if stats["nC"] and stats["nb"]:
            lines.add(f"reduce {cls} {_lg(stats['npivot'])} {_lg(stats['nC'])} {_lg(stats['nb'])} 1 0 0 -1")
            lines.add(f"rref {cls} {_lg(stats['nC'])} {_lg(stats['nb'])} 0 2 0 0 0")
    table = tmp_path / "dense.txt"
    table.write_text("# every bucket of this run set to the tensor-core schedules\n" + "\n".join(sorted(lines)) + "\n")
    with gb.Context(arena_bytes=2 << 30, keep_step=True) as ctx:
        gb.gb_tune_load(ctx.h, str(table))
        g0 = gb.gb_graph_launches()
        got, basis_got = _steps(ctx, system)
        graphs = gb.gb_graph_launches() - g0
    assert basis_got == basis_want
    assert graphs > 0
    for (x, dx, rx), (y, dy, ry) in zip(want, got):
        assert np.array_equal(dx, dy) and np.array_equal(rx, ry)
        # the dense path counts its block updates as its work: equal counts, same schedule
        assert x["axpy_fma"] == y["axpy_fma"]


def test_tune_rejects_bad_input(tmp_path):
    with gb.Context(arena_bytes=1 << 30) as ctx:
        bad = tmp_path / "bad.txt"
        bad.write_text("reduce 0 3 3\n")
        with pytest.raises(gb.GbError) as e:
            gb.gb_tune_load(ctx.h, str(bad))
        assert e.value.status == -1  # GB_EINVAL
        bad.write_text("rref 0 3 3 0 7 0 0 0\n")  # no schedule 7
        with pytest.raises(gb.GbError):
            gb.gb_tune_load(ctx.h, str(bad))
        bad.write_text("scan 0 12 3 0 1 0 0 0\n")  # a scan bucket has one size
        with pytest.raises(gb.GbError):
            gb.gb_tune_load(ctx.h, str(bad))
        with pytest.raises(gb.GbError):
            gb.gb_tune_load(ctx.h, str(tmp_path / "missing.txt"))
        # a system that has already run a step cannot be tuned on
        h = gb.gb_system_create(ctx.h, SYSTEMS[0])
        gb.gb_f4_step(h)
        with pytest.raises(gb.GbError) as e:
            gb.gb_autotune(ctx.h, [h])
        assert e.value.status == -1  # GB_EINVAL
        gb.gb_system_destroy(h)


def test_scan_tiles_from_a_loaded_table_keep_results(tmp_path):
    """Every prefix-sum tile (4, 8, 16 values per thread) gives the same plans: a table that sets
    each size bucket to one tile in turn leaves every step of a run bit-identical."""
    system = synth.dense_n6(0)
    with gb.Context(arena_bytes=1 << 30, keep_step=True) as ctx:
        want, basis = _steps(ctx, system)
    for choice in range(3):
        table = tmp_path / f"scan{choice}.txt"
        table.write_text("".join(f"scan 0 {b} 0 0 {choice} 0 0 0\n" for b in range(0, 33)))
        with gb.Context(arena_bytes=1 << 30, keep_step=True) as ctx:
            gb.gb_tune_load(ctx.h, str(table))
            got, basis_got = _steps(ctx, system)
        assert basis_got == basis
        for (x, dx, rx), (y, dy, ry) in zip(want, got):
            assert x["nnz"] == y["nnz"] and np.array_equal(dx, dy) and np.array_equal(rx, ry)
