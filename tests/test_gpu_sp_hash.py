"""The hash dictionary of symbolic preprocessing (GB_CTX_SP_HASH) and its two exits, against the
oracle bit for bit.

The hash path keys every term by an additive 64-bit monomial key and checks every lookup against
the stored monomial.  Two monomials sharing a key (forced here by keeping only a few key bits,
GB_SP_KEY_MASK) must send the step through the exact rank path, and a table that fills up (forced
by starting it with 64 slots, GB_SP_TABLE_SLOTS) must grow; either way every dictionary, CSR plan,
D', RREF(D') and the reduced basis equal the oracle's (the dictionary-correctness and
matrix-materialisation theorems of Sec. 11)."""
from __future__ import annotations

import pytest

import paper_2601_06765_b300 as gb
from paper_2601_06765_b300 import synth
from tests.test_gpu_parity import compare_step  # noqa: F401  (the per-step comparison)
from tests.test_gpu_parity import run_parity

pytestmark = pytest.mark.gpu

SYSTEMS = [("dense_n6", synth.dense_n6(0)),
           ("sparse_n5_cubic_p31", synth.sparse_system(5, 5, 2147483647, 71, (6, 14), degree=3))]


def _redo_counts(system, **ctx_kw):
    with gb.Context(arena_bytes=2 << 30, sp="hash", **ctx_kw) as ctx, gb.System(ctx, system) as S:
        out = []
        while True:
            st, stats = S.step()
            if st != gb.GB_OK:
                break
            out.append(stats["sp_redo"])
        return out


@pytest.mark.parametrize("name,system", SYSTEMS, ids=[n for n, _ in SYSTEMS])
def test_hash_path_needs_no_redo_on_the_workloads(name, system):
    assert _redo_counts(system) and all(r == 0 for r in _redo_counts(system))


@pytest.mark.parametrize("mask", ["0x0", "0xff"])
@pytest.mark.parametrize("name,system", SYSTEMS, ids=[n for n, _ in SYSTEMS])
def test_shared_keys_fall_back_to_the_rank_path(monkeypatch, mask, name, system):
    monkeypatch.setenv("GB_SP_KEY_MASK", mask)
    redo = _redo_counts(system)
    assert any(r > 0 for r in redo)  # the clash was seen and the step built again
    with gb.Context(arena_bytes=2 << 30, keep_step=True, sp="hash") as ctx:
        assert run_parity(ctx, system) > 0


@pytest.mark.parametrize("name,system", SYSTEMS, ids=[n for n, _ in SYSTEMS])
def test_a_full_table_grows(monkeypatch, name, system):
    monkeypatch.setenv("GB_SP_TABLE_SLOTS", "64")
    redo = _redo_counts(system)
    assert any(r > 0 for r in redo)
    with gb.Context(arena_bytes=2 << 30, keep_step=True, sp="hash") as ctx:
        assert run_parity(ctx, system) > 0


def test_rank_path_context_flag_gives_the_same_steps():
    s = synth.sparse_system(6, 6, 65521, 77, (8, 20))
    for sp in ("hash", "ranks"):
        with gb.Context(arena_bytes=2 << 30, keep_step=True, sp=sp) as ctx:
            assert run_parity(ctx, s) > 0
