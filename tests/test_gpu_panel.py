"""The panel solve of RREF(D') spread over a thread-block cluster (k_panel_rref_cl) against the
oracle and against the one-block panel solves, bit for bit.

RREF(D') is unique (Sec. 9.2), so every schedule of the panel elimination must give the same bits.
The library routes panels of rows with at least 1024 columns to the cluster kernel;
GB_PANEL_CLUSTER_MIN_NB moves that bound here: down to 16, so that the oracle-checked systems'
panels take the cluster path, and up past every row length, so that the n=13 run's wide panels
take the one-block kernels for the comparison."""
from __future__ import annotations

import numpy as np
import pytest

import paper_2601_06765_b300 as gb
from paper_2601_06765_b300 import synth
from tests.test_gpu_parity import run_parity

pytestmark = pytest.mark.gpu

SYSTEMS = [("dense_n6", synth.dense_n6(0)), ("dense_n10", synth.dense_n10(0)),
           ("sparse_n5_cubic_p31", synth.sparse_system(5, 5, 2147483647, 71, (6, 14), degree=3)),
           ("sparse_n6_p65521", synth.sparse_system(6, 6, 65521, 77, (8, 20)))]


@pytest.mark.parametrize("name,system", SYSTEMS, ids=[n for n, _ in SYSTEMS])
def test_cluster_panels_equal_the_oracle(monkeypatch, name, system):
    monkeypatch.setenv("GB_PANEL_CLUSTER_MIN_NB", "16")
    with gb.Context(arena_bytes=4 << 30, keep_step=True, sketch=False) as ctx:
        assert run_parity(ctx, system) > 0


def _echelons(system, steps, **kw):
    out = []
    with gb.Context(arena_bytes=48 << 30, keep_step=True, **kw) as ctx, gb.System(ctx, system) as S:
        for _ in range(steps):
            st, stats = S.step()
            assert st == gb.GB_OK
            _, eh = gb.gb_system_last_step(S.h)
            ech = gb.gb_echelon_export(eh)
            out.append((stats["nb"], ech["rref_piv"].copy(), ech["rref"].copy()))
    return out


def test_wide_panels_equal_the_one_block_solves(monkeypatch):
    """The n=13 run's first 10 steps (rows of D' up to 8529 columns, D' up to 6864 rows) without
    the sketch, so that every panel of the full D' is solved: the cluster kernel against the
    one-block kernels (shared or global memory), RREF(D') bit for bit."""
    system = synth.sparse_n13(0)
    a = _echelons(system, 10, sketch=False)
    monkeypatch.setenv("GB_PANEL_CLUSTER_MIN_NB", str(1 << 30))
    b = _echelons(system, 10, sketch=False)
    assert max(nb for nb, _, _ in a) > 3200  # panels wider than one block's shared memory
    for (nb, piv_a, rr_a), (_, piv_b, rr_b) in zip(a, b):
        assert np.array_equal(piv_a, piv_b) and np.array_equal(rr_a, rr_b), nb
