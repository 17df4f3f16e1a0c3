"""The rounds of RREF(D') (Sec. 9.2) recorded as one CUDA graph whose loop runs on the device, against
the same rounds launched one by one from the host (GB_CTX_NO_GRAPHS).  Every step's D', RREF(D')
and pivot columns, and the reduced basis, must agree bit for bit; the oracle pins the basis."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2601_06765_b300 as gb
from paper_2601_06765_b300 import synth

pytestmark = pytest.mark.gpu

CASES = [
    ("dense_n6", synth.dense_n6(0), "auto"),
    ("sparse_n7_p31", synth.sparse_system(7, 7, 2147483647, 21, (10, 30)), "auto"),
    # forced dense: the rounds also hold the tensor-core trailing update (k_mm) of each panel
    ("dense_n6_p16_tc", synth.dense_system(6, 6, 65521, 22), "dense"),
]


def _run(system, reduce, graphs):
    steps = []
    with gb.Context(arena_bytes=2 << 30, keep_step=True, reduce=reduce, graphs=graphs) as ctx:
        with gb.System(ctx, system) as S:
            graphs0 = gb.gb_graph_launches()
            while S.step()[0] == gb.GB_OK:
                _, ech = S.last_step()
                steps.append((ech["dprime"].copy(), ech["rref"].copy(), ech["rref_piv"].copy()))
            S.groebner()
            return steps, S.basis(), gb.gb_graph_launches() - graphs0


@pytest.mark.parametrize("name,system,reduce", CASES, ids=[c[0] for c in CASES])
def test_graph_rounds_match_host_rounds(name, system, reduce):
    g_steps, g_basis, g_graphs = _run(system, reduce, True)
    h_steps, h_basis, h_graphs = _run(system, reduce, False)
    assert len(g_steps) == len(h_steps)
    for i, (a, b) in enumerate(zip(g_steps, h_steps)):
        for what, x, y in zip(("D'", "RREF", "pivots"), a, b):
            assert np.array_equal(x, y), f"{name} step {i + 1}: {what}"
    assert g_basis == h_basis
    assert g_basis == oracle.Oracle(system).run()
    # the first run took the graph path at least once (D' of three panels or more), the second never
    assert g_graphs > 0 and h_graphs == 0
