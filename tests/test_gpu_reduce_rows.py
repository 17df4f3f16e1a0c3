"""The multi-row sparse reduction (k_reduce_rows: several non-pivot rows per block, sharing the
pivot-row entries staged in shared memory), bit for bit against the oracle.

The n=10 workload's middle steps have more non-pivot rows than the GPU has SMs and a 16-bit
prime, the shape that takes this kernel.  Its staging window normally holds a whole chunk of 32
pivot rows; GB_ROWS_WINDOW caps it so that every chunk is applied in many windows, down to eight
entries, where a window boundary falls inside almost every pivot row."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2601_06765_b300 as gb
from paper_2601_06765_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("window", [None, 1000, 8])
def test_dense_n10_steps_with_rows_kernel(window, monkeypatch):
    if window is not None:
        monkeypatch.setenv("GB_ROWS_WINDOW", str(window))
    system = synth.dense_n10(0)
    o = oracle.Oracle(system)
    ctx = gb.Context(arena_bytes=6 << 30, keep_step=True, reduce="sparse")
    try:
        with gb.System(ctx, system) as S:
            most_rows = 0
            for step in range(1, 9):
                st, stats = S.step()
                assert st == gb.GB_OK and o.step()
                d = o.dump()
                mac, ech = S.last_step()
                assert np.array_equal(mac["val"], d.val), f"step {step}: matrix"
                assert np.array_equal(ech["dprime"], d.dprime), f"step {step}: D'"
                assert np.array_equal(ech["rref"], d.rref), f"step {step}: RREF(D')"
                most_rows = max(most_rows, int(stats["nC"]))
            # the shape rule of the kernel: more non-pivot rows than SMs
            import torch
            assert most_rows > torch.cuda.get_device_properties(0).multi_processor_count
    finally:
        ctx.close()
