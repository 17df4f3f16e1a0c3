"""gb_reduce_rows_noalloc: the sparse row reduction for callers that cannot allocate device memory.

Such callers record their work into a CUDA graph by stream capture (a cudaMalloc during capture
breaks the capture), or own all device memory through another allocator that must not see the
library grow between its calls.  The entry point works on caller-owned buffers (torch tensors
here) plus a fixed scratch array inside the library.  Its D' must equal the one the ordinary
entry point gb_reduce_macaulay computes, bit for bit, on consecutive calls with different
matrices (the scratch keeps the previous call's contents).
"""
from __future__ import annotations

import numpy as np
import pytest

import paper_2601_06765_b300 as gb
from paper_2601_06765_b300 import synth

pytestmark = pytest.mark.gpu


def _matrix_after_steps(ctx, system, steps):
    """Pi of the last of `steps` F4 steps, and D' from gb_reduce_macaulay on it."""
    S = gb.System(ctx, system)
    for _ in range(steps):
        assert S.step()[0] == gb.GB_OK
    mac, _ = gb.gb_system_last_step(S.h)
    ech = gb.gb_reduce_macaulay(mac)
    want = gb.gb_echelon_export(ech)
    gb.gb_echelon_destroy(ech)
    return S, gb.gb_macaulay_export(mac), want


def _device_u32(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def _run_noalloc(torch, p, m, want):
    npiv = int(m["npivot"])
    rp = m["row_ptr"]
    nC = len(rp) - 1 - npiv
    nb = len(want["nonpiv"])
    N = m["dict_exps"].shape[0]
    pcols = m["col"][rp[:npiv]]  # leading column of each pivot row
    bufs = [_device_u32(torch, x) for x in (rp, m["col"], m["val"], pcols, want["nonpiv"])]
    out = torch.full((max(nC * nb, 1),), -1, dtype=torch.int32, device="cuda")  # poisoned
    gb.gb_reduce_rows_noalloc(p, N, npiv, nC, nb, *(b.data_ptr() for b in bufs), out.data_ptr(),
                              torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32)[:nC * nb].reshape(nC, nb)


def test_noalloc_matches_gb_reduce_macaulay_on_consecutive_calls():
    import torch
    with gb.Context(arena_bytes=1 << 30, keep_step=True) as ctx:
        S1, m1, w1 = _matrix_after_steps(ctx, synth.dense_n6(0), 5)                         # p = 65521
        S2, m2, w2 = _matrix_after_steps(ctx, synth.dense_system(5, 5, 2147483647, 7), 4)  # 31-bit p
        assert w1["dprime"].size and w2["dprime"].size
        first = _run_noalloc(torch, 65521, m1, w1)
        assert np.array_equal(first, w1["dprime"])
        second = _run_noalloc(torch, 2147483647, m2, w2)
        assert np.array_equal(second, w2["dprime"])
        # once the scratch address is known, a call adds no device allocation
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        third = _run_noalloc(torch, 65521, m1, w1)
        assert np.array_equal(third, w1["dprime"])
        assert torch.cuda.mem_get_info()[0] >= free_before - (8 << 20)  # torch's own copies only
        S1.close()
        S2.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    with pytest.raises(gb.GbError) as e:
        gb.gb_reduce_rows_noalloc(65521, 60000, 10, 10, 10, 1, 1, 1, 1, 1, 1)
    assert e.value.status == -1
    with pytest.raises(gb.GbError):
        gb.gb_reduce_rows_noalloc(2147483647, 30000, 10, 10, 10, 1, 1, 1, 1, 1, 1)
    with pytest.raises(gb.GbError):
        gb.gb_reduce_rows_noalloc(65521, 1000, 20000, 10, 10, 1, 1, 1, 1, 1, 1)
    with pytest.raises(gb.GbError):
        gb.gb_reduce_rows_noalloc(65535, 100, 10, 10, 10, 1, 1, 1, 1, 1, 1)
