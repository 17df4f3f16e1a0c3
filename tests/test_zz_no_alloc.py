"""gb_reduce_rows_noalloc: the sparse row reduction for callers that cannot allocate device memory.

Such a caller owns all device memory through another allocator (a framework's caching allocator,
a pool fixed at start-up) that must not see the library take memory between its calls.  The
entry point works on caller-owned buffers (torch tensors here) plus a fixed scratch array inside
the library.  Its D' must equal the one the ordinary entry point gb_reduce_macaulay computes, and
the oracle's D' of the same F4 step, bit for bit, on consecutive calls with different matrices
(the scratch keeps the previous call's contents), and when the call is recorded into a CUDA graph
and replayed.  A matrix with a column index out of range
must leave D' at 0xFFFFFFFF, and the next valid call must be unaffected.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import paper_2601_06765_b300 as gb
from paper_2601_06765_b300 import synth

pytestmark = pytest.mark.gpu


def _matrix_after_steps(ctx, system, steps):
    """Pi of the last of `steps` F4 steps, D' from gb_reduce_macaulay on it, and the oracle's D'
    of the same step."""
    S = gb.System(ctx, system)
    for _ in range(steps):
        assert S.step()[0] == gb.GB_OK
    mac, _ = gb.gb_system_last_step(S.h)
    ech = gb.gb_reduce_macaulay(mac)
    want = gb.gb_echelon_export(ech)
    gb.gb_echelon_destroy(ech)
    o = oracle.Oracle(system)
    for _ in range(steps):
        assert o.step()
    return S, gb.gb_macaulay_export(mac), want, o.dump().dprime


def _device_u32(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def _run_noalloc(torch, p, m, want, col=None):
    npiv = int(m["npivot"])
    rp = m["row_ptr"]
    nC = len(rp) - 1 - npiv
    nb = len(want["nonpiv"])
    N = m["dict_exps"].shape[0]
    col = m["col"] if col is None else col
    pcols = m["col"][rp[:npiv]]  # leading column of each pivot row
    bufs = [_device_u32(torch, x) for x in (rp, col, m["val"], pcols, want["nonpiv"])]
    out = torch.full((max(nC * nb, 1),), 7, dtype=torch.int32, device="cuda")
    gb.gb_reduce_rows_noalloc(p, N, npiv, nC, nb, *(b.data_ptr() for b in bufs), out.data_ptr(),
                              torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32)[:nC * nb].reshape(nC, nb)


def test_noalloc_matches_gb_reduce_macaulay_and_the_oracle_on_consecutive_calls():
    import torch
    with gb.Context(arena_bytes=1 << 30, keep_step=True) as ctx:
        S1, m1, w1, o1 = _matrix_after_steps(ctx, synth.dense_n6(0), 5)                         # p = 65521
        S2, m2, w2, o2 = _matrix_after_steps(ctx, synth.dense_system(5, 5, 2147483647, 7), 4)  # 31-bit p
        assert w1["dprime"].size and w2["dprime"].size
        assert np.array_equal(w1["dprime"], o1) and np.array_equal(w2["dprime"], o2)
        first = _run_noalloc(torch, 65521, m1, w1)
        assert np.array_equal(first, w1["dprime"])
        second = _run_noalloc(torch, 2147483647, m2, w2)
        assert np.array_equal(second, w2["dprime"])
        # once the scratch address is known, a call adds no device allocation
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        third = _run_noalloc(torch, 65521, m1, w1)
        assert np.array_equal(third, o1)
        assert torch.cuda.mem_get_info()[0] >= free_before - (8 << 20)  # torch's own copies only
        S1.close()
        S2.close()


def test_noalloc_call_captured_in_a_cuda_graph_replays_exactly():
    """The call recorded into a CUDA graph on a side stream (after a first call on the device, as
    gb.h asks) and replayed twice, the second time after another matrix has gone through the
    scratch: every replay gives the captured matrix's D' (the job description is a kernel
    parameter of the graph's nodes, not a host buffer)."""
    import torch
    with gb.Context(arena_bytes=1 << 30, keep_step=True) as ctx:
        S1, m1, w1, o1 = _matrix_after_steps(ctx, synth.dense_n6(0), 5)                         # p = 65521
        S2, m2, w2, o2 = _matrix_after_steps(ctx, synth.dense_system(5, 5, 2147483647, 7), 4)  # 31-bit p
        assert np.array_equal(_run_noalloc(torch, 65521, m1, w1), o1)  # the first call on the device
        npiv = int(m1["npivot"])
        rp = m1["row_ptr"]
        nC, nb, N = len(rp) - 1 - npiv, len(w1["nonpiv"]), m1["dict_exps"].shape[0]
        bufs = [_device_u32(torch, x) for x in (rp, m1["col"], m1["val"], m1["col"][rp[:npiv]], w1["nonpiv"])]
        out = torch.full((nC * nb,), 7, dtype=torch.int32, device="cuda")
        side = torch.cuda.Stream()
        graph = torch.cuda.CUDAGraph()
        torch.cuda.synchronize()
        with torch.cuda.graph(graph, stream=side):
            gb.gb_reduce_rows_noalloc(65521, N, npiv, nC, nb, *(b.data_ptr() for b in bufs), out.data_ptr(),
                                      side.cuda_stream)
        for replay in range(2):
            out.fill_(7)
            graph.replay()
            torch.cuda.synchronize()
            got = out.cpu().numpy().view(np.uint32).reshape(nC, nb)
            assert np.array_equal(got, o1), f"replay {replay}"
            assert np.array_equal(_run_noalloc(torch, 2147483647, m2, w2), o2)  # the scratch changes hands
        S1.close()
        S2.close()


def test_noalloc_marks_dprime_when_an_index_is_out_of_range():
    """The device-side checks turn a column index >= ndict into D' = 0xFFFFFFFF everywhere
    (never a residue) instead of a write past the scratch; the next valid call is exact."""
    import torch
    with gb.Context(arena_bytes=1 << 30, keep_step=True) as ctx:
        S, m, w, o = _matrix_after_steps(ctx, synth.dense_n6(1), 4)
        N = m["dict_exps"].shape[0]
        bad = m["col"].copy()
        last_row = int(m["row_ptr"][-2])
        bad[last_row] = N + 5  # first entry of the last non-pivot row
        got = _run_noalloc(torch, 65521, m, w, col=bad)
        assert got.size and (got == 0xFFFFFFFF).all()
        assert np.array_equal(_run_noalloc(torch, 65521, m, w), o)
        S.close()


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
