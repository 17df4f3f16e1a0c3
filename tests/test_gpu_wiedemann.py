"""gb_block_wiedemann (Sec. 9.3; Prop. 3.2) against the oracle, bit for bit: the block Krylov
sequence S_i = X^T M^(i+1) Z and the canonical basis W of the kernel vectors found, on the same
step matrices and the same random blocks.  At sizes the oracle cannot reach, what holds at any
size: W has min(b, dim ker A^T) rows, every row w satisfies w^T A = 0 (recomputed here on the
host from the exported matrix), and the device's own check agrees."""
from __future__ import annotations

import numpy as np
import pytest

import paper_2601_06765_b300 as gb
from oracle import wiedemann as OW
from paper_2601_06765_b300 import synth
from tests.test_oracle_wiedemann import CASES, random_inputs, step_matrix

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = gb.Context(arena_bytes=8 << 30, keep_step=True)
    yield c
    c.close()


def gpu_step(ctx, system, step):
    S = gb.System(ctx, system)
    for _ in range(step):
        st, stats = S.step()
        assert st == gb.GB_OK
    mac, _ = gb.gb_system_last_step(S.h)
    return S, mac, stats


@pytest.mark.parametrize("b", [2, 4, 8, 32])
@pytest.mark.parametrize("name,system,step", CASES, ids=[c[0] for c in CASES])
def test_sequence_and_kernel_basis_equal_the_oracle(ctx, name, system, step, b):
    _, d = step_matrix(system, step)
    p = system["p"]
    r, N = len(d.row_k), d.N
    X, Z, delta = random_inputs(r, N, b, p, 11 + b)
    want = OW.block_wiedemann(d.row_ptr, d.col, d.val, N, p, X, Z, delta)
    S, mac, _ = gpu_step(ctx, system, step)
    got = gb.gb_block_wiedemann(mac, b, np.array(X), np.array(Z), np.array(delta), wcap=64)
    S.close()
    assert got["d"] == want["d"] and got["nterms"] == len(want["seq"])
    for i, s in enumerate(want["seq"]):
        assert np.array_equal(got["seq"][i], np.array(s, dtype=np.int64).astype(np.uint32)), f"S_{i}"
    assert got["hankel_rank"] == len(want["H_piv"])
    assert np.array_equal(got["W"], np.array(want["W"], dtype=np.int64).astype(np.uint32).reshape(-1, r))
    assert got["found"] == want["W"].shape[0] and got["verified"] == got["found"]


def _left_product(m: dict, w: np.ndarray, p: int) -> np.ndarray:
    """w^T A mod p from the exported CSR (Python integers: exact for any p)."""
    rp, col, val = m["row_ptr"].astype(np.int64), m["col"].astype(np.int64), m["val"].astype(object)
    lens = np.diff(rp)
    coef = np.repeat(np.array([int(x) for x in w], dtype=object), lens)
    out = np.zeros(m["dict_exps"].shape[0], dtype=object)
    np.add.at(out, col, coef * val)
    return np.array([int(x) % p for x in out], dtype=np.int64)


@pytest.mark.parametrize("system,step,b", [(synth.dense_n10(0), 6, 32), (synth.sparse_n13(0), 4, 16)],
                         ids=["dense_n10_step6_b32", "sparse_n13_step4_b16"])
def test_kernel_vectors_at_size(ctx, system, step, b):
    S, mac, stats = gpu_step(ctx, system, step)
    m = gb.gb_macaulay_export(mac)
    p = system["p"]
    r, N = len(m["row_ptr"]) - 1, m["dict_exps"].shape[0]
    X, Z, delta = random_inputs(r, N, b, p, 5)
    got = gb.gb_block_wiedemann(mac, b, np.array(X), np.array(Z), np.array(delta), want_seq=False)
    S.close()
    nullity = stats["nC"] - stats["rank"]
    assert got["found"] == min(b, nullity) > 0
    assert got["verified"] == got["found"]
    for w in got["W"][:3]:
        assert w.any() and not _left_product(m, w, p).any()


def test_rejected_arguments(ctx):
    S, mac, _ = gpu_step(ctx, synth.dense_n6(0), 3)
    m = gb.gb_macaulay_export(mac)
    r, N = len(m["row_ptr"]) - 1, m["dict_exps"].shape[0]
    for b in (0, 33):
        with pytest.raises(gb.GbError):
            gb.gb_block_wiedemann(mac, b, np.zeros((r, max(b, 1)), np.uint32), np.zeros((r, max(b, 1)), np.uint32),
                                  np.ones(N, np.uint32))
    with pytest.raises(gb.GbError):  # delta must be non-zero
        gb.gb_block_wiedemann(mac, 4, np.zeros((r, 4), np.uint32), np.zeros((r, 4), np.uint32), np.zeros(N, np.uint32))
    S.close()
