"""The signature-filtered path (gb_sig_filter, gb_f5_groebner) against the oracle and against
what holds at any size.

- gb_sig_filter: the admissible keys of random and extreme bitmaps, bit for bit against the
  definition (candidate j admissible iff bit j is clear; key (i << 40) | (e << 32) | j).
- gb_f5_groebner on small homogeneous systems: every block's counts, every new basis element and
  the reduced basis equal the oracle's (oracle/f5.py), with and without the criterion.
- At sizes the oracle cannot reach (homogeneous quadratics in 8 variables, the homogenised dense
  n=7 system): every block's rank growth is the Hilbert-series dimension of a regular sequence, no
  admissible row reduces to zero, and the reduced basis equals the one the F4 path computes.
"""
from __future__ import annotations

import numpy as np
import pytest

import paper_2601_06765_b300 as gb
from oracle import f5 as O
from paper_2601_06765_b300 import synth
from tests.test_oracle_f5 import REGULAR, hilbert_ideal_dims

pytestmark = pytest.mark.gpu
P = 65521


@pytest.fixture(scope="module")
def ctx():
    c = gb.Context(arena_bytes=16 << 30)
    yield c
    c.close()


def _filter(ctx, index, e, bits: np.ndarray | None, ncand: int) -> np.ndarray:
    import torch
    keys = torch.zeros(max(ncand, 1), dtype=torch.int64, device="cuda")
    forb = None
    if bits is not None:
        words = np.zeros((ncand + 31) // 32 or 1, dtype=np.uint32)
        for j in np.nonzero(bits)[0]:
            words[j >> 5] |= np.uint32(1) << np.uint32(j & 31)
        forb = torch.from_numpy(words.view(np.int32)).cuda()
    count = gb.gb_sig_filter(ctx.h, index, e, ncand, forb.data_ptr() if forb is not None else None, keys.data_ptr())
    torch.cuda.synchronize()
    return keys[:count].cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("ncand", [0, 1, 31, 32, 33, 1000, 100003])
def test_sig_filter_equals_its_definition(ctx, ncand):
    rng = np.random.default_rng(ncand)
    for index, e, bits in [(1, 0, None), (7, 3, rng.random(ncand) < 0.5), (2 ** 24 - 1, 255, np.ones(ncand, bool)),
                           (3, 9, np.zeros(ncand, bool)), (5, 2, rng.random(ncand) < 0.97)]:
        got = _filter(ctx, index, e, bits, ncand)
        keep = np.arange(ncand) if bits is None else np.nonzero(~bits)[0]
        want = np.array([O.pack_key(index, e, int(j)) for j in keep], dtype=np.uint64)
        assert np.array_equal(got, want), (index, e)


def test_sig_filter_rejects_bad_keys(ctx):
    import torch
    keys = torch.zeros(4, dtype=torch.int64, device="cuda")
    for index, e in ((1 << 24, 0), (1, 256)):
        with pytest.raises(gb.GbError):
            gb.gb_sig_filter(ctx.h, index, e, 4, None, keys.data_ptr())


def _run(ctx, system, dmax, criterion=True):
    with gb.System(ctx, system) as S:
        blocks, stats = S.f5(dmax, criterion)
        running = S.basis(reduced=False)
        reduced = S.basis(reduced=True)
    return blocks, stats, running, reduced


CASES = [(name, s, D) for name, s, D in REGULAR] + [
    ("hq_n5_m4_p31", synth.homogeneous_system(5, 4, 2147483647, 41), 6),
]


@pytest.mark.parametrize("criterion", [True, False], ids=["criterion", "unfiltered"])
@pytest.mark.parametrize("name,system,dmax", CASES, ids=[c[0] for c in CASES])
def test_blocks_elements_and_basis_equal_the_oracle(ctx, name, system, dmax, criterion):
    want = O.f5(system, dmax, criterion=criterion)
    blocks, stats, running, reduced = _run(ctx, system, dmax, criterion)
    assert [(b["degree"], b["index"], b["candidates"], b["admissible"], b["rank"], b["zero_reductions"])
            for b in blocks] == [(w["degree"], w["index"], w["candidates"], w["admissible"], w["new"],
                                  w["zero_reductions"]) for w in want["blocks"]]
    m = len(O.normalised_inputs(system))
    assert running[m:] == want["elements"]
    assert reduced == want["basis"]
    assert stats["zero_reductions"] == sum(w["zero_reductions"] for w in want["blocks"])


def test_non_regular_sequence_equals_the_oracle(ctx):
    s = synth.homogeneous_system(3, 2, P, 31)
    f1 = O.normalised_inputs(s)[0]
    lo, hi = int(s["poly_off"][1]), int(s["poly_off"][2])
    f3 = [(tuple(int(x) for x in s["exps"][q]), int(s["coeffs"][q])) for q in range(lo, hi)]
    system = synth._pack(3, P, [list(f1.items()), [((e[0] + 1,) + e[1:], c) for e, c in f1.items()], f3])
    want = O.f5(system, 6)
    blocks, stats, running, reduced = _run(ctx, system, 6)
    assert stats["zero_reductions"] >= 1
    assert [b["zero_reductions"] for b in blocks] == [w["zero_reductions"] for w in want["blocks"]]
    assert running[3:] == want["elements"] and reduced == want["basis"]


def _f4_basis(ctx, system):
    with gb.System(ctx, system) as S:
        S.groebner()
        return S.basis(reduced=True)


@pytest.mark.parametrize("name,system,dmax", [
    ("hq_n8_m8", synth.homogeneous_system(8, 8, P, 51), 9),
    ("homogenised_dense_n7", synth.homogenize(synth.dense_system(7, 7, P, 52)), 9),
], ids=["hq_n8_m8", "homogenised_dense_n7"])
def test_at_size_hilbert_ranks_no_zero_reductions_and_the_f4_basis(ctx, name, system, dmax):
    blocks, stats, _, reduced = _run(ctx, system, dmax)
    n = int(system["n"])
    degs = [sum(next(iter(f))) for f in O.normalised_inputs(system)]
    H = {i: hilbert_ideal_dims(n, degs[:i], dmax) for i in range(len(degs) + 1)}
    for b in blocks:
        i, d = b["index"], b["degree"]
        assert b["admissible"] - b["zero_reductions"] == H[i][d] - H[i - 1][d], (d, i)
        assert b["zero_reductions"] == 0, (d, i)
    assert stats["candidates"] > stats["admissible"]
    assert reduced == _f4_basis(ctx, system)


def test_rejected_systems(ctx):
    inhom = synth.dense_system(3, 3, P, 61)
    with gb.System(ctx, inhom) as S, pytest.raises(gb.GbError):
        S.f5(4)
    s = synth.homogeneous_system(3, 3, P, 62)
    with gb.System(ctx, s) as S, pytest.raises(gb.GbError):
        S.f5(1)  # below the least input degree
    with gb.System(ctx, s) as S:
        S.step()
        with pytest.raises(gb.GbError):
            S.f5(4)  # a system that has run a step
