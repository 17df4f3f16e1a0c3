"""Batched and served F4: every result equals the same system's result alone and the oracle's.

gb_batch_groebner runs many independent systems in lockstep (each kernel launch covers the rows of
every system that takes a step); gb_server admits submitted systems between lockstep iterations
under an HBM cap while others run (continuous batching).  Exactness means the mix changes nothing:
the reduced bases are bit-identical."""
from __future__ import annotations

import time

import pytest

import oracle
import paper_2601_06765_b300 as gb
from paper_2601_06765_b300 import synth

pytestmark = pytest.mark.gpu

MIXED_SMALL = (1, 3, 0, 14, 18, 9, 13, 33)  # quadratic n = 5..8 and one n = 5 cubic member


@pytest.fixture(scope="module")
def ctx():
    c = gb.Context(arena_bytes=8 << 30)
    yield c
    c.close()


def _workload():
    mixed = synth.mixed_batch(256)
    primes = synth.largest_primes_below(2 ** 31, 128)
    return [mixed[i] for i in MIXED_SMALL] + synth.multi_prime_system([primes[0], primes[1], primes[127]])


def _alone(ctx, system):
    with gb.System(ctx, system) as S:
        S.groebner()
        return S.basis()


def test_batch_equals_alone_and_oracle(ctx):
    systems = _workload()
    alone = [_alone(ctx, s) for s in systems]
    handles = [gb.gb_system_create(ctx.h, s) for s in systems]
    try:
        stats = gb.gb_batch_groebner(ctx.h, handles)
        for h, s, a, st in zip(handles, systems, alone, stats):
            got = gb.basis_terms(*gb.gb_basis_export(h, s["n"], True))
            assert got == a
            assert st["nbasis"] == len(a) and st["steps"] > 0
    finally:
        for h in handles:
            gb.gb_system_destroy(h)
    for s, a in zip(systems[:5] + systems[-1:], alone[:5] + alone[-1:]):
        assert a == oracle.groebner(s)


def test_batch_of_one_and_of_none(ctx):
    assert gb.gb_batch_groebner(ctx.h, []) == []
    s = synth.dense_n6(4)
    h = gb.gb_system_create(ctx.h, s)
    try:
        gb.gb_batch_groebner(ctx.h, [h])
        assert gb.basis_terms(*gb.gb_basis_export(h, s["n"], True)) == oracle.groebner(s)
    finally:
        gb.gb_system_destroy(h)


def _serve_loop(ctx, systems, cap_bytes, slots, stagger_s):
    """Submit with gaps, poll continuously; returns the reduced bases in submission order."""
    srv = gb.gb_server_create(ctx.h, cap_bytes, slots)
    pending = {}
    results = {}

    def drain():
        for t in list(pending):
            h, st = gb.gb_server_poll(srv, t)
            if h is None:
                continue
            assert st == gb.GB_OK
            i = pending.pop(t)
            results[i] = gb.basis_terms(*gb.gb_basis_export(h, systems[i]["n"], True))
            gb.gb_system_destroy(h)

    try:
        for i, s in enumerate(systems):
            pending[gb.gb_server_submit(srv, gb.gb_system_create(ctx.h, s))] = i
            if stagger_s:
                time.sleep(stagger_s)
            drain()
        deadline = time.time() + 300
        while pending and time.time() < deadline:
            drain()
            time.sleep(0.002)
        assert not pending, "requests did not finish"
    finally:
        gb.gb_server_destroy(srv)
    return [results[i] for i in range(len(systems))]


def test_served_results_equal_alone(ctx):
    """Continuous batching: requests arrive while others run (staggered submits, 4 slots); each
    result is the same as the system's result alone."""
    systems = [synth.served_request(i) for i in range(12)]
    alone = [_alone(ctx, s) for s in systems]
    served = _serve_loop(ctx, systems, cap_bytes=4 << 30, slots=4, stagger_s=0.003)
    assert served == alone
    for i in (0, 1, 3):  # n <= 9: the oracle finishes in seconds
        assert alone[i] == oracle.groebner(systems[i])


def test_server_admission_under_a_tight_cap(ctx):
    """A cap below one system's footprint admits one request at a time; all still finish."""
    systems = [synth.served_request(100 + i) for i in range(5)]
    alone = [_alone(ctx, s) for s in systems]
    assert _serve_loop(ctx, systems, cap_bytes=1, slots=4, stagger_s=0) == alone


def test_server_poll_reports_busy_and_unknown(ctx):
    srv = gb.gb_server_create(ctx.h, 4 << 30, 2)
    try:
        s = synth.dense_n10(0)
        t = gb.gb_server_submit(srv, gb.gb_system_create(ctx.h, s))
        h, st = gb.gb_server_poll(srv, t)
        if h is None:
            assert st == -7  # GB_EBUSY while the request runs
        deadline = time.time() + 120
        while h is None and time.time() < deadline:
            time.sleep(0.005)
            h, st = gb.gb_server_poll(srv, t)
        assert h is not None and st == gb.GB_OK
        gb.gb_system_destroy(h)
        with pytest.raises(gb.GbError):
            gb.gb_server_poll(srv, 987654321)
    finally:
        gb.gb_server_destroy(srv)


def test_cubic_n8_member_in_a_batch():
    """A cubic member with eight variables (mixed batch index 47; its steps reach degree 19 and
    10^8 nonzeros): its first five F4 steps equal the oracle's step for step, and its reduced
    basis is the same alone and inside a batch with two small members."""
    from tests.test_gpu_parity import run_parity
    mixed = synth.mixed_batch(256)
    cubic = mixed[47]
    assert cubic["n"] == 8 and int(cubic["exps"].reshape(-1, 8).sum(axis=1).max()) == 3
    with gb.Context(arena_bytes=16 << 30, keep_step=True) as c:
        assert run_parity(c, cubic, max_steps=5, final=False) == 5
    with gb.Context(arena_bytes=16 << 30) as c:
        alone = _alone(c, cubic)
        systems = [cubic, mixed[1], mixed[3]]
        handles = [gb.gb_system_create(c.h, s) for s in systems]
        try:
            gb.gb_batch_groebner(c.h, handles)
            assert gb.basis_terms(*gb.gb_basis_export(handles[0], 8, True)) == alone
            for h, s in zip(handles[1:], systems[1:]):
                assert gb.basis_terms(*gb.gb_basis_export(h, s["n"], True)) == oracle.groebner(s)
        finally:
            for h in handles:
                gb.gb_system_destroy(h)
