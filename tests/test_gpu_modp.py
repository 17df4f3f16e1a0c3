"""The device F_p primitives, each on its own, against plain integer arithmetic (numpy uint64 and
Python integers): Barrett reduction with k = 64 and k = 32 (Sec. 8.3), the modular multiply-add
(Sec. 8.1), Montgomery reduction, domain conversion and the Montgomery product of the sparse
update (Sec. 8.4), both inverses, and the lazy accumulation windows of Rem. 8.1 at their largest
window.  Exhaustive for every odd prime below 256, the boundary values 0, 1, p - 1, (p - 1)^2 and
the top of each input range, and 10^6 random triples for each of the 128 largest primes below
2^31, 65521 and 2^31 - 1.  gb_modp_apply runs the same device functions, with the same constants,
as the reduction kernels."""
from __future__ import annotations

import numpy as np
import pytest

import paper_2601_06765_b300 as gb
from paper_2601_06765_b300 import synth

pytestmark = pytest.mark.gpu

R = 1 << 32
SMALL_PRIMES = [q for q in range(3, 256) if synth.is_prime_trial(q)]
BIG_PRIMES = synth.largest_primes_below(1 << 31, 128)


def _dev(torch, a):
    a = np.ascontiguousarray(a, dtype=np.uint32)
    return torch.from_numpy(a.view(np.int32)).cuda()


def _apply(torch, op, p, a, b=None, c=None, window=0):
    n = len(a) // window if window else len(a)
    A = _dev(torch, a)
    B = _dev(torch, b) if b is not None else None
    C = _dev(torch, c) if c is not None else None
    out = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    gb.gb_modp_apply(op, p, n, window, A.data_ptr(), B.data_ptr() if B is not None else None,
                     C.data_ptr() if C is not None else None, out.data_ptr(),
                     torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32)[:n].astype(np.uint64)


def _u64(x):
    return np.asarray(x, dtype=np.uint64)


def _check_all_ops(torch, p, a, b, c):
    """a, b, c: uint64 arrays of residues in [0, p) (a > 0 where an inverse is taken)."""
    P = np.uint64(p)
    # Barrett, 64-bit input: x = a 2^32 + b spans all high words below p
    got = _apply(torch, gb.GB_MODP_REDUCE64, p, a, b)
    assert np.array_equal(got, ((a << np.uint64(32)) | b) % P)
    got = _apply(torch, gb.GB_MODP_MULADD, p, a, b, c)
    assert np.array_equal(got, (a * b + c) % P)
    # Montgomery: redc(t) for t = a 2^32 + b < p 2^32 is t R^-1 mod p, below 2p
    rinv = np.uint64(pow(R, -1, p))
    got = _apply(torch, gb.GB_MODP_REDC, p, a, b)
    t_mod = ((a << np.uint64(32)) | b) % P
    assert (got < 2 * P).all() and np.array_equal(got % P, (t_mod * rinv) % P)
    got = _apply(torch, gb.GB_MODP_TO_MONT, p, a)
    assert np.array_equal(got, (a << np.uint64(32)) % P)
    got = _apply(torch, gb.GB_MODP_MONT_MUL, p, a, b)
    assert (got < 2 * P).all() and np.array_equal(got % P, (a * b) % P)
    nz = a[a > 0]
    got = _apply(torch, gb.GB_MODP_INV, p, nz)
    assert (got < P).all() and ((got * nz) % P == 1).all()
    if p < 65536:
        got = _apply(torch, gb.GB_MODP_INV_SMALL, p, nz)
        assert (got < P).all() and ((got * nz) % P == 1).all()


@pytest.mark.parametrize("p", SMALL_PRIMES)
def test_every_residue_pair_for_primes_below_256(p):
    import torch
    r = np.arange(p, dtype=np.uint64)
    a = np.repeat(r, p)
    b = np.tile(r, p)
    c = (a * np.uint64(7) + b) % np.uint64(p)
    _check_all_ops(torch, p, a, b, c)
    # 32-bit Barrett over every 16-bit input and the top of the 32-bit range
    x = np.concatenate([np.arange(1 << 16, dtype=np.uint64),
                        np.arange((1 << 32) - (1 << 16), 1 << 32, dtype=np.uint64)])
    assert np.array_equal(_apply(torch, gb.GB_MODP_REDUCE32, p, x), x % np.uint64(p))


@pytest.mark.parametrize("p", [3, 7, 251, 65519, 65521, 2147483629, 2147483647])
def test_boundary_values(p):
    import torch
    P = np.uint64(p)
    edge = _u64([0, 1, 2, p - 2, p - 1, p // 2, (p + 1) // 2])
    a = np.repeat(edge, len(edge))
    b = np.tile(edge, len(edge))
    _check_all_ops(torch, p, a, b, b[::-1].copy())
    # the top of every input range: x = 2^64 - 1, (p - 1)^2, t = p 2^32 - 1
    hi = _u64([0xFFFFFFFF, p - 1, p - 1, 0])
    lo = _u64([0xFFFFFFFF, 0xFFFFFFFF, 0, 0])
    x = (hi << np.uint64(32)) | lo
    assert np.array_equal(_apply(torch, gb.GB_MODP_REDUCE64, p, hi, lo), x % P)
    sq = _u64([(p - 1) * (p - 1)])
    assert np.array_equal(_apply(torch, gb.GB_MODP_REDUCE64, p, sq >> np.uint64(32), sq & np.uint64(R - 1)),
                          sq % P)
    got = _apply(torch, gb.GB_MODP_REDC, p, _u64([p - 1]), _u64([R - 1]))
    assert got[0] < 2 * p and int(got[0]) % p == ((p * R - 1) * pow(R, -1, p)) % p
    full = _u64([0xFFFFFFFF, 0xFFFFFFFF, 0])
    assert np.array_equal(_apply(torch, gb.GB_MODP_MULADD, p, full, full, full),
                          _u64([(0xFFFFFFFF ** 2 + 0xFFFFFFFF) % p, (0xFFFFFFFF ** 2 + 0xFFFFFFFF) % p, 0]))
    if p < 65536:
        x32 = _u64([0, 1, p - 1, p, (p - 1) ** 2, 0xFFFFFFFF])
        assert np.array_equal(_apply(torch, gb.GB_MODP_REDUCE32, p, x32), x32 % P)


@pytest.mark.parametrize("group", range(8))
def test_random_triples_for_the_128_primes(group):
    """10^6 random (a, b, c) for each prime; 16 primes per test case."""
    import torch
    primes = BIG_PRIMES[16 * group:16 * group + 16]
    if group == 0:
        primes = primes + [65521, 2147483647]
    rng = np.random.default_rng(20260765 + group)
    for p in primes:
        a, b, c = (rng.integers(0, p, 10 ** 6, dtype=np.uint64) for _ in range(3))
        a[0] = max(a[0], 1)
        _check_all_ops(torch, p, a, b, c)


@pytest.mark.parametrize("p", [65521, 65519, 251, 7])
def test_lazy_32_bit_window_at_its_limit(p):
    """Rem. 8.1: reduced products summed in 32 bits without reduction in between are exact while
    fewer than 2^16 of them meet one column (the host's bound for the 32-bit accumulator); the
    worst case p - 1 at every term with a start residue of p - 1 included."""
    import torch
    w = (1 << 16) - 1
    P = np.uint64(p)
    rng = np.random.default_rng(p)
    a = np.concatenate([np.full(w, p - 1, np.uint64), rng.integers(0, p, 3 * w, dtype=np.uint64)])
    b = np.concatenate([np.full(w, p - 1, np.uint64), rng.integers(0, p, 3 * w, dtype=np.uint64)])
    c = _u64([p - 1, 0, 1, rng.integers(0, p)])
    want = (c + ((a * b) % P).reshape(4, w).sum(axis=1, dtype=np.uint64)) % P
    assert np.array_equal(_apply(torch, gb.GB_MODP_LAZY32, p, a, b, c, window=w), want)


@pytest.mark.parametrize("p", [2147483647, 2147483629, 65521])
def test_lazy_montgomery_window(p):
    """The 64-bit sum of Montgomery products (each below 2p) of the 31-bit sparse update, reduced
    once: exact for any window a 64-bit sum holds; windows of 2^20 worst-case terms checked."""
    import torch
    w = 1 << 20
    P = np.uint64(p)
    rng = np.random.default_rng(p + 1)
    a = np.concatenate([np.full(w, p - 1, np.uint64), rng.integers(0, p, w, dtype=np.uint64)])
    b = np.concatenate([np.full(w, p - 1, np.uint64), rng.integers(0, p, w, dtype=np.uint64)])
    c = _u64([p - 1, rng.integers(0, p)])
    prod = (a * b) % P
    want = (c + prod.reshape(2, w).sum(axis=1, dtype=np.uint64) % P) % P
    assert np.array_equal(_apply(torch, gb.GB_MODP_LAZY_MONT, p, a, b, c, window=w), want)


def test_rejected_arguments():
    with pytest.raises(gb.GbError):
        gb.gb_modp_apply(gb.GB_MODP_REDUCE32, 2147483647, 1, 0, 1, None, None, 1)
    with pytest.raises(gb.GbError):
        gb.gb_modp_apply(gb.GB_MODP_MULADD, 65535, 1, 0, 1, 1, 1, 1)
    with pytest.raises(gb.GbError):
        gb.gb_modp_apply(gb.GB_MODP_LAZY32, 65521, 1, 1 << 16, 1, 1, 1, 1)
    with pytest.raises(gb.GbError):
        gb.gb_modp_apply(42, 65521, 1, 0, 1, 1, 1, 1)


def _chain(torch, op, p, a, b, c, steps):
    A, B, C = _dev(torch, a), _dev(torch, b), _dev(torch, c)
    out = torch.empty(len(a), dtype=torch.int32, device="cuda")
    gb.gb_modp_apply(op, p, len(a), steps, A.data_ptr(), B.data_ptr(), C.data_ptr(), out.data_ptr(),
                     torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return [int(x) for x in out.cpu().numpy().view(np.uint32)]


def _chain_closed_form(a, b, c, w, p):
    """x_w of x <- x b + c from x_0 = a: a b^w + c (b^w - 1) / (b - 1), or a + c w when b = 1."""
    bw = pow(b, w, p)
    if b % p == 1:
        return (a + c * w) % p
    return (a * bw + c * (bw - 1) * pow(b - 1, -1, p)) % p


@pytest.mark.parametrize("p", [3, 251, 65521, 2147483647] + BIG_PRIMES[:4])
@pytest.mark.parametrize("steps", [1, 7, 1000])
def test_multiply_add_chains_against_the_geometric_sum(p, steps):
    """The register chains of the inner-loop microbenchmark, Barrett and Montgomery, against the
    closed form of the recurrence (and therefore against each other), including b = 0, 1, p - 1
    and residues at the top of the range."""
    import torch
    rng = np.random.default_rng(p * 31 + steps)
    n = 4096
    a = rng.integers(0, p, n, dtype=np.uint64)
    b = rng.integers(0, p, n, dtype=np.uint64)
    c = rng.integers(0, p, n, dtype=np.uint64)
    a[:6], b[:6], c[:6] = [p - 1] * 6, [0, 1, p - 1, p - 1, 1, 0], [p - 1, p - 1, p - 1, 0, 0, 0]
    want = [_chain_closed_form(int(x), int(y), int(z), steps, p) for x, y, z in zip(a, b, c)]
    for op in (gb.GB_MODP_CHAIN_BARRETT, gb.GB_MODP_CHAIN_MONT):
        assert _chain(torch, op, p, a, b, c, steps) == want, op


def test_chain_needs_a_step():
    with pytest.raises(gb.GbError):
        gb.gb_modp_apply(gb.GB_MODP_CHAIN_BARRETT, 65521, 1, 0, 1, 1, 1, 1)
