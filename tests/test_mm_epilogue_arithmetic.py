"""The integer arithmetic of the tensor-core product's epilogue (csrc/mm.cu), modelled with exact
Python integers: every intermediate stays in the range the kernel's types give it, and the result
is (C -/+ sum_s D_s 256^s) mod p.

The kernel receives, per output, the FP32 digit-diagonal sums D_s (|D_s| <= c_s K 2^14 with c_s
products per K step, K <= 512 / L) and C in [0, p).  It pairs adjacent small diagonals in 32 bits,
sums signed 32 x 32 -> 64-bit products with the multipliers rd[s] = (-/+ 256^s mod p) 2^32 mod p
on top of a bias 2^31 p, applies one Montgomery reduction (R = 2^32) and two corrections.  This
test checks that model at the extreme diagonal values (every digit product +-2^14) and on random
ones, for primes at both ends of each digit count; the device kernel itself is checked against
int64 products in tests/test_gpu_matmul.py.
"""
from __future__ import annotations

import random

import pytest

I32 = (-(2 ** 31), 2 ** 31 - 1)
I64 = (-(2 ** 63), 2 ** 63 - 1)


def digits(p: int) -> int:
    return 2 if p < 65536 else 4


def diag_bounds(L: int) -> list[int]:
    """Largest |D_s| at the longest K of one launch: c_s products of magnitude <= 2^14 per step."""
    K = 512 // L
    return [min(s + 1, 2 * L - 1 - s) * K * 2 ** 14 for s in range(2 * L - 1)]


def epilogue(p: int, D: list[int], c: int, sub: bool) -> int:
    """The kernel's steps for one output; asserts every range on the way."""
    L = digits(p)
    R = 2 ** 32
    pinv_neg = (-pow(p, -1, R)) % R
    rd = []
    for s in range(7):
        x = pow(256, s, p)
        y = p - x if sub and x else x
        rd.append((y << 32) % p)
    big = p << 31
    if L == 4:
        e0, e5 = D[0] + 256 * D[1], D[5] + 256 * D[6]
        for e in (e0, e5):
            assert I32[0] <= e <= I32[1]
        terms = [(e0, rd[0]), (D[2], rd[2]), (D[3], rd[3]), (D[4], rd[4]), (e5, rd[5])]
    else:
        e1 = D[1] + 256 * D[2]
        assert I32[0] <= e1 <= I32[1]
        terms = [(D[0], rd[0]), (e1, rd[1])]
    acc = big
    for x, r in terms:
        assert I32[0] <= x <= I32[1] and 0 <= r < 2 ** 31  # signed 32 x 32 -> 64
        acc += x * r
        assert I64[0] <= acc <= I64[1]
    assert 0 < acc < R * p  # the range of one Montgomery reduction
    m = (acc % R) * pinv_neg % R
    t = acc + m * p
    assert t < 2 ** 64 and t % R == 0
    u = t >> 32
    assert u < 2 * p
    u = min(u, (u - p) % R)  # "u - p if u >= p" as min(u, u - p) in 32-bit unsigned arithmetic
    assert u < p
    s = c + u
    assert s < 2 ** 32
    return min(s, (s - p) % R)


PRIMES = [3, 257, 32749, 65521, 65537, 1000003, 2 ** 31 - 19, 2 ** 31 - 1]


@pytest.mark.parametrize("p", PRIMES)
@pytest.mark.parametrize("sub", [False, True], ids=["add", "sub"])
def test_extremes_and_random_diagonals(p, sub):
    L = digits(p)
    B = diag_bounds(L)
    rng = random.Random(p * 2 + sub)
    cases = [[sgn * b for b in B] for sgn in (1, -1)]
    cases += [[rng.choice((-1, 1)) * b for b in B] for _ in range(64)]
    cases += [[rng.randint(-b, b) for b in B] for _ in range(512)]
    for D in cases:
        D = D + [0] * (7 - len(D))
        for c in (0, 1, p - 1, rng.randrange(p)):
            value = sum(D[s] * 256 ** s for s in range(2 * L - 1))
            want = (c - value) % p if sub else (c + value) % p
            assert epilogue(p, D, c, sub) == want


def test_the_pairings_fit_and_wider_groups_do_not():
    """At K = 512 / L the pairs the kernel forms fit 32 bits; the pair of diagonals 2 and 3 of
    L = 4, the pair 0, 1 of L = 2 and any three adjacent diagonals do not."""
    B4, B2 = diag_bounds(4), diag_bounds(2)
    pair = lambda B, s: B[s] + 256 * B[s + 1]
    assert pair(B4, 0) < 2 ** 31 and pair(B4, 5) < 2 ** 31 and pair(B2, 1) < 2 ** 31
    assert pair(B4, 2) >= 2 ** 31 and pair(B2, 0) >= 2 ** 31
    assert all(B4[s] + 256 * B4[s + 1] + 65536 * B4[s + 2] >= 2 ** 31 for s in range(5))
    # the diagonals converted through the 1.5 2^23 bias are those within 2^22
    assert [b <= 2 ** 22 for b in B4] == [True, True, False, False, False, True, True]
    assert [b <= 2 ** 22 for b in B2] == [True, False, True]
    # and every partial sum is an integer FP32 holds exactly
    assert max(B4) <= 2 ** 23 and max(B2) <= 2 ** 23
