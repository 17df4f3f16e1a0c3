"""Seeded synthetic polynomial systems over F_p.

The paper's third benchmark family is "dense random quadratic systems over F_p" (§12.3).  This
module draws such systems, and the sparse, mixed-degree and multi-prime variants used by the
batched and served workloads, from a counter-free SplitMix64 stream (Steele, Lea and Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014).

It holds no arithmetic of the F4 method: it only emits terms (exponent vector, coefficient) in
generation order.  Normalisation (merging, sorting, making monic) belongs to whoever consumes the
system.  Both the CUDA path and the CPU oracle read systems produced here.

A system is a dict::

    {"n": nvars, "p": prime, "m": npolys,
     "poly_off": uint32[m+1],   # term range of polynomial i is [poly_off[i], poly_off[i+1])
     "exps": uint8[T, n],       # exponent vectors, row-major
     "coeffs": uint32[T]}       # coefficients in [1, p-1] (0 allowed only after reduction mod p)
"""
from __future__ import annotations

import math

import numpy as np

MASK64 = (1 << 64) - 1
BASE_SEED = 20260765
P16 = 65521
P31 = 2147483647


class SplitMix64:
    """SplitMix64 as published by Steele, Lea and Flood (2014), constants from that paper."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def below(self, bound: int) -> int:
        """Uniform integer in [0, bound) by rejection (no modulo bias)."""
        if bound <= 0:
            raise ValueError("bound must be positive")
        limit = ((1 << 64) // bound) * bound
        while True:
            x = self.next()
            if x < limit:
                return x % bound

    def between(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi]."""
        return lo + self.below(hi - lo + 1)


def monomials_upto(n: int, d: int) -> list[tuple[int, ...]]:
    """All exponent vectors in n variables of total degree <= d, degree by degree; within a degree,
    exponent tuples in descending lexicographic order.  This is only an enumeration order for
    drawing supports, not a term order."""
    out: list[tuple[int, ...]] = []

    def comps(k: int, total: int):
        if k == 1:
            yield (total,)
            return
        for first in range(total, -1, -1):
            for rest in comps(k - 1, total - first):
                yield (first,) + rest

    for deg in range(d + 1):
        out.extend(comps(n, deg))
    return out


def _pack(n: int, p: int, polys: list[list[tuple[tuple[int, ...], int]]]) -> dict:
    off = [0]
    exps: list[tuple[int, ...]] = []
    coeffs: list[int] = []
    for f in polys:
        for e, c in f:
            exps.append(e)
            coeffs.append(c)
        off.append(len(exps))
    return {
        "n": n,
        "p": p,
        "m": len(polys),
        "poly_off": np.asarray(off, dtype=np.uint32),
        "exps": np.asarray(exps, dtype=np.uint8).reshape(-1, n),
        "coeffs": np.asarray(coeffs, dtype=np.uint32),
    }


def dense_system(n: int, m: int, p: int, seed: int, degree: int = 2) -> dict:
    """Every monomial of degree <= `degree` in every polynomial, coefficients uniform in [1, p-1]."""
    rng = SplitMix64(seed)
    mons = monomials_upto(n, degree)
    polys = [[(e, rng.between(1, p - 1)) for e in mons] for _ in range(m)]
    return _pack(n, p, polys)


def sparse_system(n: int, m: int, p: int, seed: int, terms: int | tuple[int, int],
                  degree: int = 2, nvars_seed_draw: bool = False) -> dict:
    """Each polynomial: `terms` distinct monomials drawn uniformly without replacement from the
    monomials of degree <= `degree` (redrawn until one has degree exactly `degree`), coefficients
    uniform in [1, p-1].  `terms` may be a (lo, hi) range drawn per polynomial; it is clamped to the
    number of available monomials."""
    rng = SplitMix64(seed)
    mons = monomials_upto(n, degree)
    polys = []
    for _ in range(m):
        k = terms if isinstance(terms, int) else rng.between(terms[0], terms[1])
        k = min(k, len(mons))
        while True:
            idx = list(range(len(mons)))
            for i in range(k):  # partial Fisher-Yates
                j = i + rng.below(len(mons) - i)
                idx[i], idx[j] = idx[j], idx[i]
            pick = idx[:k]
            if any(sum(mons[i]) == degree for i in pick):
                break
        polys.append([(mons[i], rng.between(1, p - 1)) for i in pick])
    return _pack(n, p, polys)


def homogeneous_system(n: int, m: int, p: int, seed: int, degree: int | list[int] = 2) -> dict:
    """Every monomial of degree exactly d_i in polynomial i (d_i = `degree`, or the i-th entry of
    a list of degrees), coefficients uniform in [1, p-1]: a homogeneous system, a regular sequence
    with high probability when m <= n."""
    rng = SplitMix64(seed)
    degs = [degree] * m if isinstance(degree, int) else list(degree)
    polys = []
    for i in range(m):
        mons = [e for e in monomials_upto(n, degs[i]) if sum(e) == degs[i]]
        polys.append([(e, rng.between(1, p - 1)) for e in mons])
    return _pack(n, p, polys)


def homogenize(system: dict) -> dict:
    """The system in n + 1 variables with every term of polynomial i raised to its degree by the
    new last variable (the smallest one in grevlex): term x^a of a degree-D polynomial becomes
    x^a h^(D - |a|)."""
    n, p = int(system["n"]), int(system["p"])
    polys = []
    for i in range(int(system["m"])):
        lo, hi = int(system["poly_off"][i]), int(system["poly_off"][i + 1])
        exps = [tuple(int(x) for x in system["exps"][q][:n]) for q in range(lo, hi)]
        if not exps:
            polys.append([])
            continue
        top = max(sum(e) for e in exps)
        polys.append([(e + (top - sum(e),), int(system["coeffs"][q])) for e, q in zip(exps, range(lo, hi))])
    return _pack(n + 1, p, polys)


# ---- the five workloads ---------------------------------------------------------------------

def dense_n6(seed_index: int = 0) -> dict:
    """n=6, m=6, all 28 monomials of degree <= 2, p=65521."""
    return dense_system(6, 6, P16, BASE_SEED + seed_index)


def dense_n10(seed_index: int = 0) -> dict:
    """n=10, m=10, all 66 monomials of degree <= 2, p=65521."""
    return dense_system(10, 10, P16, BASE_SEED + seed_index)


def sparse_n13(seed_index: int = 0) -> dict:
    """n=13, m=13, 30 of the 105 monomials of degree <= 2 per polynomial, p=2^31-1."""
    return sparse_system(13, 13, P31, BASE_SEED + seed_index, 30)


def mixed_batch(count: int = 256, seed_index: int = 0) -> list[dict]:
    """Independent systems: n ~ U{5..9}, m = n, degree ~ U{2,3}, terms ~ U{10..40} (clamped),
    p = 65521.  System i is drawn from seed BASE_SEED + seed_index + i."""
    out = []
    for i in range(count):
        rng = SplitMix64(BASE_SEED + seed_index + i)
        n = rng.between(5, 9)
        deg = rng.between(2, 3)
        sub_seed = rng.next()
        out.append(sparse_system(n, n, P16, sub_seed, (10, 40), degree=deg))
    return out


def is_prime_trial(q: int) -> bool:
    """Plain trial division (inputs < 2^32 only)."""
    if q < 2:
        return False
    if q % 2 == 0:
        return q == 2
    r = math.isqrt(q)
    f = 3
    while f <= r:
        if q % f == 0:
            return False
        f += 2
    return True


def largest_primes_below(bound: int, count: int) -> list[int]:
    out = []
    q = bound - 1
    while len(out) < count:
        if is_prime_trial(q):
            out.append(q)
        q -= 1
    return out


def multi_prime_system(primes: list[int], seed_index: int = 0, n: int = 8) -> list[dict]:
    """One dense quadratic system (n=8: 45 monomials per polynomial) whose integer coefficients are
    drawn once in [1, 2^31-2] and reduced modulo each prime."""
    rng = SplitMix64(BASE_SEED + 1000 + seed_index)
    mons = monomials_upto(n, 2)
    ints = [[rng.between(1, P31 - 1) for _ in mons] for _ in range(n)]
    out = []
    for p in primes:
        polys = [[(e, c % p) for e, c in zip(mons, row)] for row in ints]
        out.append(_pack(n, p, polys))
    return out


def served_request(index: int, seed_index: int = 0) -> dict:
    """Request `index` of the served stream: n ~ U{5..11}, m = n, quadratic,
    terms ~ U{20..66} (clamped), p = 65521 or 2^31-1 with probability 1/2 each."""
    rng = SplitMix64(BASE_SEED + 5000 + seed_index * 100003 + index)
    n = rng.between(5, 11)
    p = P16 if rng.below(2) == 0 else P31
    return sparse_system(n, n, p, rng.next(), (20, 66), degree=2)


def poisson_arrivals(count: int, rate: float, seed_index: int = 0) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process with the given rate (exponential gaps drawn by
    inversion of a 53-bit uniform)."""
    rng = SplitMix64(BASE_SEED + 7000 + seed_index)
    t = 0.0
    out = np.empty(count, dtype=np.float64)
    for i in range(count):
        u = ((rng.next() >> 11) + 1) * (1.0 / 9007199254740993.0)  # (0, 1]
        t += -math.log(u) / rate
        out[i] = t
    return out
