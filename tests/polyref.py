"""Plain-Python polynomial arithmetic over F_p used only to pin the oracle.

Written independently of both the oracle and the CUDA path.  Polynomials are dicts
{exponent tuple: coefficient in [0, p)}; the term order is sympy's own `grevlex` monomial key
(x1 > x2 > ... > xn), a library routine.
"""
from __future__ import annotations

import itertools

import numpy as np
from sympy.polys.orderings import grevlex


def system_polys(system: dict) -> list[dict]:
    """The input system as dict polynomials (duplicates merged, zeros dropped)."""
    p, n = system["p"], system["n"]
    out = []
    for i in range(system["m"]):
        f: dict = {}
        for j in range(int(system["poly_off"][i]), int(system["poly_off"][i + 1])):
            e = tuple(int(x) for x in system["exps"][j][:n])
            f[e] = (f.get(e, 0) + int(system["coeffs"][j])) % p
        out.append({e: c for e, c in f.items() if c})
    return out


def terms_to_dict(terms) -> dict:
    return {tuple(e): int(c) for e, c in terms}


def lm(f: dict):
    return max(f, key=grevlex)


def divides(a, b) -> bool:
    return all(x <= y for x, y in zip(a, b))


def mono_mul(a, b):
    return tuple(x + y for x, y in zip(a, b))


def mono_div(b, a):
    return tuple(y - x for x, y in zip(a, b))


def lcm(a, b):
    return tuple(max(x, y) for x, y in zip(a, b))


def axpy(f: dict, c: int, t, g: dict, p: int) -> dict:
    """f + c * t * g."""
    h = dict(f)
    for e, v in g.items():
        m = mono_mul(t, e)
        w = (h.get(m, 0) + c * v) % p
        if w:
            h[m] = w
        else:
            h.pop(m, None)
    return h


def spoly(f: dict, g: dict, p: int) -> dict:
    lf, lg = lm(f), lm(g)
    L = lcm(lf, lg)
    a = pow(f[lf], p - 2, p)
    b = pow(g[lg], p - 2, p)
    h = axpy({}, a, mono_div(L, lf), f, p)
    return axpy(h, (p - b) % p, mono_div(L, lg), g, p)


def remainder(f: dict, G: list[dict], p: int) -> dict:
    """Multivariate division of f by G (Cox-Little-O'Shea, Thm. 2.3.3): the remainder."""
    f = dict(f)
    r: dict = {}
    lms = [(lm(g), g) for g in G if g]
    while f:
        m = lm(f)
        c = f[m]
        for lg, g in lms:
            if divides(lg, m):
                f = axpy(f, (p - c * pow(g[lg], p - 2, p)) % p, mono_div(m, lg), g, p)
                break
        else:
            r[m] = c
            del f[m]
    return r


def is_groebner(G: list[dict], p: int) -> bool:
    """Buchberger's criterion: every S-polynomial reduces to 0 modulo G."""
    for i in range(len(G)):
        for j in range(i + 1, len(G)):
            if remainder(spoly(G[i], G[j], p), G, p):
                return False
    return True


def is_reduced(G: list[dict], p: int) -> bool:
    """Monic, and no term of any element divisible by another element's leading monomial."""
    lms = [lm(g) for g in G]
    for i, g in enumerate(G):
        if g[lms[i]] != 1:
            return False
        for e in g:
            for j, l in enumerate(lms):
                if j != i and divides(l, e):
                    return False
    return True


def zeros(F: list[dict], n: int, p: int) -> set:
    """All points of F_p^n where every polynomial of F vanishes (brute force)."""
    pts = np.array(list(itertools.product(range(p), repeat=n)), dtype=np.int64)
    alive = np.ones(len(pts), dtype=bool)
    for f in F:
        v = np.zeros(len(pts), dtype=np.int64)
        for e, c in f.items():
            t = np.full(len(pts), c, dtype=np.int64)
            for i, k in enumerate(e):
                for _ in range(k):
                    t = (t * pts[:, i]) % p
            v = (v + t) % p
        alive &= v == 0
    return {tuple(int(x) for x in pt) for pt in pts[alive]}


def sympy_reduced_gb(system: dict) -> list[list[tuple[tuple[int, ...], int]]]:
    """sympy's reduced Groebner basis over GF(p) in grevlex, as term lists sorted by leading
    monomial descending, coefficients in [0, p)."""
    from sympy import Poly, groebner, symbols
    n, p = system["n"], system["p"]
    X = symbols(f"x1:{n + 1}")
    F = [Poly.from_dict(f, *X, modulus=p).as_expr() for f in system_polys(system) if f]
    if not F:
        return []
    G = groebner(F, *X, modulus=p, order="grevlex")
    out = []
    for g in G.polys:
        terms = [(tuple(int(x) for x in m), int(c) % p) for m, c in g.terms(order="grevlex")]
        out.append(terms)
    out.sort(key=lambda t: grevlex(t[0][0]), reverse=True)
    return out


def mono_deg(a) -> int:
    return sum(a)


def coprime(a, b) -> bool:
    return all(x == 0 or y == 0 for x, y in zip(a, b))


class PairModel:
    """Critical-pair bookkeeping written from the textbook, independently of the oracle: the
    procedure UPDATE of Becker-Weispfenning, *Groebner Bases* (1993) -- the Gebauer-Moeller
    criteria -- and the normal selection strategy (every pair whose lcm has the least degree,
    the "degree-driven" selection of Sec. 3.1 / Sec. 4.2).

    It sees only the leading monomial of each basis element, in the order the elements are
    inserted.  Pairs are (i, j) with i < j (basis indices).  `in_g[i]` is False once element i has
    left G because a newer leading monomial divides its own."""

    def __init__(self):
        self.lms: list[tuple] = []
        self.in_g: list[bool] = []
        self.B: set[tuple[int, int]] = set()

    def insert(self, h_lm: tuple) -> None:
        """UPDATE(G_old, B_old, h): the pairs of h with G_old (visited oldest first) are kept
        when coprime or when no other pair of h -- still waiting, or already kept -- has an lcm
        dividing theirs; the coprime ones are then dropped (product criterion).  An old pair
        {g1, g2} is dropped when LM(h) divides its lcm and that lcm differs from both lcm(g1, h)
        and lcm(g2, h) (chain criterion).  Elements of G_old whose leading monomial LM(h) divides
        leave G."""
        h = len(self.lms)
        g_old = [g for g in range(h) if self.in_g[g]]
        self.lms.append(tuple(h_lm))
        self.in_g.append(True)
        lh = self.lms[h]
        waiting = list(g_old)
        kept: list[int] = []
        while waiting:
            g1 = waiting.pop(0)
            l1 = lcm(lh, self.lms[g1])
            if coprime(lh, self.lms[g1]):
                kept.append(g1)
                continue
            shadowed = any(divides(lcm(lh, self.lms[g2]), l1) for g2 in waiting) or \
                any(divides(lcm(lh, self.lms[g2]), l1) for g2 in kept)
            if not shadowed:
                kept.append(g1)
        new_pairs = {(g, h) for g in kept if not coprime(lh, self.lms[g])}
        survivors = set()
        for g1, g2 in self.B:
            l12 = lcm(self.lms[g1], self.lms[g2])
            if (not divides(lh, l12) or lcm(self.lms[g1], lh) == l12
                    or lcm(self.lms[g2], lh) == l12):
                survivors.add((g1, g2))
        self.B = survivors | new_pairs
        for g in g_old:
            if divides(lh, self.lms[g]):
                self.in_g[g] = False

    def select(self) -> tuple[int, set[tuple[int, int]]]:
        """Normal strategy: remove and return every pair whose lcm has the least degree."""
        d = min(mono_deg(lcm(self.lms[i], self.lms[j])) for i, j in self.B)
        chosen = {q for q in self.B if mono_deg(lcm(self.lms[q[0]], self.lms[q[1]])) == d}
        self.B -= chosen
        return d, chosen

    def pair_rows(self, chosen) -> set[tuple[tuple, int]]:
        """The rows (lcm / LM(g_i), i) and (lcm / LM(g_j), j) of the chosen pairs, as a set: equal
        rows of different pairs are one row of the matrix."""
        rows = set()
        for i, j in chosen:
            L = lcm(self.lms[i], self.lms[j])
            rows.add((mono_div(L, self.lms[i]), i))
            rows.add((mono_div(L, self.lms[j]), j))
        return rows
