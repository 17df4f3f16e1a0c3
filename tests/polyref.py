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
