"""THE ORACLE for the signature-filtered Macaulay matrices (F5 criterion) -- test infrastructure
only.

Only tests/, the package smoke check and bench.py's CPU-baseline leg may import it; the product
path never does, and it shares no code with the CUDA path.  Dense numpy int64 matrices over F_p
(entries below p < 2^31, so every product fits in 63 bits), for small systems.

What it computes.  The paper states the mechanism (Sec. 14, "GPU-facing reformulation": a packed
signature key per candidate row, the admissibility predicate evaluated over row metadata, the
survivors compacted; Thm. "signature-sound compilation": a sound predicate removes only rows the
admissible ones already span) and leaves the signature discipline open.  The discipline taken
here is the F5 criterion in the degree-by-degree (matrix) form, for a homogeneous system
f_1 .. f_m of degrees d_1 .. d_m, monic, in grevlex (x1 > x2 > ... > xn):

  - signatures are module terms x^a e_i, position over term with e_1 < e_2 < ... < e_m;
  - block (d, i), for d = 1, 2, ..., D and i = 1 .. m with d_i <= d: the candidate rows are
    x^a f_i for every monomial x^a of degree e = d - d_i, taken in descending grevlex order;
    candidate j (the j-th monomial of degree e) has the packed key (i << 40) | (e << 32) | j;
  - Adm(x^a e_i): x^a is not the leading monomial of an element of the degree-e part of
    <f_1 .. f_{i-1}>.  When it is, say LM(h) = x^a with h = sum_{j<i} q_j f_j, the syzygy
    h e_i - f_i sum_j q_j e_j has leading term x^a e_i, so LC(h) x^a f_i equals
    sum_j q_j f_i f_j - (h - LC(h) x^a) f_i: a combination of rows of smaller signature.
    By induction over the signature order the admissible rows span every row of the block;
  - M_{d,i}: the admissible rows of blocks (d, 1 .. i); L_{i,d}: the leading monomials of its row
    space (the pivot columns of RREF(M_{d,i})), the set the criterion reads at degree d + d_{i+1};
  - the block's new elements: the rows of RREF(M_{d,i}) whose leading monomial is not the leading
    monomial of a row of the block (L_{i-1,d}, and x^a LM(f_i) for the admissible x^a), in
    descending order of leading monomial.  These are the reduced echelon rows of the block's
    non-pivot part (the rows of the row space that vanish on those leading columns);
  - the reduced Groebner basis up to degree D: for every leading monomial t of some L_{m,d} that
    no monomial of L_{m,d-1} divides (times one variable), the row of RREF(M_{d,m}) with leading
    monomial t (it is monic and its other terms lie outside L_{m,d}).

Readings where the paper is silent: the signature order (position over term, e_i increasing with
i), the criterion (F5's, with the full leading-monomial set of the earlier generators' ideal at the
right degree), the candidate order (descending grevlex within a block), degree-by-degree blocks for
homogeneous input.
"""
from __future__ import annotations

import numpy as np

KEY_INDEX_SHIFT = 40
KEY_DEGREE_SHIFT = 32


def grevlex_key(e: tuple) -> tuple:
    """A key whose order is grevlex: higher total degree first; on equal degree the monomial with
    the smaller exponent in the last variable where they differ is the larger one."""
    return (sum(e), tuple(-x for x in reversed(e)))


def monomials_of_degree(n: int, e: int) -> list[tuple[int, ...]]:
    """All exponent vectors of total degree e in n variables, descending grevlex."""
    out: list[tuple[int, ...]] = []

    def rec(prefix: tuple, left: int, k: int):
        if k == n - 1:
            out.append(prefix + (left,))
            return
        for a in range(left, -1, -1):
            rec(prefix + (a,), left - a, k + 1)

    if n == 0:
        return [()] if e == 0 else []
    rec((), e, 0)
    out.sort(key=grevlex_key, reverse=True)
    return out


def mono_mul(a: tuple, b: tuple) -> tuple:
    return tuple(x + y for x, y in zip(a, b))


def pack_key(i: int, e: int, j: int) -> int:
    """The packed signature key of candidate j of generator i at shift degree e."""
    return (i << KEY_INDEX_SHIFT) | (e << KEY_DEGREE_SHIFT) | j


def normalised_inputs(system: dict) -> list[dict]:
    """The input polynomials as {exponent tuple: coefficient} dicts, equal terms merged, zero
    polynomials dropped, each made monic (leading coefficient 1)."""
    p, n = int(system["p"]), int(system["n"])
    out = []
    for i in range(int(system["m"])):
        f: dict = {}
        for q in range(int(system["poly_off"][i]), int(system["poly_off"][i + 1])):
            e = tuple(int(x) for x in system["exps"][q][:n])
            f[e] = (f.get(e, 0) + int(system["coeffs"][q])) % p
        f = {e: c for e, c in f.items() if c}
        if not f:
            continue
        lead = max(f, key=grevlex_key)
        inv = pow(f[lead], p - 2, p)
        out.append({e: c * inv % p for e, c in f.items()})
    return out


def is_homogeneous(f: dict) -> bool:
    return len({sum(e) for e in f}) <= 1


def rref(rows: np.ndarray, p: int) -> tuple[np.ndarray, list[int]]:
    """Reduced row echelon form over F_p by Gauss-Jordan elimination, column by column from the
    left: (the non-zero rows, their pivot columns in ascending order)."""
    A = np.array(rows, dtype=np.int64) % p
    if A.size == 0:
        return A.reshape(0, A.shape[1] if A.ndim == 2 else 0), []
    r = 0
    piv: list[int] = []
    nrows, ncols = A.shape
    for c in range(ncols):
        if r == nrows:
            break
        nz = np.nonzero(A[r:, c])[0]
        if nz.size == 0:
            continue
        k = r + int(nz[0])
        if k != r:
            A[[r, k]] = A[[k, r]]
        A[r] = A[r] * pow(int(A[r, c]), p - 2, p) % p
        f = A[:, c].copy()
        f[r] = 0
        hit = np.nonzero(f)[0]
        if hit.size:
            A[hit] = (A[hit] - (f[hit, None] * A[r][None, :]) % p) % p
        piv.append(c)
        r += 1
    return A[:r], piv


def row_of(f: dict, shift: tuple, col_of: dict, ncols: int) -> np.ndarray:
    """The dense row of x^shift f over the columns of its degree."""
    v = np.zeros(ncols, dtype=np.int64)
    for e, c in f.items():
        v[col_of[mono_mul(shift, e)]] = c
    return v


def forbidden_set(L: dict, i: int, e: int) -> set:
    """The F5 criterion's set for block (e + d_i, i): the leading monomials of the degree-e part
    of <f_1 .. f_{i-1}> (empty for i = 1 and below the least input degree)."""
    return L.get((i - 1, e), set())


def block_leading_monomials(prev: set, cand: list, adm: list, lead_f: tuple) -> set:
    """Leading monomials of the block's rows: those of the echelon rows of M_{d,i-1} and x^a LM(f_i)
    for the admissible candidates."""
    return prev | {mono_mul(cand[j], lead_f) for j in adm}


def f5(system: dict, dmax: int, criterion: bool = True) -> dict:
    """Degree-by-degree blocks up to degree dmax (see the module docstring).

    Returns {"blocks": [...], "elements": [...], "basis": [...], "L": {(i, d): set}} where each
    block is {"degree", "index", "candidates", "admissible", "keys", "rank", "new",
    "zero_reductions"}, "elements" the new elements of all blocks in order (term lists
    [(exponents, coefficient)] in descending grevlex) and "basis" the reduced Groebner basis up to
    degree dmax, sorted by leading monomial descending."""
    p, n = int(system["p"]), int(system["n"])
    F = normalised_inputs(system)
    for f in F:
        if not is_homogeneous(f):
            raise ValueError("the signature-filtered path takes homogeneous systems")
    deg = [sum(next(iter(f))) for f in F]
    L: dict = {}
    blocks, elements = [], []
    top: dict = {}  # d -> (RREF(M_{d,m}) rows, pivot monomials, columns)
    dmin = min(deg) if deg else 1
    for d in range(dmin, dmax + 1):
        cols = monomials_of_degree(n, d)
        col_of = {m: c for c, m in enumerate(cols)}
        R = np.zeros((0, len(cols)), dtype=np.int64)
        prev: set = set()
        for i, f in enumerate(F, start=1):
            if deg[i - 1] > d:
                L[(i, d)] = prev
                continue
            e = d - deg[i - 1]
            cand = monomials_of_degree(n, e)
            forbidden = forbidden_set(L, i, e) if criterion else set()
            adm = [j for j, a in enumerate(cand) if a not in forbidden]
            lead_f = max(f, key=grevlex_key)
            new_rows = [row_of(f, cand[j], col_of, len(cols)) for j in adm]
            stacked = np.vstack([R] + [r[None, :] for r in new_rows]) if new_rows else R
            R, piv = rref(stacked, p)
            now = {cols[c] for c in piv}
            block_leads = block_leading_monomials(prev, cand, adm, lead_f)
            new = []
            for row, c in zip(R, piv):
                if cols[c] in block_leads:
                    continue
                new.append([(cols[k], int(row[k])) for k in np.nonzero(row)[0]])
            blocks.append({
                "degree": d, "index": i, "candidates": len(cand), "admissible": len(adm),
                "keys": [pack_key(i, e, j) for j in adm],
                "rank": len(now) - len(prev), "new": len(new),
                "zero_reductions": len(adm) - (len(now) - len(prev)),
            })
            elements.extend(new)
            L[(i, d)] = now
            prev = now
        top[d] = (R, {cols[c]: k for k, c in enumerate(piv)}, cols)
    basis = []
    m = len(F)
    for d in range(dmin, dmax + 1):
        R, row_at, cols = top[d]
        below = L.get((m, d - 1), set())
        for t, k in row_at.items():
            minimal = True
            for v in range(n):
                if t[v] and tuple(t[u] - (u == v) for u in range(n)) in below:
                    minimal = False
                    break
            if minimal:
                row = R[k]
                basis.append([(cols[c], int(row[c])) for c in np.nonzero(row)[0]])
    basis.sort(key=lambda g: grevlex_key(g[0][0]), reverse=True)
    return {"blocks": blocks, "elements": elements, "basis": basis, "L": L}

