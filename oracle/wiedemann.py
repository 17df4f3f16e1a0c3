"""THE ORACLE for the block Wiedemann kernel-vector path -- test infrastructure only.

Only tests/, the package smoke check and bench.py's CPU-baseline leg may import it; the product
path never does, and it shares no code with the CUDA path.  Plain Python integers (numpy object
arrays) for small matrices.

What it computes (Sec. 9.3, Krylov methods; Prop. 3.2, kernel vectors are syzygies).  A is one
F4 step's Macaulay matrix (r rows, N columns, CSR).  A vector v with v^T A = 0 is a relation
sum_i v_i t_i g_{k_i} = 0 among the step's shifted rows.  The block Wiedemann method finds such
vectors with nothing but products of A and A^T with blocks of b vectors:

  1. the operator M = A diag(delta) A^T (r x r, symmetric; the random diagonal delta keeps
     ker M = ker A^T with high probability);
  2. the block Krylov sequence S_i = X^T M^(i+1) Z (b x b), i = 0 .. 2d - 1, d = ceil(r / b) + 1,
     for random blocks X, Z (r x b);
  3. the relations among the sequence: the right kernel of the block Hankel matrix
     H[i b + a][j b + c] = S_{i+j}[a][c] (i < d, j <= d), one basis vector per free column of
     RREF(H) -- a linear generator of the sequence written as an exact linear system instead of
     the Berlekamp-Massey recursion;
  4. for each such vector c = (c_0 .. c_d): y(c) = sum_j M^j Z c_j.  Then X^T M^(i+1) y(c) = 0 for
     i < d, so y(c) is orthogonal to the range of the symmetric M and lies in ker M;
  5. W = RREF of the vectors y(c): a canonical basis of the kernel vectors found.

Readings where the paper is silent: the operator (A diag(delta) A^T) and the generator (exact
Hankel solve); the random blocks and delta are inputs; d = ceil(r / b) + 1 sequence blocks.
"""
from __future__ import annotations

import numpy as np


def _obj(a) -> np.ndarray:
    return np.array(a, dtype=object)


def dense_matrix(row_ptr, col, val, N: int) -> np.ndarray:
    """A as an r x N object array (Def. of the Macaulay matrix: row i is t_i g_{k_i} on T)."""
    r = len(row_ptr) - 1
    A = np.zeros((r, N), dtype=object)
    for i in range(r):
        for q in range(int(row_ptr[i]), int(row_ptr[i + 1])):
            A[i, int(col[q])] = int(val[q])
    return A


def operator(A: np.ndarray, delta, p: int) -> np.ndarray:
    """M = A diag(delta) A^T mod p."""
    D = _obj(delta)
    return ((A * D[None, :]).dot(A.T)) % p


def sequence(M: np.ndarray, X, Z, nterms: int, p: int) -> list[np.ndarray]:
    """S_i = X^T M^(i+1) Z mod p, i < nterms (each b x b)."""
    X, Z = _obj(X), _obj(Z)
    Y = M.dot(Z) % p
    out = []
    for _ in range(nterms):
        out.append(X.T.dot(Y) % p)
        Y = M.dot(Y) % p
    return out


def rref(Mat: np.ndarray, p: int) -> tuple[np.ndarray, list[int]]:
    """Gauss-Jordan over F_p (textbook): rows of the reduced row echelon form and pivot columns."""
    R = np.array(Mat, dtype=object) % p
    rows, cols = R.shape
    piv = []
    k = 0
    for c in range(cols):
        if k == rows:
            break
        nz = [i for i in range(k, rows) if R[i, c] % p]
        if not nz:
            continue
        i = nz[0]
        if i != k:
            R[[k, i]] = R[[i, k]]
        R[k] = (R[k] * pow(int(R[k, c]), p - 2, p)) % p
        for i2 in range(rows):
            if i2 != k and R[i2, c] % p:
                R[i2] = (R[i2] - R[i2, c] * R[k]) % p
        piv.append(c)
        k += 1
    return R[:k], piv


def hankel(seq: list[np.ndarray], d: int, b: int) -> np.ndarray:
    H = np.zeros((d * b, (d + 1) * b), dtype=object)
    for i in range(d):
        for j in range(d + 1):
            H[i * b:(i + 1) * b, j * b:(j + 1) * b] = seq[i + j]
    return H


def kernel_basis(Rh: np.ndarray, piv: list[int], ncols: int, p: int) -> list[np.ndarray]:
    """One vector per free column f of RREF(H), ascending: 1 at f, -RREF[k][f] at pivot column k."""
    out = []
    pivset = set(piv)
    for f in range(ncols):
        if f in pivset:
            continue
        v = np.zeros(ncols, dtype=object)
        v[f] = 1
        for k, pc in enumerate(piv):
            v[pc] = (-Rh[k, f]) % p
        out.append(v)
    return out


def block_wiedemann(row_ptr, col, val, N: int, p: int, X, Z, delta) -> dict:
    """The whole path on one matrix: the sequence, RREF(H) with its pivots, and W (rows)."""
    A = dense_matrix(row_ptr, col, val, N)
    r = A.shape[0]
    b = len(X[0]) if r else 0
    d = -(-r // b) + 1
    M = operator(A, delta, p)
    seq = sequence(M, X, Z, 2 * d, p)
    H = hankel(seq, d, b)
    Rh, piv = rref(H, p)
    Zo = _obj(Z)
    ys = []
    for c in kernel_basis(Rh, piv, (d + 1) * b, p):
        y = np.zeros(r, dtype=object)
        for j in reversed(range(d + 1)):  # Horner: y <- M y + Z c_j
            y = (M.dot(y) + Zo.dot(c[j * b:(j + 1) * b])) % p
        ys.append(y)
    if ys:
        W, _ = rref(np.array(ys, dtype=object), p)
    else:
        W = np.zeros((0, r), dtype=object)
    return {"d": d, "seq": seq, "H_rref": Rh, "H_piv": piv, "W": W, "M": M, "A": A}
