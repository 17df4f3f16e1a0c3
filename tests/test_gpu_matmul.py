"""The exact tensor-core update C <- C -/+ A B mod p (gb_matmul_modp, the GEMM-like block update of
Sec. 9.2 with the modular arithmetic of Sec. 8) against its plain definition, computed here with
int64 numpy products of 16-bit halves.  Integer work: results must agree bit for bit."""
from __future__ import annotations

import numpy as np
import pytest

import paper_2601_06765_b300 as gb

pytestmark = pytest.mark.gpu

P16, P31 = 65521, 2147483647


def mulmod_ref(A: np.ndarray, B: np.ndarray, p: int) -> np.ndarray:
    """(A B) mod p exactly: A = A1 2^16 + A0, B = B1 2^16 + B0, every partial product below 2^63."""
    A = A.astype(np.int64)
    B = B.astype(np.int64)
    A0, A1 = A & 0xFFFF, A >> 16
    B0, B1 = B & 0xFFFF, B >> 16
    s16 = (1 << 16) % p
    s32 = (1 << 32) % p
    r = (A0 @ B0) % p
    r = (r + ((A0 @ B1) % p) * s16) % p
    r = (r + ((A1 @ B0) % p) * s16) % p
    r = (r + ((A1 @ B1) % p) * s32) % p
    return r


def run_case(ctx, p, m, n, k, rng, values=None, subtract=True, pad=(0, 0, 0)):
    import torch
    lda, ldb, ldc = k + pad[0], n + pad[1], n + pad[2]
    if values is None:
        A = rng.integers(0, p, size=(m, lda), dtype=np.int64)
        B = rng.integers(0, p, size=(k, ldb), dtype=np.int64)
        C = rng.integers(0, p, size=(m, ldc), dtype=np.int64)
    else:
        A = rng.choice(values, size=(m, lda)).astype(np.int64)
        B = rng.choice(values, size=(k, ldb)).astype(np.int64)
        C = rng.choice(values, size=(m, ldc)).astype(np.int64)
    dA = torch.from_numpy(A.astype(np.int32)).cuda()
    dB = torch.from_numpy(B.astype(np.int32)).cuda()
    dC = torch.from_numpy(C.astype(np.int32)).cuda()
    torch.cuda.synchronize()
    gb.gb_matmul_modp(ctx.h, p, m, n, k, dA.data_ptr(), lda, dB.data_ptr(), ldb, dC.data_ptr(), ldc, subtract)
    got = dC.cpu().numpy().astype(np.int64)
    prod = mulmod_ref(A[:, :k], B[:, :n], p)
    want = C.copy()
    want[:, :n] = (C[:, :n] - prod) % p if subtract else (C[:, :n] + prod) % p
    assert np.array_equal(got, want), f"p={p} m={m} n={n} k={k}: {np.count_nonzero(got != want)} entries differ"


@pytest.fixture(scope="module")
def ctx():
    c = gb.Context(arena_bytes=2 << 30)
    yield c
    c.close()


SHAPES = [(1, 1, 1), (5, 7, 3), (128, 64, 64), (130, 70, 65), (257, 200, 300), (300, 129, 513), (64, 300, 256)]


@pytest.mark.parametrize("p", [P16, P31, 7, 65519, 2147483629])
@pytest.mark.parametrize("shape", SHAPES)
def test_matmul_random(ctx, p, shape):
    run_case(ctx, p, *shape, np.random.default_rng(hash((p, shape)) & 0xFFFFFFFF))


@pytest.mark.parametrize("p", [P16, P31])
def test_matmul_extreme_digits(ctx, p):
    # values whose balanced digits sit at the ends of [-128, 127], at the full exact K per launch
    T = 32639 if p < 65536 else 2139062143
    vals = [0, 1, p - 1, T, T + 1, p // 2, p // 2 + 1, 128, 255, 256, p - 128, p - 129]
    kmax = 256 if p < 65536 else 128
    for k in (kmax, kmax + 64, 3 * kmax):
        run_case(ctx, p, 200, 130, k, np.random.default_rng(k), values=vals)


def test_matmul_add_and_pitches(ctx):
    rng = np.random.default_rng(5)
    run_case(ctx, P16, 150, 90, 200, rng, subtract=False, pad=(3, 5, 7))
    run_case(ctx, P31, 150, 90, 200, rng, subtract=False, pad=(1, 2, 3))


def test_matmul_rejects_bad_prime(ctx):
    with pytest.raises(gb.GbError):
        gb.gb_matmul_modp(ctx.h, 65536, 1, 1, 1, 0, 1, 0, 1, 0, 1)


def mulmod_rows_f64(A: np.ndarray, B: np.ndarray, p: int) -> np.ndarray:
    """(A B) mod p exactly for k <= 2^11: the products of 16-bit halves summed over k stay below
    2^43, which float64 holds exactly, so BLAS gives the exact integer sums."""
    A = A.astype(np.int64)
    B = B.astype(np.int64)
    assert A.shape[1] <= 1 << 11
    A0, A1 = (A & 0xFFFF).astype(np.float64), (A >> 16).astype(np.float64)
    B0, B1 = (B & 0xFFFF).astype(np.float64), (B >> 16).astype(np.float64)
    s16, s32 = (1 << 16) % p, (1 << 32) % p
    q = lambda X, Y: (X @ Y).astype(np.int64) % p
    r = q(A0, B0)
    r = (r + q(A0, B1) * s16) % p
    r = (r + q(A1, B0) * s16) % p
    r = (r + q(A1, B1) * s32) % p
    return r


@pytest.mark.parametrize("p,k", [(P16, 1024), (P31, 512)])
def test_matmul_at_the_benchmark_shape(ctx, p, k):
    """The shapes the benchmark times (4096 x 8192, K = 1024 at p = 65521 and K = 512 at
    p = 2^31 - 1: 4096 output tiles of 128 x 64 or 8192 of 128 x 32 over 148 SMs, so every CTA
    takes many tiles and both accumulator sets), checked entry by entry on 320 full rows: 256 random ones plus the first and
    last 32 (the first and last row tiles)."""
    import torch
    m, n = 4096, 8192
    rng = np.random.default_rng(p + k)
    A = rng.integers(0, p, size=(m, k), dtype=np.int64)
    B = rng.integers(0, p, size=(k, n), dtype=np.int64)
    C = rng.integers(0, p, size=(m, n), dtype=np.int64)
    dA, dB, dC = (torch.from_numpy(X.astype(np.int32)).cuda() for X in (A, B, C))
    torch.cuda.synchronize()
    gb.gb_matmul_modp(ctx.h, p, m, n, k, dA.data_ptr(), k, dB.data_ptr(), n, dC.data_ptr(), n, True)
    rows = np.unique(np.concatenate([rng.choice(m, 256, replace=False), np.arange(32), np.arange(m - 32, m)]))
    got = dC[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.int64)
    want = (C[rows] - mulmod_rows_f64(A[rows], B, p)) % p
    assert np.array_equal(got, want), f"{np.count_nonzero(got != want)} entries differ"
