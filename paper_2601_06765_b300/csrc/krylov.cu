// krylov.cu -- the block Wiedemann kernel-vector path (Sec. 9.3; Prop. 3.2): vectors v with
// v^T A = 0 for one step's Macaulay matrix A (r x N), i.e. relations sum_i v_i t_i g_{k_i} = 0
// among its shifted rows, found with products of A and A^T and blocks of vectors only.
//
//   M = A diag(delta) A^T (symmetric); S_i = X^T M^(i+1) Z, i < 2d, d = ceil(r / b) + 1;
//   the right kernel of the block Hankel matrix H[i b + a][j b + c] = S_{i+j}[a][c] (i < d,
//   j <= d), one vector c per free column of RREF(H); y(c) = sum_j M^j Z c_j lies in ker M;
//   W = RREF of the y(c): a canonical basis of the vectors found.
//
// Device layout: a block of vectors is r x 32 u32, row-major (one 128-byte row per matrix row,
// lane c of a warp owns column c); b <= 32 columns are used, the others stay zero.  The sequence
// is one SpMM with A^T (warp per column of A, its entries gathered through a transposed CSR built
// once) scaled by delta, then one SpMM with A whose epilogue adds the row's outer product
// X[i] (x) Y[i] into S_i -- the Krylov sequence never leaves the device until the end.  The
// generator is the exact RREF of H on the device (the panel kernels and tensor-core updates of
// the echelon form of D'), a linear-algebra replacement for the Berlekamp-Massey recursion that
// the paper places on the host: at r in the tens of thousands the host recursion would dominate.
#include <algorithm>

#include "internal.hpp"

namespace gb {

namespace {

constexpr int KB = 32;  // vector block width on the device (the lanes of a warp)

__global__ void k_col_count(const uint32_t *__restrict__ col, uint64_t nnz, uint32_t *__restrict__ cnt) {
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < nnz; q += (uint64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[col[q]], 1u);
}

// entries of A into the rows of A^T (one row per column of A); within a row the order is the
// scatter's, which changes no sum mod p
__global__ void k_transpose_fill(uint32_t rows, const uint32_t *__restrict__ row_ptr, const uint32_t *__restrict__ col,
                                 const uint32_t *__restrict__ val, const uint32_t *__restrict__ tptr,
                                 uint32_t *__restrict__ cursor, uint32_t *__restrict__ tcol, uint32_t *__restrict__ tval) {
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= rows) return;
    for (uint32_t q = row_ptr[warp] + lane; q < row_ptr[warp + 1]; q += 32) {
        const uint32_t c = col[q];
        const uint32_t pos = tptr[c] + atomicAdd(&cursor[c], 1u);
        tcol[pos] = warp;
        tval[pos] = val[q];
    }
}

struct SpmmArgs {
    uint32_t rows;
    const uint32_t *row_ptr, *col, *val;
    const uint32_t *in;       // (columns of the operator) x 32
    uint32_t *out;            // rows x 32
    const uint32_t *scale;    // per output row, or null
    const uint32_t *X;        // projection: S[a][c] += X[i][a] out[i][c] (a, c < b), or null
    unsigned long long *S;    // 32 x 32 sums
    const uint32_t *Z, *C;    // epilogue: out[i][c] += sum_a Z[i][a] C[a][c] (a < b), or null
    uint32_t b;
    Fp fp;
};

// out = scale * (op in) [+ Z C]; warp per row (grid-stride), lane c = column c.  Products are
// reduced (31-bit p) or raw (16-bit p) and summed in 64 bits: exact for 2^32 terms.
template <bool SMALLP>
__global__ void __launch_bounds__(256) k_spmm(SpmmArgs a) {
    __shared__ unsigned long long Sb[KB * KB];
    __shared__ uint32_t Cs[KB * KB];
    const uint32_t lane = threadIdx.x & 31;
    if (a.X)
        for (uint32_t t = threadIdx.x; t < KB * KB; t += blockDim.x) Sb[t] = 0ull;
    if (a.C)  // rows j b .. j b + b - 1 of the kernel-vector block: only b rows exist past j b
        for (uint32_t t = threadIdx.x; t < a.b * KB; t += blockDim.x) Cs[t] = a.C[t];
    __syncthreads();
    const Fp fp = a.fp;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < a.rows; i += nwarps) {
        const uint32_t q0 = a.row_ptr[i], q1 = a.row_ptr[i + 1];
        unsigned long long acc = 0;
        for (uint32_t qb = q0; qb < q1; qb += 32) {
            const uint32_t q = qb + lane;
            const uint32_t mc = q < q1 ? a.col[q] : 0u, mv = q < q1 ? a.val[q] : 0u;
            const uint32_t cnt = min(32u, q1 - qb);
            for (uint32_t k = 0; k < cnt; ++k) {
                const uint32_t cc = __shfl_sync(0xffffffffu, mc, k), vv = __shfl_sync(0xffffffffu, mv, k);
                const uint32_t x = a.in[(size_t)cc * KB + lane];
                if (SMALLP) acc += (unsigned long long)(vv * x);
                else acc += fp_mul(vv, x, fp);
            }
        }
        uint32_t y = fp_reduce(acc, fp);
        if (a.scale) y = fp_mul(y, a.scale[i], fp);
        if (a.C) {
            const uint32_t zme = a.Z[(size_t)i * KB + lane];
            unsigned long long s = y;
            for (uint32_t t = 0; t < a.b; ++t) s += fp_mul(__shfl_sync(0xffffffffu, zme, t), Cs[t * KB + lane], fp);
            y = fp_reduce(s, fp);
        }
        a.out[(size_t)i * KB + lane] = y;
        if (a.X) {
            const uint32_t xme = a.X[(size_t)i * KB + lane];
            for (uint32_t t = 0; t < a.b; ++t) {
                const uint32_t xa = __shfl_sync(0xffffffffu, xme, t);
                if (xa && y) atomicAdd(&Sb[t * KB + lane], (unsigned long long)fp_mul(xa, y, fp));
            }
        }
    }
    if (a.X) {
        __syncthreads();
        for (uint32_t t = threadIdx.x; t < KB * KB; t += blockDim.x)
            if (Sb[t]) atomicAdd(&a.S[t], Sb[t]);
    }
}

// H[i b + a][j b + c] = S_{i+j}[a][c] (sums reduced mod p here)
__global__ void k_hankel(const unsigned long long *__restrict__ S, uint32_t d, uint32_t b, Fp fp, uint32_t *__restrict__ H) {
    const uint64_t nb = (uint64_t)(d + 1) * b, total = (uint64_t)d * b * nb;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total; t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t row = t / nb, colh = t % nb;
        const uint32_t i = (uint32_t)(row / b), aa = (uint32_t)(row % b), j = (uint32_t)(colh / b), c = (uint32_t)(colh % b);
        H[t] = fp_reduce(S[(size_t)(i + j) * KB * KB + aa * KB + c], fp);
    }
}

// 32 random combinations (batch t) of all nf kernel vectors of H: R[i][l] = coefficient of
// kernel vector i in combination l; C[F[i]][l] = R[i][l] and C[P_k][l] = -sum_i RREF[k][F[i]] R[i][l]
__global__ void k_combination_coeffs(uint32_t nf, uint32_t t, uint32_t p, uint32_t *__restrict__ R) {
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < (uint64_t)nf * KB; x += (uint64_t)gridDim.x * blockDim.x)
        R[x] = (uint32_t)(splitmix64(0x6a09e667f3bcc908ull + ((unsigned long long)t << 40) + x) % p);
}

__global__ void k_combine(const uint32_t *__restrict__ rref, const uint32_t *__restrict__ rpiv, uint32_t rank,
                          uint32_t nbh, const uint32_t *__restrict__ freec, uint32_t nf, const uint32_t *__restrict__ R,
                          Fp fp, uint32_t *__restrict__ C) {
    const uint32_t lane = threadIdx.x & 31, warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t k = warp; k < rank + nf; k += nwarps) {
        if (k >= rank) {  // a free column: its combination coefficients
            const uint32_t i = k - rank;
            C[(size_t)freec[i] * KB + lane] = R[(size_t)i * KB + lane];
            continue;
        }
        const uint32_t *row = rref + (size_t)k * nbh;
        unsigned long long acc = 0;
        for (uint32_t i = 0; i < nf; ++i) {
            const uint32_t v = row[freec[i]];
            if (v) acc += fp_mul(v, R[(size_t)i * KB + lane], fp);
        }
        const uint32_t s = fp_reduce(acc, fp);
        C[(size_t)rpiv[k] * KB + lane] = s ? fp.p - s : 0u;
    }
}

// kernel vectors of H for free columns free[l0 + l], l < 32: C[row][l] (rows (d + 1) b), 1 at the
// free column, p - RREF[k][f] at the pivot column of row k
__global__ void k_kernel_vectors(const uint32_t *__restrict__ rref, const uint32_t *__restrict__ rpiv, uint32_t rank,
                                 uint32_t nbh, const uint32_t *__restrict__ freec, uint32_t nfree, uint32_t p,
                                 uint32_t *__restrict__ C) {
    const uint32_t l = threadIdx.x & 31;
    if (l >= nfree) return;
    const uint32_t f = freec[l];
    if (blockIdx.x == 0 && threadIdx.x < 32) C[(size_t)f * KB + l] = 1u;
    for (uint32_t k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < rank; k += (gridDim.x * blockDim.x) >> 5) {
        const uint32_t v = rref[(size_t)k * nbh + f];
        C[(size_t)rpiv[k] * KB + l] = v ? p - v : 0u;
    }
}

// rows of the found vectors: Ws[l0 + l][i] = Y[i][l]
__global__ void k_gather_rows(const uint32_t *__restrict__ Y, uint32_t r, uint32_t n, uint32_t *__restrict__ Ws) {
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < (uint64_t)n * r; t += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t l = (uint32_t)(t / r), i = (uint32_t)(t % r);
        Ws[t] = Y[(size_t)i * KB + l];
    }
}

// W rows l0.. as the columns of a block, for the check A^T w = 0
__global__ void k_rows_to_block(const uint32_t *__restrict__ Wr, uint32_t r, uint32_t n, uint32_t *__restrict__ B) {
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < (uint64_t)r * KB; t += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t i = (uint32_t)(t / KB), l = (uint32_t)(t % KB);
        B[t] = l < n ? Wr[(size_t)l * r + i] : 0u;
    }
}

// bit l of *nonzero: column l of the block has a non-zero entry
__global__ void k_nonzero_columns(const uint32_t *__restrict__ B, uint32_t rows, uint32_t *__restrict__ nonzero) {
    uint32_t m = 0;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < (uint64_t)rows * KB; t += (uint64_t)gridDim.x * blockDim.x)
        if (B[t]) m |= 1u << (t % KB);
    for (int o = 16; o; o >>= 1) m |= __shfl_xor_sync(0xffffffffu, m, o);
    if ((threadIdx.x & 31) == 0 && m) atomicOr(nonzero, m);
}

unsigned grid_for(uint64_t items, unsigned per_block) {
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((items + per_block - 1) / per_block, 148ull * 16));
}

}  // namespace

void block_wiedemann(const gb_macaulay *mac, uint32_t b, const uint32_t *hX, const uint32_t *hZ,
                     const uint32_t *hdelta, uint32_t *hseq, uint32_t *hW, uint32_t wcap, gb_krylov_stats *stats) {
    gb_system *S = mac->sys;
    gb_ctx *ctx = S->ctx;
    Arena &ar = ctx->arena;
    cudaStream_t st = ctx->stream;
    const Fp fp = S->fp;
    const uint32_t r = mac->nrows, N = mac->ndict;
    if (b < 1 || b > (uint32_t)KB) fail(GB_EINVAL, "gb_block_wiedemann: block width b must be in [1, 32]");
    if (!r || !N) fail(GB_EINVAL, "gb_block_wiedemann: empty matrix");
    if (!hX || !hZ || !hdelta) fail(GB_EINVAL, "gb_block_wiedemann: null input block");
    for (uint32_t j = 0; j < N; ++j)
        if (!hdelta[j] || hdelta[j] >= fp.p) fail(GB_EINVAL, "gb_block_wiedemann: delta entries must be in [1, p)");
    const uint32_t d = (r + b - 1) / b + 1, L = 2 * d;
    const uint64_t hrows = (uint64_t)d * b, hcols = (uint64_t)(d + 1) * b;
    if (hrows * hcols >= (1ull << 34)) fail(GB_EUNSUPPORTED, "gb_block_wiedemann: block Hankel system above 2^34 entries");
    gb_krylov_stats ks{};
    ks.b = b;
    ks.d = d;
    ks.nterms = L;
    cudaEvent_t ev[4];
    for (auto &e : ev) GB_CUDA(cudaEventCreate(&e));
    struct EvGuard {
        cudaEvent_t *e;
        ~EvGuard() { for (int i = 0; i < 4; ++i) cudaEventDestroy(e[i]); }
    } evg{ev};
    GB_CUDA(cudaEventRecord(ev[0], st));

    // inputs: X and Z padded to 32 columns, delta
    DBuf<uint32_t> X, Z, delta, Y0, Y1, T, tptr, tcnt, tcol, tval;
    X.alloc(ar, (size_t)r * KB, st);
    Z.alloc(ar, (size_t)r * KB, st);
    delta.alloc(ar, N, st);
    {
        const size_t bytes = 8ull * r * KB + 4ull * N;
        uint32_t *hp = static_cast<uint32_t *>(ctx_pinned(ctx, bytes + 64));
        std::memset(hp, 0, 8ull * r * KB);
        for (uint32_t i = 0; i < r; ++i)
            for (uint32_t c = 0; c < b; ++c) {
                if (hX[(size_t)i * b + c] >= fp.p || hZ[(size_t)i * b + c] >= fp.p)
                    fail(GB_EINVAL, "gb_block_wiedemann: X and Z entries must be in [0, p)");
                hp[(size_t)i * KB + c] = hX[(size_t)i * b + c];
                hp[(size_t)r * KB + (size_t)i * KB + c] = hZ[(size_t)i * b + c];
            }
        std::memcpy(hp + 2ull * r * KB, hdelta, 4ull * N);
        GB_CUDA(cudaMemcpyAsync(X.p, hp, 4ull * r * KB, cudaMemcpyHostToDevice, st));
        GB_CUDA(cudaMemcpyAsync(Z.p, hp + (size_t)r * KB, 4ull * r * KB, cudaMemcpyHostToDevice, st));
        GB_CUDA(cudaMemcpyAsync(delta.p, hp + 2ull * r * KB, 4ull * N, cudaMemcpyHostToDevice, st));
    }
    // the rows of A^T
    const uint64_t nnz = mac->nnz;
    tcnt.alloc(ar, (size_t)N + 1, st);
    tptr.alloc(ar, (size_t)N + 1, st);
    tcol.alloc(ar, nnz, st);
    tval.alloc(ar, nnz, st);
    GB_CUDA(cudaMemsetAsync(tcnt.p, 0, 4ull * (N + 1), st));
    k_col_count<<<grid_for(nnz, 256), 256, 0, st>>>(mac->col.p, nnz, tcnt.p);
    counted();
    exclusive_scan(ctx, tcnt.p, tptr.p, (size_t)N + 1, st);
    GB_CUDA(cudaMemsetAsync(tcnt.p, 0, 4ull * (N + 1), st));
    k_transpose_fill<<<(r + 7) / 8, 256, 0, st>>>(r, mac->row_ptr.p, mac->col.p, mac->val.p, tptr.p, tcnt.p, tcol.p, tval.p);
    counted();

    Y0.alloc(ar, (size_t)r * KB, st);
    Y1.alloc(ar, (size_t)r * KB, st);
    T.alloc(ar, (size_t)N * KB, st);
    DBuf<unsigned long long> Sacc;
    Sacc.alloc(ar, (size_t)L * KB * KB, st);
    GB_CUDA(cudaMemsetAsync(Sacc.p, 0, 8ull * L * KB * KB, st));
    const bool smallp = fp.small != 0;
    auto spmm = [&](const SpmmArgs &a) {
        if (smallp) k_spmm<true><<<grid_for((uint64_t)a.rows * 32, 256), 256, 0, st>>>(a);
        else k_spmm<false><<<grid_for((uint64_t)a.rows * 32, 256), 256, 0, st>>>(a);
        counted();
    };
    // out = M in (+ Z C), with the projection into S when X is given
    auto apply_M = [&](const uint32_t *in, uint32_t *out, unsigned long long *Sdst, const uint32_t *Cj) {
        SpmmArgs t{};
        t.rows = N;
        t.row_ptr = tptr.p;
        t.col = tcol.p;
        t.val = tval.p;
        t.in = in;
        t.out = T.p;
        t.scale = delta.p;
        t.b = b;
        t.fp = fp;
        spmm(t);
        SpmmArgs y{};
        y.rows = r;
        y.row_ptr = mac->row_ptr.p;
        y.col = mac->col.p;
        y.val = mac->val.p;
        y.in = T.p;
        y.out = out;
        y.b = b;
        y.fp = fp;
        if (Sdst) {
            y.X = X.p;
            y.S = Sdst;
        }
        if (Cj) {
            y.Z = Z.p;
            y.C = Cj;
        }
        spmm(y);
        ks.spmm_products += 2ull * nnz * KB;
    };
    // the sequence: Y <- M Y, S_i = X^T Y
    GB_CUDA(cudaMemcpyAsync(Y0.p, Z.p, 4ull * r * KB, cudaMemcpyDeviceToDevice, st));
    uint32_t *cur = Y0.p, *nxt = Y1.p;
    for (uint32_t i = 0; i < L; ++i) {
        apply_M(cur, nxt, Sacc.p + (size_t)i * KB * KB, nullptr);
        std::swap(cur, nxt);
    }
    GB_CUDA(cudaEventRecord(ev[1], st));

    // the generator: RREF of the block Hankel matrix
    gb_echelon Eh;
    Eh.nC = (uint32_t)hrows;
    Eh.nb = (uint32_t)hcols;
    Eh.dprime.alloc(ar, hrows * hcols, st);
    k_hankel<<<grid_for(hrows * hcols, 256), 256, 0, st>>>(Sacc.p, d, b, fp, Eh.dprime.p);
    counted();
    DBuf<uint32_t> derr;
    derr.alloc(ar, 1, st);
    GB_CUDA(cudaMemsetAsync(derr.p, 0, 4, st));
    echelon_stage(ctx, {&Eh}, {fp}, derr.p);
    Eh.dprime.reset();
    const uint32_t rank = Eh.rank;
    std::vector<uint32_t> piv(rank);
    if (rank) {
        uint32_t *hp = static_cast<uint32_t *>(ctx_pinned(ctx, 4ull * rank + 16));
        GB_CUDA(cudaMemcpyAsync(hp, Eh.rpiv.p, 4ull * rank, cudaMemcpyDeviceToHost, st));
        ctx_sync(ctx);
        piv.assign(hp, hp + rank);
    }
    GB_CUDA(cudaEventRecord(ev[2], st));
    std::vector<uint32_t> freec;
    {
        std::vector<uint8_t> isp(hcols, 0);
        for (uint32_t k : piv) isp[k] = 1;
        for (uint32_t c = 0; c < hcols; ++c)
            if (!isp[c]) freec.push_back(c);
    }
    ks.hankel_rank = rank;
    ks.free_columns = (uint32_t)freec.size();

    // y(c) = sum_j M^j Z c_j by Horner, 32 vectors c at a time, their rows gathered and
    // echelonised.  With at most 32 free columns the vectors c are H's kernel basis itself.  With
    // more, most y(c) vanish (a kernel vector with c_0 = 0 gives M times another one), so the
    // vectors c are random combinations of the whole kernel basis, 32 per batch, until a batch
    // leaves the span's dimension below the number of combinations taken: the span then holds
    // the image of every kernel vector (with high probability), and W is its canonical basis.
    const uint32_t nf = (uint32_t)freec.size();
    const uint32_t maxb = (nf + KB - 1) / KB;
    DBuf<uint32_t> Ys, Cb, fdev, Rc;
    Ys.alloc(ar, (size_t)std::max<uint32_t>(maxb, 1) * KB * r, st);
    Cb.alloc(ar, hcols * KB, st);
    fdev.alloc(ar, std::max<uint32_t>(nf, 1), st);
    Rc.alloc(ar, (size_t)std::max<uint32_t>(nf, 1) * KB, st);
    if (nf) {
        uint32_t *hp = static_cast<uint32_t *>(ctx_pinned(ctx, 4ull * nf + 16));
        std::memcpy(hp, freec.data(), 4ull * nf);
        GB_CUDA(cudaMemcpyAsync(fdev.p, hp, 4ull * nf, cudaMemcpyHostToDevice, st));
    }
    gb_echelon Ew;
    uint32_t w = 0, nrows_y = 0;
    for (uint32_t t = 0; t < maxb; ++t) {
        const uint32_t nl = nf <= KB ? nf : KB;
        GB_CUDA(cudaMemsetAsync(Cb.p, 0, 4ull * hcols * KB, st));
        if (nf <= KB) {
            k_kernel_vectors<<<grid_for((uint64_t)rank * 32, 256), 256, 0, st>>>(Eh.rref.p, Eh.rpiv.p, rank,
                                                                                  (uint32_t)hcols, fdev.p, nl, fp.p, Cb.p);
            counted();
        } else {
            k_combination_coeffs<<<grid_for((uint64_t)nf * KB, 256), 256, 0, st>>>(nf, t, fp.p, Rc.p);
            k_combine<<<grid_for((uint64_t)(rank + nf) * 32, 256), 256, 0, st>>>(Eh.rref.p, Eh.rpiv.p, rank, (uint32_t)hcols,
                                                                                  fdev.p, nf, Rc.p, fp, Cb.p);
            counted(2);
        }
        GB_CUDA(cudaMemsetAsync(cur, 0, 4ull * r * KB, st));
        for (uint32_t j = d + 1; j-- > 0;) {
            apply_M(cur, nxt, nullptr, Cb.p + (size_t)j * b * KB);
            std::swap(cur, nxt);
        }
        k_gather_rows<<<grid_for((uint64_t)nl * r, 256), 256, 0, st>>>(cur, r, nl, Ys.p + (size_t)nrows_y * r);
        counted();
        nrows_y += nl;
        // W: the canonical basis of the vectors found so far
        Ew = gb_echelon{};
        Ew.nC = nrows_y;
        Ew.nb = r;
        Ew.dprime.alloc(ar, (size_t)nrows_y * r, st);
        GB_CUDA(cudaMemcpyAsync(Ew.dprime.p, Ys.p, 4ull * nrows_y * r, cudaMemcpyDeviceToDevice, st));
        echelon_stage(ctx, {&Ew}, {fp}, derr.p);
        w = Ew.rank;
        if (nf <= KB || w < nrows_y) break;
    }
    ks.found = w;
    // check A^T w = 0 for every row of W, 32 rows at a time
    uint32_t verified = 0;
    DBuf<uint32_t> flags;
    flags.alloc(ar, (w + KB - 1) / KB + 1, st);
    GB_CUDA(cudaMemsetAsync(flags.p, 0, 4ull * ((w + KB - 1) / KB + 1), st));
    for (uint32_t l0 = 0; l0 < w; l0 += KB) {
        const uint32_t nl = std::min<uint32_t>(KB, w - l0);
        k_rows_to_block<<<grid_for((uint64_t)r * KB, 256), 256, 0, st>>>(Ew.rref.p + (size_t)l0 * r, r, nl, cur);
        counted();
        SpmmArgs t{};
        t.rows = N;
        t.row_ptr = tptr.p;
        t.col = tcol.p;
        t.val = tval.p;
        t.in = cur;
        t.out = T.p;
        t.b = b;
        t.fp = fp;
        spmm(t);
        k_nonzero_columns<<<grid_for((uint64_t)N * KB, 256), 256, 0, st>>>(T.p, N, flags.p + l0 / KB);
        counted();
    }
    GB_CUDA(cudaEventRecord(ev[3], st));
    // results to the host in one synchronisation
    const size_t nflag = (w + KB - 1) / KB;
    const size_t wrows = std::min<uint32_t>(w, wcap);
    const size_t seqw = hseq ? (size_t)L * KB * KB : 0;
    const size_t pin = 8 * seqw + 4 * nflag + 4 + 16;
    char *hp = static_cast<char *>(ctx_pinned(ctx, pin));
    unsigned long long *hs = reinterpret_cast<unsigned long long *>(hp);
    uint32_t *hf = reinterpret_cast<uint32_t *>(hp + 8 * seqw);
    uint32_t *herr = hf + nflag;
    if (seqw) GB_CUDA(cudaMemcpyAsync(hs, Sacc.p, 8 * seqw, cudaMemcpyDeviceToHost, st));
    if (nflag) GB_CUDA(cudaMemcpyAsync(hf, flags.p, 4 * nflag, cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaMemcpyAsync(herr, derr.p, 4, cudaMemcpyDeviceToHost, st));
    if (hW && wrows) GB_CUDA(cudaMemcpyAsync(hW, Ew.rref.p, 4ull * wrows * r, cudaMemcpyDeviceToHost, st));
    ctx_sync(ctx);
    if (*herr) fail(GB_ETIMEOUT, "block Wiedemann: a bounded wait in the tensor-core kernel gave up");
    for (uint32_t l = 0; l < w; ++l)
        if (!((hf[l / KB] >> (l % KB)) & 1u)) ++verified;
    ks.verified = verified;
    if (seqw)
        for (uint32_t i = 0; i < L; ++i)
            for (uint32_t a = 0; a < b; ++a)
                for (uint32_t c = 0; c < b; ++c)
                    hseq[((size_t)i * b + a) * b + c] = (uint32_t)(hs[(size_t)i * KB * KB + a * KB + c] % fp.p);
    float ms = 0.f;
    GB_CUDA(cudaEventElapsedTime(&ms, ev[0], ev[1]));
    ks.ms_sequence = ms;
    GB_CUDA(cudaEventElapsedTime(&ms, ev[1], ev[2]));
    ks.ms_hankel = ms;
    GB_CUDA(cudaEventElapsedTime(&ms, ev[2], ev[3]));
    ks.ms_vectors = ms;
    GB_CUDA(cudaEventElapsedTime(&ms, ev[0], ev[3]));
    ks.ms_total = ms;
    if (stats) *stats = ks;
}

}  // namespace gb
