// dense.cu -- the reduction of the non-pivot rows by the pivot rows (the PSGE trailing update of
// Sec. 9.2) as dense blocked elimination on the tensor cores, for steps whose non-pivot rows fill
// in.
//
// Columns are renumbered q(c): the pivot columns first in pivot order (pivot row i has leading
// column q = i), zero columns up to nAp = nA rounded up to 64, then the non-pivot columns in
// order.  With W the pivot rows (nA x N', unit upper triangular on its first nA columns) and M the
// non-pivot rows (nC x N'), the reduction is
//     F W[:, :nA] = M[:, :nA],    D' = M[:, nAp:] - F W[:, nAp:],
// and F is found block by block (right-looking, blocks of BS pivots):
//     F_J = M[:, J] U_J^{-1}                  (U_J = W[J, J]; four digits: M[:, J] + M[:, J] X_J on
//                                              the tensor cores, X_J = U_J^{-1} - I from k_block_inv;
//                                              two digits: the CUDA-core solve k_trsm_block)
//     M[:, j1:] <- M[:, j1:] - F_J W[J, j1:]  (tensor cores: mm_update)
// D' is unique (the pivot rows have distinct leading columns), so this schedule gives the same
// bits as the row-by-row sparse reduction.  BS = 512 / L (L digits per residue) is the longest K
// one exact tensor-core accumulation covers.
//
// Inside a block, the solve runs 32 pivots at a time with the 32 x 32 inverses of the chunk
// triangles that the sparse path also uses (Montgomery form for p >= 2^16): a warp owns one row,
// lane j holds the row's entries at columns j, j + 32, ... of the block; the chunk's multipliers
// are f = v_c U_c^{-1} (32 independent products per lane), then the later chunks of the block are
// updated with the rows of U_J held densely in Ub.
#include "internal.hpp"

namespace gb {

namespace {

constexpr int DW = 4;  // warps (rows) per block of the row kernels

__device__ __forceinline__ uint32_t qcol(uint32_t cp, uint32_t nAp) {
    return (cp & 0x80000000u) ? (cp & 0x7FFFFFFFu) : nAp + cp;
}

// balanced base-256 digits of a residue x as BF16 bits, digit l in d[l]
template <int L>
__device__ __forceinline__ void digits_bf16(uint32_t x, uint32_t p, uint16_t (&d)[L]) {
    const uint32_t T = L == 2 ? 32639u : 2139062143u;  // 127 (1 + 256 + ... + 256^{L-1})
    int v = x <= T ? (int)x : (int)(x - p);
#pragma unroll
    for (int l = 0; l < L; ++l) {
        const int a = l + 1 < L ? (int)(((uint32_t)v & 0xFFu) ^ 0x80u) - 0x80 : v;
        if (l + 1 < L) v = (v - a) >> 8;
        d[l] = (uint16_t)(__float_as_uint((float)a) >> 16);
    }
}

// balanced base-256 digits of a residue x as BF16 bits, digit l at dst[l * plane]
template <int L>
__device__ __forceinline__ void put_digits(uint32_t x, uint32_t p, uint16_t *dst, uint64_t plane) {
    uint16_t d[L];
    digits_bf16<L>(x, p, d);
#pragma unroll
    for (int l = 0; l < L; ++l) dst[(size_t)l * plane] = d[l];
}

// pivot row i: the entries inside its own block, right of the diagonal, go to the dense block Ub.
// They are pivot columns q in (i, j1), i.e. dictionary columns up to pcols[j1 - 1]: a prefix of
// the row (its columns ascend), so the warp stops at the first column past it.
__global__ void k_scatter_ub(DenseJob J) {
    const uint32_t i = blockIdx.x * DW + (threadIdx.x >> 5);
    if (i >= J.nA) return;
    const int lane = threadIdx.x & 31;
    const uint32_t j0 = i / J.bs * J.bs, j1 = min(j0 + J.bs, J.nA);
    if (i + 1 >= j1) return;  // the block's last pivot: nothing right of the diagonal inside it
    const uint32_t last = J.pcols[j1 - 1];
    uint32_t *ub = J.Ub + (size_t)(i / J.bs) * J.bs * J.bs + (size_t)(i - j0) * J.bs;
    for (uint32_t e0 = J.row_ptr[i]; e0 < J.row_ptr[i + 1]; e0 += 32) {
        const uint32_t e = e0 + lane;
        const bool in = e < J.row_ptr[i + 1] && J.col[e] <= last;
        if (in) {
            const uint32_t q = qcol(J.colpos[J.col[e]], J.nAp);
            if (q > i && q < j1) ub[q - j0] = J.val[e];
        }
        if (__ballot_sync(0xffffffffu, in) != 0xffffffffu) break;  // past the prefix
    }
}

// W^T as digit planes, every entry the update reads written once, zeros included (no memset of
// the planes, no scattered 2-byte writes): block (b, s) takes the 64 pivot rows [64 b, 64 b + 64)
// and the dictionary columns [s FS, (s + 1) FS), finds each row's first entry there by binary
// search and walks the segment in windows of FW, each row's CSR cursor advancing with the windows
// (a row's columns ascend).  A window's entries gather in a shared tile; then, per column c of the
// window and digit plane l, the 64 K entries of row q(c) of W^T go out as one 128-byte store of a
// warp.  Entries left of the end j1 of the pivots' own block (q < j1) are not written: the
// tensor-core update of that block starts at column j1 and never reads them (that skips the
// diagonal blocks and the zeros below them, about half of the pivot columns' part of the planes).
// Rows q in [nA, nAp) (the padding columns) come from no dictionary column; the caller zeroes
// them.
constexpr int FW = 128;      // dictionary columns per window
constexpr int FS = 16 * FW;  // dictionary columns per block
constexpr int FT = 256;      // threads per block (8 warps)
template <int L>
__global__ void __launch_bounds__(FT) k_fill_wt(DenseJob J) {
    __shared__ uint32_t tile[FW][65];
    __shared__ uint32_t cur[64], fin[64];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t i0 = blockIdx.x * 64, cs = blockIdx.y * FS, ce = min(cs + FS, J.N);
    if (threadIdx.x < 64) {
        const uint32_t i = i0 + threadIdx.x;
        uint32_t lo = 0, hi = 0;
        if (i < J.nA) {
            lo = J.row_ptr[i];
            hi = J.row_ptr[i + 1];
            fin[threadIdx.x] = hi;
            while (lo < hi) {  // the row's first entry at a column >= cs
                const uint32_t mid = (lo + hi) >> 1;
                if (J.col[mid] < cs) lo = mid + 1; else hi = mid;
            }
        } else {
            fin[threadIdx.x] = 0u;
        }
        cur[threadIdx.x] = lo;
    }
    const uint64_t plane = (uint64_t)J.Np * J.wkpad;
    for (uint32_t c0 = cs; c0 < ce; c0 += FW) {
        for (uint32_t k = threadIdx.x; k < FW * 64; k += FT) tile[k >> 6][k & 63] = 0u;
        __syncthreads();
        const uint32_t cend = min(c0 + FW, ce);
        for (uint32_t r = warp; r < 64; r += FT / 32) {
            uint32_t a = cur[r];
            const uint32_t e = fin[r];
            for (;;) {
                const uint32_t idx = a + lane;
                const uint32_t c = idx < e ? J.col[idx] : 0xFFFFFFFFu;
                const bool in = c < cend;
                if (in) tile[c - c0][r] = J.val[idx];
                const unsigned m = __ballot_sync(0xffffffffu, in);
                a += __popc(m);
                if (m != 0xffffffffu) break;
            }
            if (lane == 0) cur[r] = a;
        }
        __syncthreads();
        for (uint32_t cc = warp; cc < FW; cc += FT / 32) {
            const uint32_t c = c0 + cc;
            if (c >= ce) break;
            const uint32_t q = qcol(J.colpos[c], J.nAp);
            if (q < min((i0 / J.bs + 1) * J.bs, J.nAp)) continue;  // left of the block's end j1: never read
            uint16_t d0[L], d1[L];
            digits_bf16<L>(tile[cc][2 * lane], J.fp.p, d0);
            digits_bf16<L>(tile[cc][2 * lane + 1], J.fp.p, d1);
            uint32_t *dst = reinterpret_cast<uint32_t *>(J.WT + (size_t)q * J.wkpad + i0) + lane;
#pragma unroll
            for (int l = 0; l < L; ++l) dst[(size_t)l * (plane / 2)] = (uint32_t)d0[l] | ((uint32_t)d1[l] << 16);
        }
        __syncthreads();
    }
}

// non-pivot row r into the dense M
__global__ void k_scatter_rows(DenseJob J) {
    const uint32_t r = blockIdx.x * DW + (threadIdx.x >> 5);
    if (r >= J.nC) return;
    const int lane = threadIdx.x & 31;
    uint32_t *row = J.M + (size_t)r * J.ldm;
    for (uint32_t e = J.row_ptr[J.nA + r] + lane; e < J.row_ptr[J.nA + r + 1]; e += 32)
        row[qcol(J.colpos[J.col[e]], J.nAp)] = J.val[e];
}

// F_J = M[:, j0:j0+jn] U_J^{-1}, written as digit planes (row r, K index k) -- warp per row
template <int L>
__global__ void __launch_bounds__(DW * 32) k_trsm_block(DenseJob J, uint32_t j0) {
    constexpr int NS = 512 / L / 32;  // 32-pivot chunks per block
    constexpr bool SMALLP = L == 2;
    const uint32_t r = blockIdx.x * DW + (threadIdx.x >> 5);
    if (r >= J.nC) return;
    const int lane = threadIdx.x & 31;
    const Fp fp = J.fp;
    const uint32_t jn = min(J.bs, J.nA - j0);  // pivots of the block (the rest is padding)
    const uint32_t *row = J.M + (size_t)r * J.ldm + j0;
    const uint32_t *Ub = J.Ub + (size_t)(j0 / J.bs) * J.bs * J.bs;
    const uint32_t *Winv = J.Uinv + (size_t)(j0 / 32) * 32 * 32;
    const uint64_t fplane = (uint64_t)J.nC * J.fkpad;
    uint16_t *frow = J.F + (size_t)r * J.fkpad;
    uint32_t v[NS];
#pragma unroll
    for (int t = 0; t < NS; ++t) {
        const uint32_t k = 32u * t + lane;
        v[t] = k < jn ? row[k] : 0u;
    }
#pragma unroll
    for (int c = 0; c < NS; ++c) {
        if (32u * c >= jn) break;  // uniform across the warp
        // multipliers of chunk c: f_lane = sum_j v_c[j] W[j][lane]
        const uint32_t x = v[c];
        const uint32_t *W = Winv + (size_t)c * 32 * 32;
        unsigned long long s = 0;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const uint32_t xj = __shfl_sync(0xffffffffu, x, j);
            const uint32_t w = W[j * 32 + lane];
            if (SMALLP) s += (unsigned long long)(xj * w);
            else s += fp_redc((uint64_t)xj * w, fp);
        }
        const uint32_t k = 32u * c + lane;
        const uint32_t f = k < jn ? fp_reduce(s, fp) : 0u;
        if (k < jn) put_digits<L>(f, fp.p, frow + k, fplane);
        const uint32_t fm = f ? (SMALLP ? fp.p - f : fp_to_mont(fp.p - f, fp)) : 0u;
        // later chunks of the block: v_t <- v_t - f U[chunk c rows][chunk t columns]; each
        // multiplier is broadcast once and feeds every later chunk (independent accumulators)
        unsigned long long a[NS];
#pragma unroll
        for (int t = 0; t < NS; ++t) a[t] = v[t];
        const uint32_t *U = Ub + (size_t)(32 * c) * J.bs + lane;
#pragma unroll 4
        for (int i = 0; i < 32; ++i) {
            const uint32_t fi = __shfl_sync(0xffffffffu, fm, i);
            const uint32_t *Ui = U + (size_t)i * J.bs;
#pragma unroll
            for (int t = c + 1; t < NS; ++t) {
                const uint32_t u = Ui[32 * t];
                if (SMALLP) a[t] += (unsigned long long)(fi * u);
                else a[t] += fp_redc((uint64_t)fi * u, fp);
            }
        }
#pragma unroll
        for (int t = c + 1; t < NS; ++t) v[t] = fp_reduce(a[t], fp);
    }
}

// X_b = U_b^{-1} - I for every pivot block b (U_b = W[J_b, J_b], unit upper triangular, its
// entries right of the diagonal in Ub), as the digit planes of X_b^T: plane row b bs + n, K index
// i holds X_b[i][n].  From X'U = I with X' = U^{-1}: X'[i][j] = -(U[i][j] + sum_{i<k<j} X'[i][k]
// U[k][j]) for j > i, X'[i][i] = 1, 0 below.  Four threads (four consecutive lanes) compute row
// i, column by column: thread q sums the terms k = i + 1 + q (mod 4), two shuffles add the four
// shares, and the row's first thread stores X'[i][j] before the next column (one warp holds
// eight whole rows, so a __syncwarp orders it).  U_b is staged in shared memory with rows padded
// by one word.  Rows and columns at or past the block's pivot count jn (the padding of the last
// block) are zero.  Shared memory: U_b and the rows of X, 2 bs (bs + 1) words; bs rows x 4
// threads per block.
__global__ void k_block_inv(DenseJob J, uint16_t *__restrict__ xt, uint64_t kpad, uint64_t plane) {
    extern __shared__ uint32_t xs[];
    const uint32_t bs = J.bs, ld = bs + 1, b = blockIdx.x, j0 = b * bs;
    const uint32_t i = threadIdx.x >> 2, q = threadIdx.x & 3;
    const uint32_t jn = min(bs, J.nA - j0);
    uint32_t *us = xs + (size_t)bs * ld;  // U_b, row k at us + k ld
    const uint32_t *U = J.Ub + (size_t)b * bs * bs;
    for (uint32_t e = threadIdx.x; e < bs * bs; e += blockDim.x) us[(e / bs) * ld + e % bs] = U[e];
    __syncthreads();
    const Fp fp = J.fp;
    uint32_t *x = xs + (size_t)i * ld;
    for (uint32_t j = 0; j < bs; ++j) {
        const bool live = j < jn && i < j;
        uint32_t part = 0;
        if (live) {
            // at most 32 terms below p, and U[i][j] for the first share: far below 2^64
            unsigned long long acc = q == 0 ? us[i * ld + j] : 0u;
            for (uint32_t k = i + 1 + q; k < j; k += 4) acc += fp_mul(x[k], us[k * ld + j], fp);
            part = fp_reduce(acc, fp);
        }
        part = fp_add(part, __shfl_xor_sync(0xffffffffu, part, 1), fp);
        part = fp_add(part, __shfl_xor_sync(0xffffffffu, part, 2), fp);
        if (q == 0) x[j] = live && part ? fp.p - part : 0u;
        __syncwarp();
    }
    // X_b^T digit planes: thread q writes the columns n = q (mod 4) of its row
    for (uint32_t n = q; n < bs; n += 4) put_digits<4>(x[n], fp.p, xt + (size_t)(j0 + n) * kpad + i, plane);
}

__global__ void k_dense_work(DenseJob J, unsigned long long macs) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        J.work[0] += J.nA;
        J.work[1] += macs;
    }
}

inline unsigned blocks_of(size_t n, unsigned t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// The dense schedule pays once the non-pivot rows are many enough to fill in and the pivot
// block is wide enough for whole tensor-core blocks; below that the sparse row-by-row reduction,
// whose work follows the nonzeros, is faster.
bool dense_pays(uint32_t p, uint32_t N, uint32_t nA, uint32_t nC) {
    // measured on B300: dense wins from about 4k pivots and 1k non-pivot rows (31-bit p, where
    // the sparse path's Montgomery updates run in 64 bits), and at any row count past 16k pivots
    // (where the sparse path has too few rows to fill the GPU)
    (void)N;
    if (p < 65536u) return nA >= 8192 && nC >= 1024;
    return nA >= 4096 && (nC >= 1024 || nA >= 16384);
}

size_t dense_bytes(uint32_t p, uint32_t N, uint32_t nA, uint32_t nC) {
    const uint64_t L = digits_for(p), bs = mm_kmax(p);
    const uint64_t nAp = (nA + 63) / 64 * 64, Np = nAp + (N - nA), ldm = (Np + 3) / 4 * 4;
    const uint64_t nblk = (nAp + bs - 1) / bs;
    // W^T planes, M, the blocks U_J, F's planes; for four digits also X_J^T's and M[:, J]'s planes
    const uint64_t tc = L == 4 ? 2 * L * nblk * bs * bs + 2 * L * nC * bs : 0;
    return 2 * L * Np * nAp + 4 * nC * ldm + 4 * nblk * bs * bs + 2 * L * nC * bs + tc + 4096;
}

void reduce_dense(DenseJob J, uint32_t *dprime, Arena &ar, uint32_t *err, cudaStream_t st) {
    const uint32_t L = digits_for(J.fp.p);
    J.bs = mm_kmax(J.fp.p);
    J.nAp = (J.nA + 63) / 64 * 64;
    J.Np = J.nAp + J.nb;
    J.ldm = (J.Np + 3) / 4 * 4;
    const uint32_t nblk = (J.nAp + J.bs - 1) / J.bs;
    DBuf<uint32_t> M, Ub;
    DigitPlanes WT, F;
    M.alloc(ar, (size_t)J.nC * J.ldm, st);
    Ub.alloc(ar, (size_t)nblk * J.bs * J.bs, st);
    WT.alloc(ar, L, J.Np, J.nAp, st);
    F.alloc(ar, L, J.nC, J.bs, st);
    GB_CUDA(cudaMemsetAsync(M.p, 0, M.bytes(), st));
    GB_CUDA(cudaMemsetAsync(Ub.p, 0, Ub.bytes(), st));
    // rows [nA, nAp) of W^T (the padding columns) come from no dictionary column: zero them; the
    // rest of the planes that the trailing updates read is written by k_fill_wt
    for (uint32_t l = 0; l < L && J.nAp > J.nA; ++l)
        GB_CUDA(cudaMemsetAsync(WT.p + (size_t)l * J.Np * WT.kpad + (size_t)J.nA * WT.kpad, 0,
                                2ull * (J.nAp - J.nA) * WT.kpad, st));
    GB_CUDA(cudaMemsetAsync(F.p, 0, F.buf.bytes(), st));  // digits past a short last block stay finite
    J.M = M.p;
    J.Ub = Ub.p;
    J.WT = WT.p;
    J.wkpad = WT.kpad;
    J.F = F.p;
    J.fkpad = F.kpad;
    const dim3 wt_grid(J.nAp / 64, (J.N + FS - 1) / FS);
    if (L == 2) k_fill_wt<2><<<wt_grid, FT, 0, st>>>(J);
    else k_fill_wt<4><<<wt_grid, FT, 0, st>>>(J);
    k_scatter_ub<<<blocks_of(J.nA, DW), DW * 32, 0, st>>>(J);
    k_scatter_rows<<<blocks_of(J.nC, DW), DW * 32, 0, st>>>(J);
    counted(3);
    unsigned long long macs = 0;
    const MmPlan plan(F, WT, J.M, J.ldm, J.nC, J.Np, J.fp);
    // Four digits (p >= 2^16): the multipliers of a block on the tensor cores as well,
    //     F_J = M[:, J] U_J^{-1} = M[:, J] + M[:, J] X_J,   X_J = U_J^{-1} - I,
    // computed in place in M[:, J] from the digit planes of M[:, J] (MJ) and of X_J^T (Xt, all
    // blocks at once by k_block_inv).  The product's epilogue also writes F_J's digit planes (the
    // A operand of the trailing update), and the trailing update's epilogue those of the next
    // block's columns (MJ for the next block), so that only block 0's MJ is converted apart.  Two
    // digits keep the CUDA-core solve (k_trsm_block).
    DigitPlanes Xt, MJ;
    std::unique_ptr<MmPlan> fplan;
    if (L == 4 && nblk) {
        Xt.alloc(ar, L, (uint64_t)nblk * J.bs, J.bs, st);
        MJ.alloc(ar, L, J.nC, J.bs, st);
        const size_t smem = 8ull * J.bs * (J.bs + 1);
        opt_in_smem(reinterpret_cast<const void *>(k_block_inv));
        k_block_inv<<<nblk, 4 * J.bs, smem, st>>>(J, Xt.p, Xt.kpad, (uint64_t)Xt.rows * Xt.kpad);
        counted();
        fplan = std::make_unique<MmPlan>(MJ, Xt, J.M, J.ldm, J.nC, J.Np, J.fp);
    }
    // a view of planes P (same buffer and pitch) with only the first kb K values
    auto view = [](const DigitPlanes &P, uint32_t kb) {
        DigitPlanes v;
        v.L = P.L;
        v.rows = P.rows;
        v.K = kb;
        v.kpad = P.kpad;
        v.p = P.p;
        return v;
    };
    if (L == 4 && nblk) to_digits(J.M, J.ldm, 1, view(MJ, std::min(J.bs, J.nAp)), J.fp.p, st);
    // four digits: the block loop launches only k_mm, timed as one span (no events between the
    // launches, so that each overlaps the one before)
    MmTimer *T = L == 4 ? t_mm_timer : nullptr;
    if (T) T->begin_span(st);
    for (uint32_t b = 0; b < nblk; ++b) {
        const uint32_t j0 = b * J.bs, j1 = std::min(j0 + J.bs, J.nAp);
        const uint32_t next = b + 1 < nblk ? std::min(j1 + J.bs, J.nAp) - j1 : 0;  // the next block's width
        if (L == 4) {
            const uint32_t kb = j1 - j0;
            fplan->update(0, 0, 0, j0, j0, 0, J.nC, kb, kb, false, err, st, &F, kb, true);
            macs += (unsigned long long)J.nC * kb * kb;
        } else {
            k_trsm_block<2><<<blocks_of(J.nC, DW), DW * 32, 0, st>>>(J, j0);
            counted();
        }
        // columns j1.. of M, K = the block's pivots (a multiple of 64: padding pivots are zero)
        plan.update(0, 0, j0, j1, j1, 0, J.nC, J.Np - j1, j1 - j0, true, err, st, L == 4 ? &MJ : nullptr,
                    L == 4 ? next : 0, L == 4);
        macs += (unsigned long long)J.nC * (j1 - j0) * (J.Np - j1);
    }
    if (T) T->end_span(st);
    k_dense_work<<<1, 32, 0, st>>>(J, macs);
    counted();
    // D' = M[:, nAp:]
    if (J.nb)
        GB_CUDA(cudaMemcpy2DAsync(dprime, 4ull * J.nb, J.M + J.nAp, 4ull * J.ldm, 4ull * J.nb, J.nC,
                                  cudaMemcpyDeviceToDevice, st));
}

}  // namespace gb
