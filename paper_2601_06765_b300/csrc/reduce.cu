// reduce.cu -- the numeric phase (Sec. 9.2): structured elimination of the Macaulay matrix.
//
// Rows of Pi come as nA pivot rows (distinct leading columns pcols[0..nA), ascending, every row
// monic) followed by nC non-pivot rows.  The result is unique (the pivot rows have distinct
// leading columns), so any schedule on the device gives the same bits as the CPU oracle.
//
//   k_reduce   each non-pivot row is loaded into a dense accumulator (shared memory, or global
//              memory for wide dictionaries); the pivot columns at or right of its leading column
//              are swept in ascending order and every nonzero entry c is cleared with
//              v <- v - v[c] * (pivot row of c), a sparse row AXPY (eq. 8.1).  Accumulation is lazy
//              (Rem. 8.1): 64-bit sums of products (p < 2^16) or of Montgomery products (p < 2^31)
//              are reduced with Barrett only when an entry is read.  Output: D' (nC x nb, dense).
//   rref_*     RREF(D') by row panels: reduce a panel by the current echelon rows (a GEMM-shaped
//              update), echelonise what is left in one block, then clear the new pivot columns
//              from the older rows and append.
//   append     echelon rows become new basis elements (Sec. 4.2 step 4), written to the device
//              basis in standard form.
#include <algorithm>

#include "internal.hpp"

namespace gb {

namespace {

constexpr int RT = 256;  // threads per block of the row-reduction kernel

inline unsigned blocks(size_t n, unsigned t) { return (unsigned)((n + t - 1) / t); }

template <bool SMALLP, bool SMEM>
__global__ void __launch_bounds__(RT) k_reduce(uint32_t nA, uint32_t N,
                                              const uint32_t *__restrict__ row_ptr,
                                              const uint32_t *__restrict__ col,
                                              const uint32_t *__restrict__ val,
                                              const uint32_t *__restrict__ pcols,
                                              const uint32_t *__restrict__ nonpiv, uint32_t nb,
                                              Fp fp, unsigned long long *__restrict__ gacc,
                                              uint32_t *__restrict__ dprime,
                                              unsigned long long *__restrict__ work) {
    extern __shared__ unsigned long long sacc[];
    uint32_t applied = 0, fmas = 0;  // pivot rows applied and mod-p multiply-adds (thread 0)
    const uint32_t i = blockIdx.x, row = nA + i;
    const uint32_t a = row_ptr[row], b = row_ptr[row + 1];
    const uint32_t lm = a < b ? col[a] : N;
    const uint32_t width = N - lm;
    unsigned long long *acc = SMEM ? sacc : gacc + (size_t)i * N;
    for (uint32_t j = threadIdx.x; j < width; j += RT) acc[j] = 0ull;
    __syncthreads();
    for (uint32_t q = a + threadIdx.x; q < b; q += RT) acc[col[q] - lm] = val[q];
    // first pivot column at or right of lm
    uint32_t lo = 0, hi = nA;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (pcols[mid] < lm) lo = mid + 1; else hi = mid;
    }
    for (uint32_t k = lo; k < nA; ++k) {
        const uint32_t c = pcols[k];
        __syncthreads();
        const uint32_t f = fp_reduce(acc[c - lm], fp);
        if (f == 0) continue;  // uniform: every thread read the same entry
        const uint32_t neg = fp.p - f;
        const uint32_t mult = SMALLP ? neg : fp_to_mont(neg, fp);
        const uint32_t pa = row_ptr[k] + 1, pb = row_ptr[k + 1];
        if (threadIdx.x == 0) {
            ++applied;
            fmas += pb - pa;
        }
        for (uint32_t q = pa + threadIdx.x; q < pb; q += RT) {
            const uint64_t prod = (uint64_t)mult * val[q];
            acc[col[q] - lm] += SMALLP ? prod : (uint64_t)fp_redc(prod, fp);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(&work[0], (unsigned long long)applied);
        atomicAdd(&work[1], (unsigned long long)fmas);
    }
    uint32_t *out = dprime + (size_t)i * nb;
    for (uint32_t jj = threadIdx.x; jj < nb; jj += RT) {
        const uint32_t c = nonpiv[jj];
        out[jj] = c >= lm ? fp_reduce(acc[c - lm], fp) : 0u;
    }
}

// ---- RREF(D') by row panels ------------------------------------------------------------------

struct Ech {
    uint32_t *E;      // rho_cap x nb echelon rows (RREF among themselves), unordered
    uint32_t *epiv;   // their pivot positions
    uint32_t *state;  // [0] rho, [1] nnew of the current panel
    uint32_t nb, cap;
};

// R[r] = D'[i0 + r] - sum_e D'[i0 + r][epiv_e] * E_e   (the E rows are zero on each other's pivots)
__global__ void k_panel_reduce(const uint32_t *__restrict__ Dp, uint32_t i0, Ech X, Fp fp,
                               uint32_t *__restrict__ R) {
    extern __shared__ uint32_t m[];
    const uint32_t r = blockIdx.x, nb = X.nb;
    const uint32_t rho = X.state[0];
    const uint32_t *src = Dp + (size_t)(i0 + r) * nb;
    for (uint32_t e = threadIdx.x; e < rho; e += blockDim.x) m[e] = src[X.epiv[e]];
    __syncthreads();
    const uint32_t j = blockIdx.y * blockDim.x + threadIdx.x;
    if (j >= nb) return;
    uint64_t acc = src[j];
    if (fp.small) {
        for (uint32_t e = 0; e < rho; ++e)
            if (m[e]) acc += (uint64_t)(fp.p - m[e]) * X.E[(size_t)e * nb + j];
        R[(size_t)r * nb + j] = fp_reduce(acc, fp);
    } else {
        for (uint32_t e = 0; e < rho; ++e)
            if (m[e]) acc += fp_mul(fp.p - m[e], X.E[(size_t)e * nb + j], fp);
        R[(size_t)r * nb + j] = fp_reduce(acc, fp);
    }
}

// one block: Gauss-Jordan over the P reduced panel rows; new rows go to E[rho..rho+nnew)
constexpr int PT = 1024;
__global__ void __launch_bounds__(PT) k_panel_solve(uint32_t *__restrict__ R, uint32_t P, Ech X,
                                                   Fp fp) {
    __shared__ uint32_t mult[64];
    __shared__ uint32_t newpiv[64];
    __shared__ uint32_t red[PT / 32];
    __shared__ uint32_t s_c, s_inv;
    const uint32_t nb = X.nb, rho = X.state[0];
    uint32_t nnew = 0;
    uint32_t *NewRows = X.E + (size_t)rho * nb;
    for (uint32_t r = 0; r < P; ++r) {
        uint32_t *row = R + (size_t)r * nb;
        // reduce by the panel's new rows (zero on each other's pivots)
        if (threadIdx.x < nnew) mult[threadIdx.x] = row[newpiv[threadIdx.x]];
        __syncthreads();
        if (nnew) {
            for (uint32_t j = threadIdx.x; j < nb; j += PT) {
                uint64_t acc = row[j];
                for (uint32_t k = 0; k < nnew; ++k)
                    if (mult[k]) acc += fp_mul(fp.p - mult[k], NewRows[(size_t)k * nb + j], fp);
                row[j] = fp_reduce(acc, fp);
            }
        }
        __syncthreads();
        // first nonzero column
        uint32_t c = 0xFFFFFFFFu;
        for (uint32_t j = threadIdx.x; j < nb; j += PT)
            if (row[j]) { c = j; break; }
        for (int d = 16; d; d >>= 1) c = min(c, __shfl_xor_sync(0xffffffffu, c, d));
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
        __syncthreads();
        if (threadIdx.x < 32) {
            uint32_t v = red[threadIdx.x];
            for (int d = 16; d; d >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, d));
            if (threadIdx.x == 0) {
                s_c = v;
                if (v != 0xFFFFFFFFu) s_inv = fp_inv(row[v], fp);
            }
        }
        __syncthreads();
        c = s_c;
        if (c == 0xFFFFFFFFu) continue;
        if (nnew == 64 || rho + nnew >= X.cap) break;  // cannot happen: P <= 64, rank <= cap
        const uint32_t inv = s_inv;
        for (uint32_t j = threadIdx.x; j < nb; j += PT) row[j] = fp_mul(row[j], inv, fp);
        if (threadIdx.x < nnew) mult[threadIdx.x] = NewRows[(size_t)threadIdx.x * nb + c];
        __syncthreads();
        // clear column c from the earlier new rows, then append the row
        for (uint32_t idx = threadIdx.x; idx < nnew * nb; idx += PT) {
            const uint32_t k = idx / nb, j = idx - k * nb;
            if (mult[k]) {
                uint32_t *x = NewRows + (size_t)k * nb + j;
                *x = fp_sub(*x, fp_mul(mult[k], row[j], fp), fp);
            }
        }
        for (uint32_t j = threadIdx.x; j < nb; j += PT) NewRows[(size_t)nnew * nb + j] = row[j];
        if (threadIdx.x == 0) {
            newpiv[nnew] = c;
            X.epiv[rho + nnew] = c;
        }
        __syncthreads();
        ++nnew;
    }
    if (threadIdx.x == 0) X.state[1] = nnew;
}

// E_e -= sum_k E_e[newpiv_k] * New_k for the rows that existed before this panel.  One block
// owns a whole row: the multipliers are entries of the row being rewritten, so they are read
// before any thread of the block writes it.
__global__ void k_panel_merge(Ech X, Fp fp) {
    __shared__ uint32_t m[64];
    const uint32_t e = blockIdx.x, nb = X.nb;
    const uint32_t rho = X.state[0], nnew = X.state[1];
    if (e >= rho || nnew == 0) return;
    uint32_t *row = X.E + (size_t)e * nb;
    const uint32_t *New = X.E + (size_t)rho * nb;
    for (uint32_t k = threadIdx.x; k < nnew; k += blockDim.x) m[k] = row[X.epiv[rho + k]];
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < nb; j += blockDim.x) {
        uint64_t acc = row[j];
        for (uint32_t k = 0; k < nnew; ++k)
            if (m[k]) acc += fp_mul(fp.p - m[k], New[(size_t)k * nb + j], fp);
        row[j] = fp_reduce(acc, fp);
    }
}

__global__ void k_panel_commit(Ech X) { X.state[0] += X.state[1]; }

// order the echelon rows by pivot position
__global__ void k_sort_rows(Ech X, uint32_t *__restrict__ out, uint32_t *__restrict__ opiv) {
    const uint32_t e = blockIdx.x, nb = X.nb, rho = X.state[0];
    if (e >= rho) return;
    __shared__ uint32_t pos;
    if (threadIdx.x == 0) {
        uint32_t c = 0;
        for (uint32_t f = 0; f < rho; ++f) c += X.epiv[f] < X.epiv[e];
        pos = c;
        opiv[c] = X.epiv[e];
    }
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < nb; j += blockDim.x)
        out[(size_t)pos * nb + j] = X.E[(size_t)e * nb + j];
}

// ---- reconstruction --------------------------------------------------------------------------

__global__ void k_count_rows(const uint32_t *__restrict__ M, uint32_t rows, uint32_t nb,
                             uint32_t *__restrict__ cnt) {
    const uint32_t r = blockIdx.x;
    if (r >= rows) return;
    uint32_t c = 0;
    for (uint32_t j = threadIdx.x; j < nb; j += blockDim.x) c += M[(size_t)r * nb + j] != 0;
    for (int d = 16; d; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
    __shared__ uint32_t s[32];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (uint32_t w = 0; w < blockDim.x / 32; ++w) t += s[w];
        cnt[r] = t;
    }
}

// write the nonzeros of row r (ascending columns = descending monomials) at out_off[r]
__global__ void k_write_rows(const uint32_t *__restrict__ M, uint32_t rows, uint32_t nb,
                             const uint32_t *__restrict__ nonpiv, const uint4 *__restrict__ dict,
                             const uint32_t *__restrict__ out_off, uint4 *__restrict__ omon,
                             uint32_t *__restrict__ ocf) {
    const uint32_t r = blockIdx.x;
    if (r >= rows) return;
    __shared__ uint32_t base;
    __shared__ uint32_t wsum[32];
    if (threadIdx.x == 0) base = out_off[r];
    __syncthreads();
    const uint32_t *src = M + (size_t)r * nb;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x / 32;
    for (uint32_t j0 = 0; j0 < nb; j0 += blockDim.x) {
        const uint32_t j = j0 + threadIdx.x;
        const uint32_t v = j < nb ? src[j] : 0u;
        const unsigned mask = __ballot_sync(0xffffffffu, v != 0);
        if (lane == 0) wsum[warp] = __popc(mask);
        __syncthreads();
        uint32_t before = 0, total = 0;
        for (int w = 0; w < nw; ++w) {
            if (w < warp) before += wsum[w];
            total += wsum[w];
        }
        if (v) {
            const uint32_t pos = base + before + __popc(mask & ((1u << lane) - 1u));
            omon[pos] = dict[nonpiv[j]];
            ocf[pos] = v;
        }
        __syncthreads();
        if (threadIdx.x == 0) base += total;
        __syncthreads();
    }
}

__global__ void k_gather_lms(uint32_t rank, const uint32_t *__restrict__ rpiv,
                             const uint32_t *__restrict__ nonpiv, const uint4 *__restrict__ dict,
                             uint4 *__restrict__ out) {
    const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < rank) out[e] = dict[nonpiv[rpiv[e]]];
}

}  // namespace

std::unique_ptr<gb_echelon> reduce_rows(gb_macaulay *Mac, bool echelon) {
    gb_system *S = Mac->sys;
    Arena &ar = S->ctx->arena;
    cudaStream_t st = S->stream;
    auto E = std::make_unique<gb_echelon>();
    E->mac = Mac;
    E->nC = Mac->nC;
    E->nb = Mac->nb;
    const uint32_t nC = Mac->nC, nb = Mac->nb, N = Mac->ndict, nA = Mac->nA;
    E->dprime.alloc(ar, (size_t)nC * nb, st);
    GB_CUDA(cudaEventRecord(S->ev[2], st));
    DBuf<unsigned long long> work;
    work.alloc(ar, 2, st);
    GB_CUDA(cudaMemsetAsync(work.p, 0, 16, st));
    if (nC && nb) {
        const size_t smem = sizeof(unsigned long long) * N;
        const bool small = S->fp.small != 0;
        const bool use_smem = smem <= 200 * 1024;
        DBuf<unsigned long long> gacc;
        if (use_smem) {
            auto kern = small ? k_reduce<true, true> : k_reduce<false, true>;
            GB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            kern<<<nC, RT, smem, st>>>(nA, N, Mac->row_ptr.p, Mac->col.p, Mac->val.p, Mac->pcols.p,
                                       Mac->nonpiv.p, nb, S->fp, nullptr, E->dprime.p, work.p);
            counted();
        } else {
            gacc.alloc(ar, (size_t)nC * N, st);
            auto kern = small ? k_reduce<true, false> : k_reduce<false, false>;
            kern<<<nC, RT, 0, st>>>(nA, N, Mac->row_ptr.p, Mac->col.p, Mac->val.p, Mac->pcols.p,
                                    Mac->nonpiv.p, nb, S->fp, gacc.p, E->dprime.p, work.p);
            counted();
        }
        GB_CUDA(cudaGetLastError());
    }
    GB_CUDA(cudaEventRecord(S->ev[3], st));
    if (echelon && nC && nb) {
        const uint32_t cap = std::min(nC, nb);
        const uint32_t P = 64;
        DBuf<uint32_t> Ebuf, epiv, state, R;
        Ebuf.alloc(ar, (size_t)cap * nb, st);
        epiv.alloc(ar, cap, st);
        state.alloc(ar, 2, st);
        R.alloc(ar, (size_t)P * nb, st);
        GB_CUDA(cudaMemsetAsync(state.p, 0, 8, st));
        Ech X{Ebuf.p, epiv.p, state.p, nb, cap};
        const size_t msm = sizeof(uint32_t) * std::max<uint32_t>(cap, 1);
        if (msm > 48 * 1024) {
            GB_CUDA(cudaFuncSetAttribute(k_panel_reduce, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)msm));
        }
        for (uint32_t i0 = 0; i0 < nC; i0 += P) {
            const uint32_t rows = std::min(P, nC - i0);
            k_panel_reduce<<<dim3(rows, blocks(nb, 256)), 256, msm, st>>>(E->dprime.p, i0, X, S->fp, R.p);
            counted();
            k_panel_solve<<<1, PT, 0, st>>>(R.p, rows, X, S->fp);
            counted();
            k_panel_merge<<<cap, 256, 0, st>>>(X, S->fp);
            counted();
            k_panel_commit<<<1, 1, 0, st>>>(X);
            counted();
            GB_CUDA(cudaGetLastError());
        }
        uint32_t *h = static_cast<uint32_t *>(pinned(S, 64));
        GB_CUDA(cudaMemcpyAsync(h, state.p, 4, cudaMemcpyDeviceToHost, st));
        GB_CUDA(cudaMemcpyAsync(h + 2, work.p, 16, cudaMemcpyDeviceToHost, st));
        sync(S);
        E->rank = h[0];
        std::memcpy(E->work, h + 2, 16);
        E->rref.alloc(ar, (size_t)E->rank * nb, st);
        E->rpiv.alloc(ar, E->rank, st);
        if (E->rank) {
            k_sort_rows<<<E->rank, 256, 0, st>>>(X, E->rref.p, E->rpiv.p);
            counted();
        }
        GB_CUDA(cudaGetLastError());
    }
    GB_CUDA(cudaEventRecord(S->ev[4], st));
    if (!echelon) {
        uint64_t *h = static_cast<uint64_t *>(pinned(S, 64));
        GB_CUDA(cudaMemcpyAsync(h, work.p, 16, cudaMemcpyDeviceToHost, st));
        sync(S);
        std::memcpy(E->work, h, 16);
    }
    sync(S);
    GB_CUDA(cudaEventElapsedTime(&E->ms_reduce, S->ev[2], S->ev[3]));
    GB_CUDA(cudaEventElapsedTime(&E->ms_rref, S->ev[3], S->ev[4]));
    return E;
}

void append_echelon(gb_system *S, gb_echelon *E, std::vector<Mono> &lms, std::vector<uint32_t> &lens) {
    Arena &ar = S->ctx->arena;
    cudaStream_t st = S->stream;
    const uint32_t rank = E->rank, nb = E->nb;
    lms.clear();
    lens.clear();
    if (!rank) return;
    gb_macaulay *Mac = E->mac;
    DBuf<uint32_t> cnt, off;
    DBuf<uint4> lmd;
    cnt.alloc(ar, rank, st);
    off.alloc(ar, (size_t)rank + 1, st);
    lmd.alloc(ar, rank, st);
    k_count_rows<<<rank, 256, 0, st>>>(E->rref.p, rank, nb, cnt.p);
    counted();
    exclusive_scan(ar, cnt.p, off.p, rank, st);
    k_gather_lms<<<blocks(rank, 128), 128, 0, st>>>(rank, E->rpiv.p, Mac->nonpiv.p, Mac->dict.p, lmd.p);
    counted();
    GB_CUDA(cudaGetLastError());
    char *h = static_cast<char *>(pinned(S, 32ull * rank + 256));
    uint32_t *hoff = reinterpret_cast<uint32_t *>(h);
    Mono *hlm = reinterpret_cast<Mono *>(h + ((4ull * (rank + 1) + 15) & ~15ull));
    GB_CUDA(cudaMemcpyAsync(hoff, off.p, 4ull * (rank + 1), cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaMemcpyAsync(hlm, lmd.p, 16ull * rank, cudaMemcpyDeviceToHost, st));
    sync(S);
    lms.assign(hlm, hlm + rank);
    const uint64_t add = hoff[rank];
    const uint64_t base = S->nterms;
    if (base + add >= (1ull << 32)) fail(GB_EUNSUPPORTED, "basis above 2^32 terms");
    const size_t ng0 = S->off.size();
    std::vector<uint32_t> noff(rank), nlen(rank);
    for (uint32_t e = 0; e < rank; ++e) {
        noff[e] = (uint32_t)(base + hoff[e]);
        nlen[e] = hoff[e + 1] - hoff[e];
    }
    if (base + add > S->bmon.n) {
        S->bmon.grow(ar, std::max<size_t>(base + add, 2 * S->bmon.n), base, st);
        S->bcf.grow(ar, std::max<size_t>(base + add, 2 * S->bcf.n), base, st);
    }
    if (ng0 + rank > S->boff.n) {
        S->boff.grow(ar, std::max<size_t>(ng0 + rank, 2 * S->boff.n), ng0, st);
        S->blen.grow(ar, std::max<size_t>(ng0 + rank, 2 * S->blen.n), ng0, st);
    }
    uint32_t *hb = reinterpret_cast<uint32_t *>(h);  // the read-back above is complete
    std::memcpy(hb, noff.data(), 4ull * rank);
    std::memcpy(hb + rank, nlen.data(), 4ull * rank);
    GB_CUDA(cudaMemcpyAsync(S->boff.p + ng0, hb, 4ull * rank, cudaMemcpyHostToDevice, st));
    GB_CUDA(cudaMemcpyAsync(S->blen.p + ng0, hb + rank, 4ull * rank, cudaMemcpyHostToDevice, st));
    k_write_rows<<<rank, 256, 0, st>>>(E->rref.p, rank, nb, Mac->nonpiv.p, Mac->dict.p,
                                       S->boff.p + ng0, S->bmon.p, S->bcf.p);
    counted();
    GB_CUDA(cudaGetLastError());
    sync(S);  // the staging buffer is reused by the next step
    S->nterms = base + add;
    lens = nlen;
    for (uint32_t e = 0; e < rank; ++e) {
        S->off.push_back(noff[e]);
        S->len.push_back(nlen[e]);
    }
}

void replace_tails(gb_system *S, gb_echelon *E, const std::vector<uint32_t> &elems,
                   std::vector<uint32_t> &off, std::vector<uint8_t> &exps, std::vector<uint32_t> &cf) {
    // the reduced tail of element elems[i] is row i of D'; its leading monomial is kept
    cudaStream_t st = S->stream;
    const uint32_t nC = E->nC, nb = E->nb, n = S->n;
    gb_macaulay *Mac = E->mac;
    std::vector<uint32_t> D((size_t)nC * nb);
    std::vector<uint32_t> npcols(nb);
    std::vector<uint4> dict(Mac->ndict);
    if (nC && nb) GB_CUDA(cudaMemcpyAsync(D.data(), E->dprime.p, 4ull * nC * nb, cudaMemcpyDeviceToHost, st));
    if (nb) GB_CUDA(cudaMemcpyAsync(npcols.data(), Mac->nonpiv.p, 4ull * nb, cudaMemcpyDeviceToHost, st));
    if (Mac->ndict) GB_CUDA(cudaMemcpyAsync(dict.data(), Mac->dict.p, 16ull * Mac->ndict, cudaMemcpyDeviceToHost, st));
    sync(S);
    off.assign(1, 0);
    exps.clear();
    cf.clear();
    for (uint32_t i = 0; i < elems.size(); ++i) {
        const Mono &l = S->lm[elems[i]];
        exps.insert(exps.end(), l.e, l.e + n);
        cf.push_back(1);
        if (i < nC)
            for (uint32_t j = 0; j < nb; ++j) {
                const uint32_t v = D[(size_t)i * nb + j];
                if (!v) continue;
                const uint8_t *e = reinterpret_cast<const uint8_t *>(&dict[npcols[j]]);
                exps.insert(exps.end(), e, e + n);
                cf.push_back(v);
            }
        off.push_back((uint32_t)cf.size());
    }
}

}  // namespace gb
