// sp.cu -- symbolic preprocessing SP : batch -> (T, R, Pi) (Def. 5.2) as the two-pass FBSP
// pipeline (the algorithm of Sec. 10), with the one-step reduction closure of Rem. 3.3 run as
// bulk frontier rounds (Sec. 7.2).
//
// Keys.  Every monomial of the batch has degree <= D (the step degree), so its dense grevlex rank
// (device.cuh) lies in [0, C(n + D, n)).  Setification + ordering of T (Sec. 5.1) is then a
// single-pass counting sort: a bitmap over the rank space (L2-resident, a few MB at most for the
// sizes this library admits) is marked with atomicOr, and the dictionary column of a rank is the
// number of marked ranks above it (word popcounts + one exclusive scan).  A newly set bit is also
// the "new monomial" test of the frontier: the atomicOr that flips it pushes the monomial once.
//
// Passes.
//   1. mark the leading monomials of the given rows (they start in Done: no reducer rows for them)
//   2. expand the given rows: every term t*m is marked; unmarked ones join the frontier queue
//   3. closure rounds: for each frontier monomial, the oldest non-redundant g with LM(g) | m gives
//      the reducer row (m / LM(g), g), whose tail is expanded into the next frontier
//   4. dictionary: popcount scan, columns, dictionary monomials scattered to their columns
//   5. row order: pivot rows by leading column (a scan over the pivot-column flags), then the
//      non-pivot given rows in the order the host fixed
//   6. CSR: count (row lengths) -> exclusive scan (row_ptr) -> fill (col_ind, val) (the race-freedom theorem of Sec. 11:
//      every row writes its own segment [row_ptr[i], row_ptr[i+1]))
#include <algorithm>

#include "internal.hpp"

namespace gb {

namespace {

constexpr uint32_t FLAG_PIVOT = 1u, FLAG_REDUCER = 2u, FLAG_TAIL = 4u;
constexpr int WPB = 8;  // warps per block in the warp-per-row kernels

struct Basis {
    const uint4 *mon;
    const uint32_t *cf;
    const uint32_t *off;
    const uint32_t *len;
};

struct Keys {
    uint32_t *bits;        // rank bitmap
    const uint32_t *tab;   // rank table (global; copied to shared memory per block)
    int n, D1, tabsz;
};

struct Queue {
    uint4 *mon;
    uint32_t *rank;
    uint32_t cap;
};

struct Counters {  // device-side counters read back after each round
    uint32_t q;    // frontier monomials pushed (all rounds)
    uint32_t red;  // reducer rows
    unsigned long long red_nnz;
    uint32_t err;
    uint32_t pad;
};

__device__ __forceinline__ void load_tab(uint32_t *sm, const Keys &K) {
    for (int i = threadIdx.x; i < K.tabsz; i += blockDim.x) sm[i] = K.tab[i];
    __syncthreads();
}

// mark rank r; true if this call flipped the bit (the monomial is new)
__device__ __forceinline__ bool test_and_set(uint32_t *bits, uint32_t r) {
    const uint32_t w = r >> 5, b = 1u << (r & 31);
    if (bits[w] & b) return false;  // bits only ever get set during a step: a set bit is final
    return !(atomicOr(&bits[w], b) & b);
}

// warp-aggregated append of the lanes' new monomials to the frontier queue
__device__ __forceinline__ void push_new(bool isnew, uint4 m, uint32_t r, const Queue &Q,
                                         Counters *C) {
    const unsigned mask = __ballot_sync(0xffffffffu, isnew);
    if (!mask) return;
    const int lane = threadIdx.x & 31, leader = __ffs(mask) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(&C->q, (uint32_t)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (isnew) {
        const uint32_t pos = base + __popc(mask & ((1u << lane) - 1u));
        if (pos < Q.cap) {
            Q.mon[pos] = m;
            Q.rank[pos] = r;
        }
    }
}

// expand terms [j0, len) of t*g into the bitmap / queue; called by a whole warp
__device__ __forceinline__ void expand_terms(uint4 t, uint32_t off, uint32_t j0, uint32_t len,
                                             const Basis &B, const Keys &K, const uint32_t *tab,
                                             const Queue &Q, Counters *C) {
    const int lane = threadIdx.x & 31;
    for (uint32_t jb = j0; jb < len; jb += 32) {
        const uint32_t j = jb + lane;
        bool isnew = false;
        uint4 m = make_uint4(0, 0, 0, 0);
        uint32_t r = 0;
        if (j < len) {
            m = mono_mul(t, B.mon[off + j]);
            r = mono_rank(m, tab, K.n, K.D1);
            isnew = test_and_set(K.bits, r);
        }
        push_new(isnew, m, r, Q, C);
    }
}

// Pass 1: leading monomials of the given rows (tail rows have none)
__global__ void k_mark_given(uint32_t nrows, const uint4 *__restrict__ rt,
                             const uint32_t *__restrict__ rk, const uint8_t *__restrict__ rflags,
                             Basis B, Keys K, uint32_t *__restrict__ lm_rank) {
    extern __shared__ uint32_t tab[];
    load_tab(tab, K);
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrows) return;
    if (rflags[i] & FLAG_TAIL) {
        lm_rank[i] = 0xFFFFFFFFu;
        return;
    }
    const uint4 m = mono_mul(rt[i], B.mon[B.off[rk[i]]]);
    const uint32_t r = mono_rank(m, tab, K.n, K.D1);
    atomicOr(&K.bits[r >> 5], 1u << (r & 31));
    lm_rank[i] = r;
}

// Pass 2: expand the given rows (warp per row)
__global__ void k_expand_given(uint32_t nrows, const uint4 *__restrict__ rt,
                               const uint32_t *__restrict__ rk, const uint8_t *__restrict__ rflags,
                               Basis B, Keys K, Queue Q, Counters *C) {
    extern __shared__ uint32_t tab[];
    load_tab(tab, K);
    const uint32_t row = blockIdx.x * WPB + (threadIdx.x >> 5);
    if (row >= nrows) return;  // whole warp leaves together
    const uint32_t k = rk[row];
    const uint32_t j0 = (rflags[row] & FLAG_TAIL) ? 1u : 0u;
    expand_terms(rt[row], B.off[k], j0, B.len[k], B, K, tab, Q, C);
}

// Pass 3: one closure round over frontier items [f0, f1) (warp per item)
__global__ void k_closure(uint32_t f0, uint32_t f1, Basis B, Keys K, Queue Q, Counters *C,
                          const uint32_t *__restrict__ nr_idx, const uint4 *__restrict__ nr_lm,
                          uint32_t nnr, uint4 *__restrict__ red_t, uint32_t *__restrict__ red_k,
                          uint32_t *__restrict__ red_rank, uint32_t red_cap) {
    extern __shared__ uint32_t tab[];
    load_tab(tab, K);
    const uint32_t item = f0 + blockIdx.x * WPB + (threadIdx.x >> 5);
    if (item >= f1) return;
    const int lane = threadIdx.x & 31;
    const uint4 m = Q.mon[item];
    // oldest non-redundant element whose leading monomial divides m (nr_idx ascending)
    int g = -1;
    uint4 lmg = make_uint4(0, 0, 0, 0);
    for (uint32_t cb = 0; cb < nnr; cb += 32) {
        const uint32_t idx = cb + lane;
        const bool ok = idx < nnr && mono_divides(nr_lm[idx], m);
        const unsigned mask = __ballot_sync(0xffffffffu, ok);
        if (mask) {
            const uint32_t hit = cb + __ffs(mask) - 1;
            g = (int)nr_idx[hit];
            lmg = nr_lm[hit];
            break;
        }
    }
    if (g < 0) return;
    const uint4 t = mono_div(m, lmg);
    const uint32_t len = B.len[g];
    if (lane == 0) {
        const uint32_t pos = atomicAdd(&C->red, 1u);
        if (pos < red_cap) {
            red_t[pos] = t;
            red_k[pos] = (uint32_t)g;
            red_rank[pos] = Q.rank[item];
        }
        atomicAdd(&C->red_nnz, (unsigned long long)len);
    }
    expand_terms(t, B.off[g], 1u, len, B, K, tab, Q, C);
}

__global__ void k_popc(const uint32_t *__restrict__ bits, uint32_t *__restrict__ cnt, uint32_t W) {
    const uint32_t w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w < W) cnt[w] = __popc(bits[w]);
}

struct Dict {
    const uint32_t *bits;
    const uint32_t *wpre;
    uint32_t N;
};

// Pass 4: dictionary monomials to their columns (queue entries, then the given rows' LMs)
__global__ void k_dict_queue(uint32_t q, const uint4 *__restrict__ qmon,
                             const uint32_t *__restrict__ qrank, Dict Dd, uint4 *__restrict__ dict,
                             uint32_t *err) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= q) return;
    const uint32_t c = rank_to_col(qrank[i], Dd.bits, Dd.wpre, Dd.N);
    if (c >= Dd.N) { atomicOr(err, 1u); return; }
    dict[c] = qmon[i];
}

__global__ void k_dict_given(uint32_t nrows, const uint4 *__restrict__ rt,
                             const uint32_t *__restrict__ rk, const uint8_t *__restrict__ rflags,
                             const uint32_t *__restrict__ lm_rank, Basis B, Dict Dd,
                             uint4 *__restrict__ dict, uint32_t *__restrict__ is_piv,
                             uint32_t *__restrict__ src, uint32_t *err) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrows || !(rflags[i] & FLAG_PIVOT)) return;
    const uint32_t c = rank_to_col(lm_rank[i], Dd.bits, Dd.wpre, Dd.N);
    if (c >= Dd.N) { atomicOr(err, 2u); return; }
    dict[c] = mono_mul(rt[i], B.mon[B.off[rk[i]]]);
    is_piv[c] = 1u;
    src[c] = 0x80000000u | i;
}

__global__ void k_piv_reducers(uint32_t nred, const uint32_t *__restrict__ red_rank, Dict Dd,
                               uint32_t *__restrict__ is_piv, uint32_t *__restrict__ src,
                               uint32_t *err) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nred) return;
    const uint32_t c = rank_to_col(red_rank[i], Dd.bits, Dd.wpre, Dd.N);
    if (c >= Dd.N) { atomicOr(err, 4u); return; }
    is_piv[c] = 1u;
    src[c] = i;
}

struct RowsOut {
    uint4 *t;
    uint32_t *k;
    uint8_t *flags;
    uint32_t *pcols, *nonpiv, *colpos;
    uint32_t nA, nb;  // allocated pivot rows / non-pivot columns
    uint32_t *err;
};

// Pass 5a: pivot rows by leading column, and the column maps
__global__ void k_place_pivots(uint32_t N, const uint32_t *__restrict__ is_piv,
                               const uint32_t *__restrict__ pidx, const uint32_t *__restrict__ src,
                               const uint4 *__restrict__ gt, const uint32_t *__restrict__ gk,
                               const uint8_t *__restrict__ gflags, const uint4 *__restrict__ red_t,
                               const uint32_t *__restrict__ red_k, RowsOut O) {
    const uint32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    if (is_piv[c]) {
        const uint32_t r = pidx[c], s = src[c];
        if (r >= O.nA) { atomicOr(O.err, 8u); return; }
        if (s & 0x80000000u) {
            const uint32_t i = s & 0x7FFFFFFFu;
            O.t[r] = gt[i];
            O.k[r] = gk[i];
            O.flags[r] = (uint8_t)(gflags[i] & (FLAG_PIVOT | FLAG_TAIL));
        } else {
            O.t[r] = red_t[s];
            O.k[r] = red_k[s];
            O.flags[r] = (uint8_t)(FLAG_PIVOT | FLAG_REDUCER);
        }
        O.pcols[r] = c;
        O.colpos[c] = r | 0x80000000u;
    } else {
        const uint32_t q = c - pidx[c];
        if (q >= O.nb) { atomicOr(O.err, 16u); return; }
        O.nonpiv[q] = c;
        O.colpos[c] = q;
    }
}

// Pass 5b: non-pivot given rows after the nA pivot rows, in the host's order
__global__ void k_place_nonpivots(uint32_t nrows, uint32_t nA, const uint4 *__restrict__ gt,
                                  const uint32_t *__restrict__ gk,
                                  const uint8_t *__restrict__ gflags,
                                  const uint32_t *__restrict__ np_index, RowsOut O) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrows || np_index[i] == 0xFFFFFFFFu) return;
    const uint32_t r = nA + np_index[i];
    O.t[r] = gt[i];
    O.k[r] = gk[i];
    O.flags[r] = (uint8_t)(gflags[i] & FLAG_TAIL);
}

// Pass 6: count
__global__ void k_row_len(uint32_t nrows, const uint32_t *__restrict__ row_k,
                          const uint8_t *__restrict__ flags, const uint32_t *__restrict__ blen,
                          uint32_t *__restrict__ out) {
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < nrows) out[r] = blen[row_k[r]] - ((flags[r] & FLAG_TAIL) ? 1u : 0u);
}

// Pass 6: fill (warp per row)
__global__ void k_fill(uint32_t nrows, const uint4 *__restrict__ row_t,
                       const uint32_t *__restrict__ row_k, const uint8_t *__restrict__ flags,
                       const uint32_t *__restrict__ row_ptr, Basis B, Keys K, Dict Dd,
                       uint32_t *__restrict__ col, uint32_t *__restrict__ val, uint32_t nnz,
                       uint32_t *err) {
    extern __shared__ uint32_t tab[];
    load_tab(tab, K);
    const uint32_t row = blockIdx.x * WPB + (threadIdx.x >> 5);
    if (row >= nrows) return;
    const int lane = threadIdx.x & 31;
    const uint32_t k = row_k[row];
    const uint32_t skip = (flags[row] & FLAG_TAIL) ? 1u : 0u;
    const uint32_t off = B.off[k] + skip, len = B.len[k] - skip, s = row_ptr[row];
    const uint4 t = row_t[row];
    if (s + len > nnz) {
        if (lane == 0) atomicOr(err, 32u);
        return;
    }
    for (uint32_t j = lane; j < len; j += 32) {
        const uint4 m = mono_mul(t, B.mon[off + j]);
        const uint32_t r = mono_rank(m, tab, K.n, K.D1);
        col[s + j] = rank_to_col(r, Dd.bits, Dd.wpre, Dd.N);
        val[s + j] = B.cf[off + j];
    }
}

inline unsigned blocks(size_t n, unsigned t) { return (unsigned)((n + t - 1) / t); }

uint64_t binom(uint32_t a, uint32_t b) {
    if (b > a) return 0;
    b = std::min(b, a - b);
    unsigned __int128 r = 1;
    for (uint32_t i = 1; i <= b; ++i) r = r * (a - b + i) / i;
    return r > (unsigned __int128)UINT64_MAX ? UINT64_MAX : (uint64_t)r;
}

}  // namespace

std::unique_ptr<gb_macaulay> symbolic_preprocess(gb_system *S, const std::vector<RowSpec> &rows,
                                                 bool closure, const std::vector<uint32_t> &nonred) {
    Arena &ar = S->ctx->arena;
    cudaStream_t st = S->stream;
    const int n = (int)S->n;
    const uint32_t ng = (uint32_t)rows.size();
    auto M = std::make_unique<gb_macaulay>();
    M->sys = S;
    M->n = S->n;
    GB_CUDA(cudaEventRecord(S->ev[0], st));

    // step degree, rank space and the rank table
    uint32_t D = 0;
    for (const RowSpec &r : rows)
        D = std::max<uint32_t>(D, (uint32_t)(mono_deg(r.t, n) + mono_deg(S->lm[r.k], n)));
    M->degree = D;
    const uint64_t space = binom((uint32_t)n + D, (uint32_t)n);
    if (space >= (1ull << 32) - 64)
        fail(GB_EUNSUPPORTED, "monomial space C(n+D, n) above 2^32 for the dense grevlex keys");
    const uint32_t D1 = D + 1, W = (uint32_t)((space + 31) / 32);
    std::vector<uint32_t> tab((size_t)D1 * n);
    for (uint32_t d = 0; d <= D; ++d) tab[d] = (uint32_t)(d ? binom(n + d - 1, n) : 0);
    for (int j = 1; j < n; ++j)
        for (uint32_t s = 0; s <= D; ++s) tab[(size_t)D1 * j + s] = (uint32_t)binom(s + j - 1, j);
    const int tabsz = (int)tab.size();
    const size_t tab_smem = sizeof(uint32_t) * tabsz;

    // given rows and the non-redundant list, staged through pinned memory
    std::vector<uint32_t> np_index(ng, 0xFFFFFFFFu);
    uint32_t npiv_given = 0, nnp = 0;
    uint64_t nnz_given = 0;
    for (uint32_t i = 0; i < ng; ++i) {
        if (rows[i].pivot) ++npiv_given;
        else np_index[i] = nnp++;
        nnz_given += S->len[rows[i].k] - rows[i].skip;
    }
    const uint32_t nnr = (uint32_t)nonred.size();
    const size_t stage = sizeof(uint4) * ng + 4 * ng + ng + 4 * ng + 4 * (size_t)tabsz +
                         4 * nnr + sizeof(uint4) * nnr + 256 * 8;
    char *h = static_cast<char *>(pinned(S, stage));
    size_t o = 0;
    auto put = [&](const void *src, size_t bytes) {
        o = (o + 15) & ~size_t(15);
        std::memcpy(h + o, src, bytes);
        size_t at = o;
        o += bytes;
        return at;
    };
    std::vector<uint4> gt(ng);
    std::vector<uint32_t> gk(ng);
    std::vector<uint8_t> gf(ng);
    std::vector<uint4> nlm(nnr);
    for (uint32_t i = 0; i < ng; ++i) {
        gt[i] = to_u4(rows[i].t);
        gk[i] = rows[i].k;
        gf[i] = (uint8_t)((rows[i].pivot ? FLAG_PIVOT : 0u) | (rows[i].skip ? FLAG_TAIL : 0u));
    }
    for (uint32_t i = 0; i < nnr; ++i) nlm[i] = to_u4(S->lm[nonred[i]]);
    const size_t o_gt = put(gt.data(), sizeof(uint4) * ng), o_gk = put(gk.data(), 4 * ng),
                 o_gf = put(gf.data(), ng), o_np = put(np_index.data(), 4 * ng),
                 o_tab = put(tab.data(), 4 * (size_t)tabsz), o_nri = put(nonred.data(), 4 * nnr),
                 o_nrl = put(nlm.data(), sizeof(uint4) * nnr);
    DBuf<char> dstage;
    dstage.alloc(ar, o, st);
    GB_CUDA(cudaMemcpyAsync(dstage.p, h, o, cudaMemcpyHostToDevice, st));
    const uint4 *d_gt = reinterpret_cast<const uint4 *>(dstage.p + o_gt);
    const uint32_t *d_gk = reinterpret_cast<const uint32_t *>(dstage.p + o_gk);
    const uint8_t *d_gf = reinterpret_cast<const uint8_t *>(dstage.p + o_gf);
    const uint32_t *d_np = reinterpret_cast<const uint32_t *>(dstage.p + o_np);
    const uint32_t *d_tab = reinterpret_cast<const uint32_t *>(dstage.p + o_tab);
    const uint32_t *d_nri = reinterpret_cast<const uint32_t *>(dstage.p + o_nri);
    const uint4 *d_nrl = reinterpret_cast<const uint4 *>(dstage.p + o_nrl);

    Basis B{S->bmon.p, S->bcf.p, S->boff.p, S->blen.p};
    DBuf<uint32_t> bits, lm_rank;
    bits.alloc(ar, W, st);
    lm_rank.alloc(ar, ng, st);
    DBuf<Counters> cnt;
    cnt.alloc(ar, 1, st);
    Keys K{bits.p, d_tab, n, (int)D1, tabsz};

    // queue and reducer-row capacity: start from an estimate, restart larger on overflow
    uint64_t cap = std::min<uint64_t>(space, std::max<uint64_t>(1u << 16, 8ull * nnz_given / 4));
    DBuf<uint4> qmon, red_t;
    DBuf<uint32_t> qrank, red_k, red_rank;
    Counters hc{};
    uint32_t rounds = 0;
    for (int attempt = 0;; ++attempt) {
        qmon.alloc(ar, cap, st);
        qrank.alloc(ar, cap, st);
        red_t.alloc(ar, cap, st);
        red_k.alloc(ar, cap, st);
        red_rank.alloc(ar, cap, st);
        Queue Q{qmon.p, qrank.p, (uint32_t)cap};
        GB_CUDA(cudaMemsetAsync(bits.p, 0, 4ull * W, st));
        GB_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(Counters), st));
        if (ng) {
            k_mark_given<<<blocks(ng, 256), 256, tab_smem, st>>>(ng, d_gt, d_gk, d_gf, B, K, lm_rank.p);
            counted();
            k_expand_given<<<blocks(ng, WPB), 32 * WPB, tab_smem, st>>>(ng, d_gt, d_gk, d_gf, B, K, Q, cnt.p);
            counted();
            GB_CUDA(cudaGetLastError());
        }
        uint32_t f0 = 0;
        rounds = 0;
        Counters *hcp = reinterpret_cast<Counters *>(h + ((o + 255) & ~size_t(255)));
        bool overflow = false;
        for (;;) {
            GB_CUDA(cudaMemcpyAsync(hcp, cnt.p, sizeof(Counters), cudaMemcpyDeviceToHost, st));
            sync(S);
            hc = *hcp;
            if (hc.q > cap || hc.red > cap) { overflow = true; break; }
            if (!closure || hc.q == f0 || nnr == 0) break;
            const uint32_t f1 = hc.q;
            k_closure<<<blocks(f1 - f0, WPB), 32 * WPB, tab_smem, st>>>(
                f0, f1, B, K, Q, cnt.p, d_nri, d_nrl, nnr, red_t.p, red_k.p, red_rank.p, (uint32_t)cap);
            counted();
            GB_CUDA(cudaGetLastError());
            ++rounds;
            f0 = f1;
        }
        if (!overflow) break;
        if (cap >= space) fail(GB_EDEVICE, "frontier queue overflow beyond the monomial space");
        cap = std::min<uint64_t>(space, 2ull * std::max<uint64_t>(hc.q, hc.red));
    }
    M->closure_rounds = rounds;

    const uint32_t nq = hc.q, nred = hc.red;
    const uint32_t N = npiv_given + nq;
    const uint32_t nA = nred + npiv_given, nrows = ng + nred;
    const uint64_t nnz = nnz_given + hc.red_nnz;
    if (nnz >= (1ull << 32)) fail(GB_EUNSUPPORTED, "more than 2^32 nonzeros in one matrix");
    M->ndict = N;
    M->nA = nA;
    M->nC = nnp;
    M->nb = N - nA;
    M->nrows = nrows;
    M->nnz = nnz;

    // dictionary
    DBuf<uint32_t> wcnt, wpre;
    wcnt.alloc(ar, W, st);
    wpre.alloc(ar, (size_t)W + 1, st);
    k_popc<<<blocks(W, 256), 256, 0, st>>>(bits.p, wcnt.p, W);
    counted();
    exclusive_scan(ar, wcnt.p, wpre.p, W, st);
    Dict Dd{bits.p, wpre.p, N};
    M->dict.alloc(ar, N, st);
    DBuf<uint32_t> is_piv, src, pidx;
    is_piv.alloc(ar, N, st);
    src.alloc(ar, N, st);
    pidx.alloc(ar, (size_t)N + 1, st);
    GB_CUDA(cudaMemsetAsync(is_piv.p, 0, 4ull * N, st));
    uint32_t *derr = &cnt.p->err;
    if (nq) {
        k_dict_queue<<<blocks(nq, 256), 256, 0, st>>>(nq, qmon.p, qrank.p, Dd, M->dict.p, derr);
        counted();
    }
    if (ng) {
        k_dict_given<<<blocks(ng, 256), 256, 0, st>>>(ng, d_gt, d_gk, d_gf, lm_rank.p, B, Dd,
                                                      M->dict.p, is_piv.p, src.p, derr);
        counted();
    }
    if (nred) {
        k_piv_reducers<<<blocks(nred, 256), 256, 0, st>>>(nred, red_rank.p, Dd, is_piv.p, src.p, derr);
        counted();
    }
    GB_CUDA(cudaGetLastError());
    exclusive_scan(ar, is_piv.p, pidx.p, N, st);

    // rows
    M->row_t.alloc(ar, nrows, st);
    M->row_k.alloc(ar, nrows, st);
    M->row_flags.alloc(ar, nrows, st);
    M->pcols.alloc(ar, nA, st);
    M->nonpiv.alloc(ar, M->nb, st);
    M->colpos.alloc(ar, N, st);
    RowsOut O{M->row_t.p, M->row_k.p, M->row_flags.p, M->pcols.p, M->nonpiv.p, M->colpos.p,
              nA, M->nb, derr};
    if (N) {
        k_place_pivots<<<blocks(N, 256), 256, 0, st>>>(N, is_piv.p, pidx.p, src.p, d_gt, d_gk, d_gf,
                                                       red_t.p, red_k.p, O);
        counted();
    }
    if (ng) {
        k_place_nonpivots<<<blocks(ng, 256), 256, 0, st>>>(ng, nA, d_gt, d_gk, d_gf, d_np, O);
        counted();
    }
    GB_CUDA(cudaGetLastError());

    // CSR: count -> scan -> fill
    DBuf<uint32_t> lens;
    lens.alloc(ar, nrows, st);
    M->row_ptr.alloc(ar, (size_t)nrows + 1, st);
    M->col.alloc(ar, nnz, st);
    M->val.alloc(ar, nnz, st);
    if (nrows) {
        k_row_len<<<blocks(nrows, 256), 256, 0, st>>>(nrows, M->row_k.p, M->row_flags.p, S->blen.p, lens.p);
        counted();
    }
    exclusive_scan(ar, lens.p, M->row_ptr.p, nrows, st);
    if (nrows) {
        k_fill<<<blocks(nrows, WPB), 32 * WPB, tab_smem, st>>>(nrows, M->row_t.p, M->row_k.p,
                                                               M->row_flags.p, M->row_ptr.p, B, K, Dd,
                                                               M->col.p, M->val.p, (uint32_t)nnz, derr);
        counted();
    }
    GB_CUDA(cudaGetLastError());
    GB_CUDA(cudaEventRecord(S->ev[1], st));

    // consistency of the plan with the host's counts (one small read-back)
    uint32_t *chk = reinterpret_cast<uint32_t *>(h + ((o + 255) & ~size_t(255)) + 256);
    GB_CUDA(cudaMemcpyAsync(chk, wpre.p + W, 4, cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaMemcpyAsync(chk + 1, pidx.p + N, 4, cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaMemcpyAsync(chk + 2, M->row_ptr.p + nrows, 4, cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaMemcpyAsync(chk + 3, derr, 4, cudaMemcpyDeviceToHost, st));
    sync(S);
    if (chk[0] != N || chk[1] != nA || chk[2] != (uint32_t)nnz || chk[3])
        fail(GB_EDEVICE, "symbolic preprocessing: device counts disagree with the plan (flags " +
                             std::to_string(chk[3]) + ")");
    GB_CUDA(cudaEventElapsedTime(&M->ms_sp, S->ev[0], S->ev[1]));
    return M;
}

}  // namespace gb
