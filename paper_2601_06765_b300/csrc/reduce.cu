// reduce.cu -- the numeric phase (Sec. 9.2): structured elimination of Macaulay matrices, for
// many independent jobs (systems) at once.
//
// Rows of Pi come as nA pivot rows (distinct leading columns pcols[0..nA), ascending, every row
// monic) followed by nC non-pivot rows.  The results are unique (the pivot rows have distinct
// leading columns), so any schedule on the device gives the same bits as the CPU oracle.
//
//   k_reduce   each non-pivot row is reduced by the pivot rows into a dense accumulator -> D'
//   rref_*     RREF(D') by right-looking panels of KP rows
//   append     echelon rows become new basis elements in the device basis (Sec. 4.2 step 4)
//   tails      the final reduction's rows become the reduced basis, packed on the device
// Every kernel serves all jobs of a launch: a prefix table maps a block to its job.
#include <algorithm>
#include <cstdlib>

#include <cooperative_groups.h>

#include <chrono>
#include <cstdio>

#include "internal.hpp"

namespace gb {

namespace {

constexpr int RT = 256;  // threads per block of the row-reduction kernel

inline unsigned blocks(size_t n, unsigned t) { return (unsigned)((n + t - 1) / t); }

// ---- sparse reduction of the non-pivot rows (PSGE trailing update, Sec. 9.2) -------------------
//
// The pivot columns are taken in chunks of CW = 32 consecutive pivots (pivot rows k..k+31, one
// contiguous CSR segment).  For a non-pivot row v the multipliers of a chunk are the solution of a
// 32 x 32 unit upper-triangular system f U = v_c, i.e. f_i = v[c_i] - sum_{j<i} f_j U[j][i], where
// U[j][i] is the entry of pivot row j at pivot column c_i.  U^{-1} is computed once per chunk
// (k_invert_chunk_tri), so the solve is the product f = v_c U^{-1}: every lane forms one
// multiplier from 32 independent products instead of a 32-step dependent chain.  Warp 0 does it
// from a shared copy of U^{-1} (prefetched by the other warps during the previous chunk); then
// every warp applies v <- v - sum_i f_i (pivot row i) to the row's accumulator with shared-memory
// atomics (each pivot row's own leading entry included, which leaves v[c_i] = 0).  Two block
// barriers per 32 pivot columns instead of one per column.
//
// Accumulators are lazy (Rem. 8.1), in one of three modes:
//   A32: p < 2^16, each product (p - f) v < 2^32 is Barrett-reduced to [0, p) and added to a 32-bit
//        sum (exact while a column takes fewer than 2^16 updates: the host requires nA < 2^16;
//        k_reduce_rows reduces each product only to [0, 2p) and takes nA < 2^15);
//   A64: p < 2^16, the raw products are added to a 64-bit sum (no reduction per update);
//   M64: p < 2^31, the Montgomery product redc(fR * v) in [0, 2p) is added to a 64-bit sum; only
//        the multiplier is converted (once per pivot row), the entries stay in standard form.
// Entries are reduced (Barrett) when read.
constexpr int CW = 32;
enum AccMode { A32 = 0, A64 = 1, M64 = 2 };
template <int MODE>
struct AccOf { using type = unsigned long long; };
template <>
struct AccOf<A32> { using type = uint32_t; };

struct RedJob {
    const uint32_t *row_ptr, *col, *val, *pcols, *colpos, *nonpiv;
    uint32_t *U, *dprime;
    void *gacc;                // global accumulators, one row of N per block, when shared memory is short
    uint32_t *split;           // k_reduce_cl: per pivot row, the first entry of each block's column range
    unsigned long long *work;  // [0] pivot rows applied, [1] modular multiply-adds
    uint32_t nA, nC, N, nb;
    Fp fp;
    uint32_t rpb, win;         // k_reduce_rows: rows per block, entries of the staging window
};

// U[chunk][j][i] for j < i: entry of pivot row chunk*32+j at pivot column pcols[chunk*32+i]
// (warp per pivot row, 8 per block)
__global__ void k_build_chunk_tri(const RedJob *__restrict__ jobs, const uint32_t *__restrict__ bstart, int nj) {
    const int jb = job_of_block(bstart, nj);
    const RedJob &J = jobs[jb];
    const uint32_t k = (blockIdx.x - bstart[jb]) * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (k >= J.nA) return;
    const int lane = threadIdx.x & 31;
    const uint32_t chunk = k / CW, j = k % CW;
    const uint32_t last = J.pcols[min(chunk * CW + CW, J.nA) - 1];
    uint32_t *Uc = J.U + (size_t)chunk * CW * CW + (size_t)j * CW;
    const uint32_t a = J.row_ptr[k] + 1, b = J.row_ptr[k + 1];
    for (uint32_t q0 = a; q0 < b; q0 += 32) {
        const uint32_t q = q0 + lane;
        bool past = true;
        if (q < b) {
            const uint32_t c = J.col[q];
            past = c > last;
            if (!past) {
                const uint32_t cp = J.colpos[c];
                if ((cp & 0x80000000u) && (cp & 0x7FFFFFFFu) / CW == chunk) Uc[(cp & 0x7FFFFFFFu) % CW] = J.val[q];
            }
        }
        if (__all_sync(0xffffffffu, past)) break;  // columns ascend: the rest lies past the chunk
    }
}

// U^{-1} of every chunk triangle, in place (warp per chunk, IW per block).  With W = U^{-1} (unit
// upper triangular): W[j][i] = -sum_{k=j}^{i-1} W[j][k] U[k][i] for j < i, a column at a time.
// Stored row-major with W[i][i] = 1 and zeros below the diagonal; in Montgomery form (W R mod p)
// when p >= 2^16, so that k_reduce can add redc(v W') terms, each below 2p, in 64 bits.
constexpr int IW = 4;
constexpr int TS = CW + 1;  // padded shared-memory row stride
__global__ void __launch_bounds__(IW * 32) k_invert_chunk_tri(const RedJob *__restrict__ jobs,
                                                             const uint32_t *__restrict__ bstart, int nj) {
    __shared__ uint32_t Us[IW][CW * TS], Ws[IW][CW * TS];
    const int jb = job_of_block(bstart, nj);
    const RedJob &J = jobs[jb];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t chunk = (blockIdx.x - bstart[jb]) * IW + warp;
    if (chunk >= (J.nA + CW - 1) / CW) return;  // whole warp leaves together
    const Fp fp = J.fp;
    uint32_t *Ug = J.U + (size_t)chunk * CW * CW;
    uint32_t *U = Us[warp], *W = Ws[warp];
    for (int r = 0; r < CW; ++r) {
        U[r * TS + lane] = Ug[r * CW + lane];
        W[r * TS + lane] = r == lane ? 1u : 0u;
    }
    __syncwarp();
    // the sums are kept lazily in 64 bits and reduced once per entry: below 31 * 2^32 for p < 2^16
    // (raw products of two residues), below 31 p for larger p (each product reduced)
    for (int i = 1; i < CW; ++i) {
        if (lane < i) {
            uint64_t acc = 0;
            if (fp.small) {
                for (int k = lane; k < i; ++k) acc += (uint64_t)(W[lane * TS + k] * U[k * TS + i]);
            } else {
                for (int k = lane; k < i; ++k) {
                    const uint32_t u = U[k * TS + i];
                    if (u) acc += fp_mul(W[lane * TS + k], u, fp);
                }
            }
            const uint32_t sum = fp_reduce(acc, fp);
            W[lane * TS + i] = sum ? fp.p - sum : 0u;
        }
        __syncwarp();
    }
    for (int r = 0; r < CW; ++r) {
        const uint32_t w = W[r * TS + lane];
        Ug[r * CW + lane] = fp.small ? w : fp_to_mont(w, fp);
    }
}

// block per non-pivot row of some job
template <int MODE, bool SMEM>
__global__ void __launch_bounds__(RT, 6) k_reduce(const RedJob *__restrict__ jobs, const uint32_t *__restrict__ bstart, int nj) {
    using Acc = typename AccOf<MODE>::type;
    constexpr bool SMALLP = MODE != M64;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint32_t Us[2][CW * CW];
    // the chunk's pivot rows with a non-zero multiplier, as segments of its CSR range: first entry,
    // multiplier (Montgomery form for p >= 2^16) and the exclusive prefix of the segment lengths
    __shared__ uint32_t seg_q[CW], seg_m[CW], seg_pre[CW + 1];
    __shared__ uint32_t s_nseg;
    const int jb = job_of_block(bstart, nj);
    const RedJob &J = jobs[jb];
    const Fp fp = J.fp;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t i = blockIdx.x - bstart[jb], row = J.nA + i;
    if (i >= J.nC) return;  // the whole block: a job emptied after a failed input check
    const uint32_t a0 = J.row_ptr[row], b0 = J.row_ptr[row + 1];
    const uint32_t base = a0 < b0 ? J.col[a0] : J.N, width = J.N - base;
    Acc *acc = SMEM ? reinterpret_cast<Acc *>(smem_raw)
                    : reinterpret_cast<Acc *>(J.gacc) + (size_t)i * J.N;
    for (uint32_t j = threadIdx.x; j < width; j += RT) acc[j] = 0;
    __syncthreads();
    for (uint32_t q = a0 + threadIdx.x; q < b0; q += RT) acc[J.col[q] - base] = J.val[q];
    // first chunk holding a pivot column >= base
    uint32_t lo = 0, hi = J.nA;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (J.pcols[mid] < base) lo = mid + 1; else hi = mid;
    }
    const uint32_t k0 = (lo / CW) * CW;
    if (k0 < J.nA)
        for (uint32_t t = threadIdx.x; t < CW * CW; t += RT) Us[0][t] = J.U[(size_t)(k0 / CW) * CW * CW + t];
    unsigned long long applied = 0, fmas = 0;
    for (uint32_t kc = k0, buf = 0; kc < J.nA; kc += CW, buf ^= 1) {
        const uint32_t cnt = min((uint32_t)CW, J.nA - kc);
        __syncthreads();  // the previous chunk's updates (and this chunk's U) are visible
        if (warp == 0) {
            // phase A: the chunk's multipliers f = v_c U^{-1}.  Lanes past cnt hold v = 0, and a
            // pivot column left of base has v = 0 as do all columns before it, so its f is 0.
            uint32_t x = 0;
            if ((uint32_t)lane < cnt) {
                const uint32_t c = J.pcols[kc + lane];
                if (c >= base) x = MODE == A32 ? fp_reduce32((uint32_t)acc[c - base], fp) : fp_reduce(acc[c - base], fp);
            }
            const uint32_t *Wc = Us[buf];
            unsigned long long s = 0;  // < 32 * 2^32 (p < 2^16) or < 32 * 2p (Montgomery terms)
#pragma unroll
            for (int j = 0; j < CW; ++j) {
                const uint32_t vj = __shfl_sync(0xffffffffu, x, j);
                const uint32_t w = Wc[j * CW + lane];
                if (SMALLP) s += (unsigned long long)(vj * w);
                else s += fp_redc((uint64_t)vj * w, fp);
            }
            const uint32_t f = (uint32_t)lane < cnt ? fp_reduce(s, fp) : 0u;
            const unsigned nzmask = __ballot_sync(0xffffffffu, f != 0u);
            uint32_t q0 = 0, len = 0;
            if (f) {
                q0 = J.row_ptr[kc + lane];
                len = J.row_ptr[kc + lane + 1] - q0;
            }
            uint32_t end = len;  // inclusive prefix of the lengths over the lanes
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, end, d);
                if (lane >= d) end += y;
            }
            if (f) {
                const uint32_t pos = __popc(nzmask & ((1u << lane) - 1u));
                seg_q[pos] = q0;
                seg_m[pos] = SMALLP ? fp.p - f : fp_to_mont(fp.p - f, fp);
                seg_pre[pos + 1] = end;
            }
            const uint32_t total = __shfl_sync(0xffffffffu, end, 31);
            if (lane == 0) {
                seg_pre[0] = 0;
                s_nseg = __popc(nzmask);
                applied += __popc(nzmask);
                fmas += total;
            }
        } else {
            // the other warps prefetch the next chunk's triangle
            const uint32_t kn = kc + CW;
            if (kn < J.nA)
                for (uint32_t t = threadIdx.x - 32u; t < CW * CW; t += RT - 32u)
                    Us[buf ^ 1][t] = J.U[(size_t)(kn / CW) * CW * CW + t];
        }
        __syncthreads();
        // phase B: the segments' entries, flattened, split evenly over the warps (a multiple of 32
        // entries each), four entries per lane in flight.  A lane finds the segment of its first
        // entry by binary search and then only moves forward; the current segment's end, CSR offset
        // and multiplier stay in registers, so the common case costs one compare.
        const uint32_t nseg = s_nseg, total = seg_pre[nseg];
        const uint32_t per = (total + RT - 1) / RT * 32;
        const uint32_t w0 = min(warp * per, total), w1 = min(w0 + per, total);
        uint32_t sg = 0, send = 0, soff = 0, smul = 0;
        if (w0 + lane < w1) {
            uint32_t lo = 0, hi = nseg - 1;  // last segment starting at or before w0 + lane
            while (lo < hi) {
                const uint32_t mid = (lo + hi + 1) >> 1;
                if (seg_pre[mid] <= w0 + lane) lo = mid; else hi = mid - 1;
            }
            sg = lo;
            send = seg_pre[sg + 1];
            soff = seg_q[sg] - seg_pre[sg];
            smul = seg_m[sg];
        }
        for (uint32_t x0 = w0; x0 < w1; x0 += 4 * 32) {
            uint32_t cc[4], vv[4], mm[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t x = x0 + 32u * u + lane;
                cc[u] = 0xFFFFFFFFu;
                vv[u] = mm[u] = 0u;
                if (x < w1) {
                    while (x >= send) {  // stops below nseg: x < seg_pre[nseg]
                        ++sg;
                        send = seg_pre[sg + 1];
                        soff = seg_q[sg] - seg_pre[sg];
                        smul = seg_m[sg];
                    }
                    cc[u] = J.col[soff + x];
                    vv[u] = J.val[soff + x];
                    mm[u] = smul;
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (cc[u] == 0xFFFFFFFFu) continue;
                Acc *dst = acc + (cc[u] - base);
                if (MODE == A32)
                    atomicAdd(reinterpret_cast<uint32_t *>(dst), fp_reduce32(mm[u] * vv[u], fp));
                else if (MODE == A64)
                    atomicAdd(reinterpret_cast<unsigned long long *>(dst), (unsigned long long)(mm[u] * vv[u]));
                else
                    atomicAdd(reinterpret_cast<unsigned long long *>(dst),
                              (unsigned long long)fp_redc((uint64_t)mm[u] * vv[u], fp));
            }
        }
    }
    __syncthreads();
    if (lane == 0 && (applied || fmas)) {
        atomicAdd(&J.work[0], applied);
        atomicAdd(&J.work[1], fmas);
    }
    uint32_t *out = J.dprime + (size_t)i * J.nb;
    for (uint32_t jj = threadIdx.x; jj < J.nb; jj += RT) {
        const uint32_t c = J.nonpiv[jj];
        out[jj] = c < base ? 0u : MODE == A32 ? fp_reduce32((uint32_t)acc[c - base], fp) : fp_reduce(acc[c - base], fp);
    }
}

// ---- the same reduction with several rows per block sharing the pivot entries ------------------
//
// With more non-pivot rows than SMs and a dictionary short enough for the A32 accumulators of R
// rows to sit in shared memory, one block of RB threads reduces R rows at once.  The entries of a
// chunk's pivot rows are one contiguous CSR range: they are staged in shared memory with 16-byte
// asynchronous copies, issued before the chunk's multipliers are formed so that the copy overlaps
// that step (R warps form the R rows' multipliers in parallel, the other warps load the next
// chunk's inverse triangle).  The staged entries are then applied to every row of the block with
// a non-zero multiplier for their pivot row, so the global reads per multiply-add fall by up to R:
// each (pivot row, block row) pair with a non-zero multiplier goes to one warp, whose lanes walk
// that pivot row's staged entries together (every lane does the same work; a lane per entry with
// a loop over the entry's rows left lanes idle whenever the rows' counts differed).  A chunk
// longer than the staging window is applied window by window.
constexpr int RB = 1024;             // threads per block
constexpr uint32_t RMAX = 16;        // rows per block at most
constexpr uint32_t WMIN = 4096;      // entries of the smallest staging window
// The update adds each product reduced only to [0, 2p) (Barrett with k = 32 without its final
// correction): a column's 32-bit sum, below p + nA (2p - 1), stays exact for nA < 2^15 pivots.
constexpr uint32_t ROWS_MAX_PIVOTS = 1u << 15;
__device__ __forceinline__ uint32_t fp_reduce32_2p(uint32_t x, const Fp &f) {
    return x - __umulhi(x, f.mu32) * f.p;  // x mod p, or x mod p + p
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__global__ void __launch_bounds__(RB, 1) k_reduce_rows(const RedJob *__restrict__ jobs, const uint32_t *__restrict__ bstart, int nj) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint32_t Us[2][CW * CW];
    __shared__ uint32_t s_pc[2][CW], s_rp[2][CW + 1];
    // per chunk row k: the block rows with a non-zero multiplier, as s_cnt[.][k] words
    // (r << 16) | (p - f) in s_list[k] (p < 2^16), in no particular order
    __shared__ uint32_t s_list[CW][RMAX], s_cnt[2][CW];
    __shared__ uint32_t s_base;
    const int jb = job_of_block(bstart, nj);
    const RedJob &J = jobs[jb];
    const Fp fp = J.fp;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t R = J.rpb, NS = (J.N + 3u) & ~3u, win = J.win;
    const uint32_t i0 = (blockIdx.x - bstart[jb]) * R, nr = min(R, J.nC - i0);
    // shared memory: R accumulator rows of NS words, then the staged columns and values
    uint32_t *acc = reinterpret_cast<uint32_t *>(smem_raw);
    uint32_t *wcol = acc + (size_t)R * NS, *wval = wcol + win + 8;
    const uint32_t wcol_s = (uint32_t)__cvta_generic_to_shared(wcol), wval_s = (uint32_t)__cvta_generic_to_shared(wval);
    for (uint32_t t = threadIdx.x; t < nr * NS; t += RB) acc[t] = 0;
    if (threadIdx.x < CW) s_cnt[0][threadIdx.x] = 0;
    if (threadIdx.x == 0) s_base = J.N;
    __syncthreads();
    for (uint32_t r = 0; r < nr; ++r) {
        const uint32_t a0 = J.row_ptr[J.nA + i0 + r], b0 = J.row_ptr[J.nA + i0 + r + 1];
        if (threadIdx.x == 0 && a0 < b0) atomicMin(&s_base, J.col[a0]);
        for (uint32_t q = a0 + threadIdx.x; q < b0; q += RB) acc[r * NS + J.col[q]] = J.val[q];
    }
    __syncthreads();
    // first chunk holding a pivot column at or right of the leftmost leading column of the rows
    const uint32_t base = s_base;
    uint32_t lo = 0, hi = J.nA;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (J.pcols[mid] < base) lo = mid + 1; else hi = mid;
    }
    const uint32_t k0 = (lo / CW) * CW;
    // a chunk's inverse triangle, pivot columns and row pointers, by threads t0, t0 + step, ...
    auto load_chunk = [&](uint32_t kc, uint32_t b, uint32_t t0, uint32_t step) {
        const uint32_t cnt = min((uint32_t)CW, J.nA - kc);
        const uint32_t *src = J.U + (size_t)(kc / CW) * CW * CW;
        for (uint32_t t = t0; t < CW * CW; t += step) Us[b][t] = src[t];
        for (uint32_t t = t0; t <= cnt; t += step) {
            if (t < cnt) {
                s_pc[b][t] = J.pcols[kc + t];
                s_cnt[b][t] = 0;
            }
            s_rp[b][t] = J.row_ptr[kc + t];
        }
    };
    // entries [a, b) of the chunk's range into the window (a a multiple of 4); the last piece reads
    // up to three entries past b, inside the CSR arrays' 256-byte-rounded device blocks
    auto stage = [&](uint32_t a, uint32_t b) {
        const uint32_t pieces = (b - a + 3) / 4;
        for (uint32_t q = threadIdx.x; q < pieces; q += RB) {
            cp_async16(wcol_s + 16u * q, J.col + a + 4u * q);
            cp_async16(wval_s + 16u * q, J.val + a + 4u * q);
        }
        cp_async_commit();
    };
    if (k0 < J.nA) load_chunk(k0, 0, threadIdx.x, RB);
    unsigned long long applied = 0, fmas = 0;
    for (uint32_t kc = k0, buf = 0; kc < J.nA; kc += CW, buf ^= 1) {
        const uint32_t cnt = min((uint32_t)CW, J.nA - kc);
        __syncthreads();  // the previous chunk is applied; this chunk's tables are visible
        const uint32_t e0 = s_rp[buf][0], e1 = s_rp[buf][cnt];
        stage(e0 & ~3u, min(e0 + win, e1));
        if (warp < nr) {
            // row `warp`: the chunk's multipliers f = v_c U^{-1}, stored as p - f
            const uint32_t x = lane < cnt ? fp_reduce32(acc[warp * NS + s_pc[buf][lane]], fp) : 0u;
            const uint32_t *Wc = Us[buf];
            unsigned long long s = 0;  // < 32 * 2^32
#pragma unroll
            for (int j = 0; j < CW; ++j) s += (unsigned long long)(__shfl_sync(0xffffffffu, x, j) * Wc[j * CW + lane]);
            const uint32_t f = lane < cnt ? fp_reduce(s, fp) : 0u;
            if (f) s_list[lane][atomicAdd(&s_cnt[buf][lane], 1u)] = (warp << 16) | (fp.p - f);
            uint32_t len = f ? s_rp[buf][lane + 1] - s_rp[buf][lane] : 0u;
#pragma unroll
            for (int d = 16; d; d >>= 1) len += __shfl_xor_sync(0xffffffffu, len, d);
            applied += __popc(__ballot_sync(0xffffffffu, f != 0u));
            fmas += len;
        } else if (kc + CW < J.nA) {
            load_chunk(kc + CW, buf ^ 1, threadIdx.x - 32u * nr, RB - 32u * nr);
        }
        cp_async_wait0();
        __syncthreads();
        // the chunk's (pivot row, block row) pairs with a non-zero multiplier: pair q is the
        // (q - pre[k])-th block row of chunk row k, pre the exclusive prefix of the counts (every
        // warp scans the 32 counts itself); a warp takes a pair and its lanes walk that pivot
        // row's entries together, so every lane does the same work
        const uint32_t nk_lane = lane < cnt ? s_cnt[buf][lane] : 0u;
        uint32_t incl = nk_lane;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= (uint32_t)d) incl += y;
        }
        const uint32_t npairs = __shfl_sync(0xffffffffu, incl, 31), excl = incl - nk_lane;
        for (uint32_t w0 = e0; w0 < e1; w0 += win) {
            const uint32_t w1 = min(w0 + win, e1), a = w0 & ~3u;
            if (w0 != e0) {
                stage(a, w1);
                cp_async_wait0();
                __syncthreads();
            }
            for (uint32_t q = warp; q < npairs; q += RB / 32) {
                const uint32_t k = __popc(__ballot_sync(0xffffffffu, incl <= q));  // chunk row of pair q
                const uint32_t w = s_list[k][q - __shfl_sync(0xffffffffu, excl, k)];
                const uint32_t lo = max(s_rp[buf][k], w0), hi = min(s_rp[buf][k + 1], w1);
                uint32_t *row = acc + (size_t)(w >> 16) * NS;
                const uint32_t m = w & 0xFFFFu;
                for (uint32_t e = lo + lane; e < hi; e += 32)
                    atomicAdd(&row[wcol[e - a]], fp_reduce32_2p(m * wval[e - a], fp));
            }
            if (w1 < e1) __syncthreads();  // every thread is done with the window
        }
    }
    __syncthreads();
    if (warp < nr && lane == 0 && (applied || fmas)) {
        atomicAdd(&J.work[0], applied);
        atomicAdd(&J.work[1], fmas);
    }
    for (uint32_t r = 0; r < nr; ++r) {
        uint32_t *out = J.dprime + (size_t)(i0 + r) * J.nb;
        for (uint32_t jj = threadIdx.x; jj < J.nb; jj += RB) out[jj] = fp_reduce32(acc[r * NS + J.nonpiv[jj]], fp);
    }
}

// ---- the same reduction with each row split over a thread-block cluster ------------------------
//
// When there are few non-pivot rows, one block per row leaves most SMs idle while each row sweeps
// its chunks one after another.  Here a row is spread over a cluster of CS blocks: block q owns the
// columns [q S, (q + 1) S) (S = ceil(N / CS)) in its shared memory, and split[k][q] gives the first
// entry of pivot row k at or right of q S (computed once per matrix).  Per chunk, the owners of the
// chunk's pivot columns publish their values into block 0's shared memory (distributed shared
// memory), one cluster barrier makes them visible, every block forms the same 32 multipliers and
// applies the part of each pivot row that falls in its own columns.  One cluster barrier per chunk.
constexpr int CS = 8;  // blocks per row

// split[k][q] = first entry of pivot row k with column >= q S, q = 0..CS (warp per pivot row)
__global__ void k_split(const RedJob *__restrict__ jobs, const uint32_t *__restrict__ bstart, int nj) {
    const int jb = job_of_block(bstart, nj);
    const RedJob &J = jobs[jb];
    const uint32_t k = (blockIdx.x - bstart[jb]) * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (k >= J.nA || lane > CS) return;
    const uint32_t S = (J.N + CS - 1) / CS, x = lane * S;
    uint32_t lo = J.row_ptr[k], hi = J.row_ptr[k + 1];
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (J.col[mid] < x) lo = mid + 1; else hi = mid;
    }
    J.split[(size_t)k * (CS + 1) + lane] = lo;
}

__device__ __forceinline__ uint32_t lower_bound_u32(const uint32_t *__restrict__ a, uint32_t lo, uint32_t hi,
                                                    uint32_t x) {
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int job_of(const uint32_t *__restrict__ bstart, int nj, uint32_t b) {
    int lo = 0, hi = nj - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (bstart[mid] <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <int MODE>
__global__ void __cluster_dims__(CS, 1, 1) __launch_bounds__(RT)
    k_reduce_cl(const RedJob *__restrict__ jobs, const uint32_t *__restrict__ bstart, int nj) {
    using Acc = typename AccOf<MODE>::type;
    constexpr bool SMALLP = MODE != M64;
    namespace cg = cooperative_groups;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint32_t Us[2][CW * CW];
    __shared__ uint32_t xs[2][CW];  // block 0's copy: the chunk's pivot-column values
    __shared__ uint32_t seg_q[CW], seg_m[CW], seg_pre[CW + 1];
    __shared__ uint32_t s_nseg;
    cg::cluster_group cl = cg::this_cluster();
    const uint32_t q = cl.block_rank();
    uint32_t *xs0 = cl.map_shared_rank(&xs[0][0], 0);
    const uint32_t rb = blockIdx.x / CS;  // the row's cluster
    const int jb = job_of(bstart, nj, rb);
    const RedJob &J = jobs[jb];
    const Fp fp = J.fp;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t i = rb - bstart[jb], row = J.nA + i;
    const uint32_t a0 = J.row_ptr[row], b0 = J.row_ptr[row + 1];
    const uint32_t base = a0 < b0 ? J.col[a0] : J.N, span = (J.N + CS - 1) / CS;
    const uint32_t lo = min(q * span, J.N), hi = min(lo + span, J.N), width = hi - lo;
    Acc *acc = reinterpret_cast<Acc *>(smem_raw);  // column c at acc[c - lo]
    for (uint32_t j = threadIdx.x; j < width; j += RT) acc[j] = 0;
    __syncthreads();
    {
        const uint32_t ea = lower_bound_u32(J.col, a0, b0, lo), eb = lower_bound_u32(J.col, ea, b0, hi);
        for (uint32_t e = ea + threadIdx.x; e < eb; e += RT) acc[J.col[e] - lo] = J.val[e];
    }
    // first chunk holding a pivot column >= base (the same in every block of the cluster)
    const uint32_t k0 = (lower_bound_u32(J.pcols, 0, J.nA, base) / CW) * CW;
    if (k0 < J.nA)
        for (uint32_t t = threadIdx.x; t < CW * CW; t += RT) Us[0][t] = J.U[(size_t)(k0 / CW) * CW * CW + t];
    unsigned long long applied = 0, fmas = 0;
    for (uint32_t kc = k0, buf = 0; kc < J.nA; kc += CW, buf ^= 1) {
        const uint32_t cnt = min((uint32_t)CW, J.nA - kc);
        __syncthreads();  // this block's updates of the previous chunk (and this chunk's U) are done
        if (warp == 0) {
            // publish the values this block owns (a column left of the row's leading column holds
            // zero: no pivot row with a nonzero multiplier reaches it); block 0 writes the zeros of
            // lanes past the chunk
            uint32_t v = 0;
            bool mine = q == 0;
            if ((uint32_t)lane < cnt) {
                const uint32_t c = J.pcols[kc + lane];
                mine = c >= lo && c < hi;
                if (mine) {
                    const Acc a = acc[c - lo];
                    v = MODE == A32 ? fp_reduce32((uint32_t)a, fp) : fp_reduce((unsigned long long)a, fp);
                }
            }
            if (mine) xs0[buf * CW + lane] = v;
        }
        cl.sync();  // every block's values of this chunk are in block 0
        if (warp == 0) {
            // the chunk's multipliers f = x U^{-1} (the same in every block), then this block's part
            // of each pivot row with f != 0 as a segment of its CSR range
            const uint32_t x = xs0[buf * CW + lane];
            const uint32_t *Wc = Us[buf];
            unsigned long long sacc = 0;
#pragma unroll
            for (int j = 0; j < CW; ++j) {
                const uint32_t vj = __shfl_sync(0xffffffffu, x, j);
                const uint32_t w = Wc[j * CW + lane];
                if (SMALLP) sacc += (unsigned long long)(vj * w);
                else sacc += fp_redc((uint64_t)vj * w, fp);
            }
            const uint32_t f = (uint32_t)lane < cnt ? fp_reduce(sacc, fp) : 0u;
            uint32_t ea = 0, len = 0;
            if (f) {
                const uint32_t *sp = J.split + (size_t)(kc + lane) * (CS + 1) + q;
                ea = sp[0];
                len = sp[1] - ea;
            }
            const unsigned segmask = __ballot_sync(0xffffffffu, len != 0u);
            uint32_t end = len;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, end, d);
                if (lane >= d) end += y;
            }
            if (len) {
                // segments in lane order; the prefix over all lanes counts only those with entries
                const uint32_t pos = __popc(segmask & ((1u << lane) - 1u));
                seg_q[pos] = ea;
                seg_m[pos] = SMALLP ? fp.p - f : fp_to_mont(fp.p - f, fp);
                seg_pre[pos + 1] = end;
            }
            const uint32_t total = __shfl_sync(0xffffffffu, end, 31);
            const unsigned fmask = __ballot_sync(0xffffffffu, f != 0u);
            if (lane == 0) {
                seg_pre[0] = 0;
                s_nseg = __popc(segmask);
                if (q == 0) applied += __popc(fmask);  // pivot rows used: counted once per row
                fmas += total;                          // multiply-adds: each block its own part
            }
        } else {
            const uint32_t kn = kc + CW;
            if (kn < J.nA)
                for (uint32_t t = threadIdx.x - 32u; t < CW * CW; t += RT - 32u)
                    Us[buf ^ 1][t] = J.U[(size_t)(kn / CW) * CW * CW + t];
        }
        __syncthreads();
        // apply this block's segments: entries flattened and split evenly over the warps
        const uint32_t nseg = s_nseg, total = seg_pre[nseg];
        const uint32_t per = (total + RT - 1) / RT * 32;
        const uint32_t w0 = min(warp * per, total), w1 = min(w0 + per, total);
        uint32_t sg = 0, send = 0, soff = 0, smul = 0;
        if (w0 + lane < w1) {
            uint32_t a = 0, b = nseg - 1;
            while (a < b) {
                const uint32_t mid = (a + b + 1) >> 1;
                if (seg_pre[mid] <= w0 + lane) a = mid; else b = mid - 1;
            }
            sg = a;
            send = seg_pre[sg + 1];
            soff = seg_q[sg] - seg_pre[sg];
            smul = seg_m[sg];
        }
        for (uint32_t x0 = w0; x0 < w1; x0 += 4 * 32) {
            uint32_t cc[4], vv[4], mm[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t x = x0 + 32u * u + lane;
                cc[u] = 0xFFFFFFFFu;
                vv[u] = mm[u] = 0u;
                if (x < w1) {
                    while (x >= send) {
                        ++sg;
                        send = seg_pre[sg + 1];
                        soff = seg_q[sg] - seg_pre[sg];
                        smul = seg_m[sg];
                    }
                    cc[u] = J.col[soff + x];
                    vv[u] = J.val[soff + x];
                    mm[u] = smul;
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (cc[u] == 0xFFFFFFFFu) continue;
                Acc *dst = acc + (cc[u] - lo);
                if (MODE == A32)
                    atomicAdd(reinterpret_cast<uint32_t *>(dst), fp_reduce32(mm[u] * vv[u], fp));
                else if (MODE == A64)
                    atomicAdd(reinterpret_cast<unsigned long long *>(dst), (unsigned long long)(mm[u] * vv[u]));
                else
                    atomicAdd(reinterpret_cast<unsigned long long *>(dst),
                              (unsigned long long)fp_redc((uint64_t)mm[u] * vv[u], fp));
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && (applied || fmas)) {
        atomicAdd(&J.work[0], applied);
        atomicAdd(&J.work[1], fmas);
    }
    // this block's columns of D' (zero left of the row's leading column)
    uint32_t *out = J.dprime + (size_t)i * J.nb;
    const uint32_t jlo = lower_bound_u32(J.nonpiv, 0, J.nb, lo);
    const uint32_t jhi = lower_bound_u32(J.nonpiv, jlo, J.nb, hi);
    for (uint32_t jj = jlo + threadIdx.x; jj < jhi; jj += RT) {
        const uint32_t c = J.nonpiv[jj];
        if (c < base) {
            out[jj] = 0u;
        } else {
            const Acc a = acc[c - lo];
            out[jj] = MODE == A32 ? fp_reduce32((uint32_t)a, fp) : fp_reduce((unsigned long long)a, fp);
        }
    }
    cl.sync();  // block 0's shared memory stays valid until every block has read its last chunk
}

// ---- RREF(D'): right-looking Gauss-Jordan by panels of KP rows --------------------------------
//
// M starts as a copy of D'.  Each round picks up to KP non-zero rows that are not pivots yet,
// brings them to reduced echelon form among themselves in one block (pivots at their leading
// columns), then eliminates the new pivot columns from every other row of M in parallel, which
// also keeps the earlier pivot rows reduced.  A pivot row's leading column never moves: it is zero
// left of its pivot, and later pivot rows are zero at it.  When no non-zero non-pivot row is left,
// the pivot rows sorted by pivot column are RREF(D'), which is unique.  The panel solves of
// different jobs run side by side, one block each.
constexpr uint32_t KP = 16;
constexpr uint32_t NOLEAD = 0xFFFFFFFFu;

struct RrefJob {
    uint32_t *M;      // nC x nb working matrix
    uint32_t *lead;   // nC: first non-zero column, NOLEAD for a zero row
    uint32_t *pcol;   // nC: pivot column of a pivot row, NOLEAD otherwise
    uint32_t *order;  // pivot rows in discovery order
    uint32_t *state;  // [0] pivots so far, [1] panel rows, [2] new pivots, [3] rows left
    uint32_t *panel;  // KP panel row ids, then KP new pivot row ids, then KP new pivot columns
    uint32_t *out, *opiv;
    uint32_t nC, nb, rank;
    Fp fp;
    uint64_t ldm;         // row pitch of M (nb rounded up to 4: rows start on 16-byte boundaries)
    uint32_t tc;          // 1: the trailing update of this job runs on the tensor cores (k_mm)
    uint16_t *fa, *fb;    // tc: digit planes of the multipliers (nC x KP) and of the pivot rows (nb x KP)
    uint64_t fkp;         // tc: their row pitch (KP rounded up to 64)
};

__device__ __forceinline__ uint32_t block_min(uint32_t v, uint32_t *red) {
    for (int d = 16; d; d >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, d));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    v = threadIdx.x < blockDim.x / 32 ? red[threadIdx.x] : NOLEAD;
    if (threadIdx.x < 32)
        for (int d = 16; d; d >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, d));
    if (threadIdx.x == 0) red[0] = v;
    __syncthreads();
    return red[0];
}

// leading columns of every row (block per row)
__global__ void k_leads(const RrefJob *__restrict__ jobs, const uint32_t *__restrict__ bstart, int nj) {
    __shared__ uint32_t red[32];
    const int jb = job_of_block(bstart, nj);
    const RrefJob &X = jobs[jb];
    const uint32_t r = blockIdx.x - bstart[jb];
    const uint32_t *row = X.M + (size_t)r * X.ldm;
    uint32_t c = NOLEAD;
    for (uint32_t j = threadIdx.x; j < X.nb; j += blockDim.x)
        if (row[j]) { c = j; break; }
    c = block_min(c, red);
    if (threadIdx.x == 0) {
        X.lead[r] = c;
        X.pcol[r] = NOLEAD;
    }
}

// the next panel of each job: its first KP non-zero rows that are not pivots (block per job)
__global__ void k_pick_panel(const RrefJob *__restrict__ jobs) {
    __shared__ uint32_t wcnt[32];
    __shared__ uint32_t s_taken;
    const RrefJob &X = jobs[blockIdx.x];
    if (!X.state) return;  // a job without a D' block
    if (threadIdx.x == 0) s_taken = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x / 32;
    uint32_t left = 0;
    for (uint32_t r0 = 0; r0 < X.nC; r0 += blockDim.x) {
        const uint32_t r = r0 + threadIdx.x;
        const bool want = r < X.nC && X.lead[r] != NOLEAD && X.pcol[r] == NOLEAD;
        left += want;
        const unsigned mask = __ballot_sync(0xffffffffu, want);
        if (lane == 0) wcnt[warp] = __popc(mask);
        __syncthreads();
        uint32_t before = s_taken;
        for (int w = 0; w < warp; ++w) before += wcnt[w];
        before += __popc(mask & ((1u << lane) - 1u));
        if (want && before < KP) X.panel[before] = r;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t t = s_taken;
            for (int w = 0; w < nw; ++w) t += wcnt[w];
            s_taken = t;
        }
        __syncthreads();
    }
    for (int d = 16; d; d >>= 1) left += __shfl_xor_sync(0xffffffffu, left, d);
    if (lane == 0) wcnt[warp] = left;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < nw; ++w) t += wcnt[w];
        X.state[3] = t;
        X.state[1] = min(s_taken, KP);
        X.state[2] = 0;
    }
}

// reduced echelon form of each job's panel rows among themselves (block per job of `list`).
// With SMEM the panel is copied to shared memory, reduced there and written back.
constexpr int PT = 1024;
constexpr uint32_t GJB = 4;  // columns of a thread handled together in the global-memory panel's sweeps
template <bool SMEM>
__global__ void __launch_bounds__(PT) k_panel_rref(const RrefJob *__restrict__ jobs, const int *__restrict__ list) {
    extern __shared__ __align__(16) uint32_t pan[];
    __shared__ uint32_t mult[KP], prow[KP], pslot[KP], pc[KP], red[32], s_row[KP];
    __shared__ uint32_t s_inv;
    // the global-memory panel batches JB columns per thread; the shared-memory one, whose rows are
    // short, one
    constexpr uint32_t JB = SMEM ? 1u : GJB;
    const RrefJob &X = jobs[list[blockIdx.x]];
    const Fp fp = X.fp;
    const uint32_t P = X.state[1], nb = X.nb;
    if (threadIdx.x < KP) s_row[threadIdx.x] = threadIdx.x < P ? X.panel[threadIdx.x] : 0u;
    __syncthreads();
    auto rowp = [&](uint32_t t) -> uint32_t * {
        return SMEM ? pan + (size_t)t * nb : X.M + (size_t)s_row[t] * X.ldm;
    };
    if (SMEM) {  // all of a thread's loads in flight before its stores
        for (uint32_t j = threadIdx.x; j < nb; j += PT) {
            uint32_t v[KP];
#pragma unroll
            for (uint32_t t = 0; t < KP; ++t)
                if (t < P) v[t] = X.M[(size_t)s_row[t] * X.ldm + j];
#pragma unroll
            for (uint32_t t = 0; t < KP; ++t)
                if (t < P) pan[(size_t)t * nb + j] = v[t];
        }
        __syncthreads();
    }
    uint32_t nnew = 0;
    for (uint32_t t = 0; t < P; ++t) {
        const uint32_t r = s_row[t];
        uint32_t *row = rowp(t);
        // multipliers: entries at the panel's earlier pivots, negated (those pivot rows are RREF
        // among themselves, so each multiplier is read from the unreduced row)
        if (threadIdx.x < nnew) {
            const uint32_t v = row[pc[threadIdx.x]];
            mult[threadIdx.x] = v ? fp.p - v : 0u;
        }
        __syncthreads();
        // a thread's columns JB at a time (j, j + PT, ...), and four earlier pivot rows per step:
        // up to 4 JB independent loads in flight (the global-memory panel waits on L2 for each)
        uint32_t c = NOLEAD;
        for (uint32_t j0 = threadIdx.x; j0 < nb; j0 += PT * JB) {
            uint64_t acc[JB];
#pragma unroll
            for (uint32_t u = 0; u < JB; ++u) acc[u] = j0 + u * PT < nb ? row[j0 + u * PT] : 0u;
            for (uint32_t k0 = 0; k0 < nnew; k0 += 4) {
#pragma unroll
                for (uint32_t v = 0; v < 4; ++v) {
                    const uint32_t k = k0 + v;
                    if (k >= nnew || !mult[k]) continue;
                    const uint32_t mk = mult[k], *pk = rowp(pslot[k]);
#pragma unroll
                    for (uint32_t u = 0; u < JB; ++u) {
                        const uint32_t j = j0 + u * PT;
                        if (j >= nb) break;
                        // raw products < 2^32 for p < 2^16 (at most KP of them), else reduced
                        acc[u] += fp.small ? (uint64_t)(mk * pk[j]) : (uint64_t)fp_mul(mk, pk[j], fp);
                    }
                }
            }
#pragma unroll
            for (uint32_t u = 0; u < JB; ++u) {
                const uint32_t j = j0 + u * PT;
                if (j >= nb) break;
                const uint32_t x = nnew ? fp_reduce(acc[u], fp) : (uint32_t)acc[u];
                if (nnew) row[j] = x;
                if (x && c == NOLEAD) c = j;
            }
        }
        c = block_min(c, red);
        if (c == NOLEAD) {
            if (threadIdx.x == 0) X.lead[r] = NOLEAD;
            continue;
        }
        if (threadIdx.x == 0) s_inv = fp.small ? fp_inv_small(row[c], fp) : fp_inv(row[c], fp);
        __syncthreads();
        const uint32_t inv = s_inv;
        for (uint32_t j0 = c + threadIdx.x; j0 < nb; j0 += PT * JB) {
            uint32_t y[JB];
#pragma unroll
            for (uint32_t u = 0; u < JB; ++u) y[u] = j0 + u * PT < nb ? row[j0 + u * PT] : 0u;
#pragma unroll
            for (uint32_t u = 0; u < JB; ++u)
                if (j0 + u * PT < nb) row[j0 + u * PT] = fp_mul(y[u], inv, fp);
        }
        if (threadIdx.x < nnew) {
            const uint32_t v = rowp(pslot[threadIdx.x])[c];
            mult[threadIdx.x] = v ? fp.p - v : 0u;
        }
        __syncthreads();
        // clear column c from the earlier new rows: a thread's columns JB at a time, every earlier
        // row at once
        for (uint32_t j0 = c + threadIdx.x; j0 < nb; j0 += PT * JB) {
            uint32_t y[JB];
#pragma unroll
            for (uint32_t u = 0; u < JB; ++u) y[u] = j0 + u * PT < nb ? row[j0 + u * PT] : 0u;
            for (uint32_t k = 0; k < nnew; ++k) {
                const uint32_t mk = mult[k];
                if (!mk) continue;
                uint32_t *dk = rowp(pslot[k]);
                uint32_t d[JB];
#pragma unroll
                for (uint32_t u = 0; u < JB; ++u) d[u] = y[u] ? dk[j0 + u * PT] : 0u;
#pragma unroll
                for (uint32_t u = 0; u < JB; ++u)
                    if (y[u]) dk[j0 + u * PT] = fp.small ? fp_add(d[u], fp_reduce32(mk * y[u], fp), fp)
                                                         : fp_reduce((uint64_t)d[u] + (uint64_t)mk * y[u], fp);
            }
        }
        if (threadIdx.x == 0) {
            prow[nnew] = r;
            pslot[nnew] = t;
            pc[nnew] = c;
            X.lead[r] = c;
            X.pcol[r] = c;
        }
        __syncthreads();
        ++nnew;
    }
    if (SMEM) {  // write the panel back (pivot rows reduced, the others now zero)
        for (uint32_t j = threadIdx.x; j < nb; j += PT) {
            uint32_t v[KP];
#pragma unroll
            for (uint32_t t = 0; t < KP; ++t)
                if (t < P) v[t] = pan[(size_t)t * nb + j];
#pragma unroll
            for (uint32_t t = 0; t < KP; ++t)
                if (t < P) X.M[(size_t)s_row[t] * X.ldm + j] = v[t];
        }
    }
    if (threadIdx.x < nnew) {
        X.panel[KP + threadIdx.x] = prow[threadIdx.x];
        X.panel[2 * KP + threadIdx.x] = pc[threadIdx.x];
        X.order[X.state[0] + threadIdx.x] = prow[threadIdx.x];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        X.state[2] = nnew;
        X.state[0] += nnew;
    }
}

// The same panel solve with the panel's columns spread over a cluster of PCS blocks: block q holds
// the columns [q S, (q + 1) S) of all panel rows in its shared memory (S = ceil(nb / PCS)).  The
// rows are taken in order (Gauss-Jordan).  Per row, every block finds its first non-zero column
// c_q and publishes, in its own shared memory, c_q, column c_q of every panel row and the inverse
// of the row's entry there; one cluster barrier; every block takes the least c_q (the row is zero
// when there is none) and reads that block's column and inverse through distributed shared
// memory; then every block scales the pivot row and subtracts its multiples from the other panel
// rows on its own columns.  The published values are double-buffered by the row's parity: a block
// overwrites them two rows later, after a barrier every block passes only once it has read them.
// So a pivot costs one cluster barrier and one sweep of a block's share of the panel, against one
// block's sweeps of whole rows in k_panel_rref.  Eliminating each pivot column from all other
// panel rows at once (instead of reducing a row by the earlier pivots when its turn comes) gives
// the same pivots and the same reduced rows: a row's reduction modulo the span of the earlier pivot
// rows, with zeros at their pivot columns, is unique, and so is the reduced echelon form of the
// panel's pivot rows.
constexpr int PCS = 8;      // blocks per cluster
constexpr int PCT = 1024;   // threads per block
constexpr uint32_t PANEL_CLUSTER_MAX_NB = PCS * 3200;  // 4 KP S bytes of shared memory per block
constexpr uint32_t PANEL_CLUSTER_MIN_NB = 1024;         // narrower panels: one block (k_panel_rref)
__global__ void __cluster_dims__(PCS, 1, 1) __launch_bounds__(PCT)
    k_panel_rref_cl(const RrefJob *__restrict__ jobs, const int *__restrict__ list) {
    namespace cg = cooperative_groups;
    extern __shared__ __align__(16) uint32_t slab[];  // KP rows of S columns
    __shared__ uint32_t s_min[2];           // this block's first non-zero column of the row, by parity
    __shared__ uint32_t s_pub[2][KP + 1];   // that column of every panel row, then the inverse, by parity
    __shared__ uint32_t s_col[KP + 1];      // the pivot block's published values, read for the update
    __shared__ uint32_t red[32], s_row[KP], s_c, s_owner;
    cg::cluster_group cl = cg::this_cluster();
    const uint32_t q = cl.block_rank();
    const RrefJob &X = jobs[list[blockIdx.x / PCS]];
    const Fp fp = X.fp;
    const uint32_t P = X.state[1], nb = X.nb, S = (nb + PCS - 1) / PCS;
    const uint32_t c0 = min(nb, q * S), w = min(nb, c0 + S) - c0;
    if (threadIdx.x < KP) s_row[threadIdx.x] = threadIdx.x < P ? X.panel[threadIdx.x] : 0u;
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < w; j += PCT)  // eight rows' loads in flight before their stores
        for (uint32_t t0 = 0; t0 < P; t0 += 8) {
            uint32_t v[8];
#pragma unroll
            for (uint32_t t = 0; t < 8; ++t)
                if (t0 + t < P) v[t] = X.M[(size_t)s_row[t0 + t] * X.ldm + c0 + j];
#pragma unroll
            for (uint32_t t = 0; t < 8; ++t)
                if (t0 + t < P) slab[(size_t)(t0 + t) * S + j] = v[t];
        }
    __syncthreads();
    uint32_t nnew = 0;
    for (uint32_t t = 0; t < P; ++t) {
        const uint32_t par = t & 1u;
        uint32_t *row = slab + (size_t)t * S;
        uint32_t c = NOLEAD;
        for (uint32_t j = threadIdx.x; j < w; j += PCT)
            if (row[j]) { c = c0 + j; break; }
        c = block_min(c, red);
        if (threadIdx.x == 0) s_min[par] = c;
        if (c != NOLEAD && threadIdx.x <= KP) {  // this block's candidate pivot column and inverse
            // (in Montgomery form for p >= 2^16: the update's products are then one redc each)
            const uint32_t u = threadIdx.x, jc = c - c0;
            uint32_t v;
            if (u < KP) v = u < P && u != t ? slab[(size_t)u * S + jc] : 0u;
            else v = fp.small ? fp_inv_small(row[jc], fp) : fp_inv(row[jc], fp);
            s_pub[par][u] = fp.small ? v : fp_to_mont(v, fp);
        }
        cl.sync();
        if (threadIdx.x < 32) {
            const uint32_t m = threadIdx.x < PCS ? *cl.map_shared_rank(&s_min[par], threadIdx.x) : NOLEAD;
            uint32_t best = m, who = threadIdx.x;
            for (int d = 16; d; d >>= 1) {  // the least column (block column ranges are disjoint)
                const uint32_t bo = __shfl_xor_sync(0xffffffffu, best, d), wo = __shfl_xor_sync(0xffffffffu, who, d);
                if (bo < best) { best = bo; who = wo; }
            }
            if (threadIdx.x == 0) {
                s_c = best;
                s_owner = who;
            }
        }
        __syncthreads();
        c = s_c;
        if (c == NOLEAD) {  // the row reduced to zero
            if (q == 0 && threadIdx.x == 0) X.lead[s_row[t]] = NOLEAD;
            continue;
        }
        if (threadIdx.x <= KP) s_col[threadIdx.x] = *cl.map_shared_rank(&s_pub[par][threadIdx.x], s_owner);
        __syncthreads();
        const uint32_t inv = s_col[KP];
        auto mulp = [&](uint32_t a, uint32_t b) -> uint32_t {  // a b mod p, b in the published form
            if (fp.small) return fp_reduce32(a * b, fp);
            const uint32_t r = fp_redc((uint64_t)a * b, fp);  // in [0, 2p)
            return r >= fp.p ? r - fp.p : r;
        };
        for (uint32_t j = (c > c0 ? c - c0 : 0) + threadIdx.x; j < w; j += PCT) {
            const uint32_t y = mulp(row[j], inv);
            row[j] = y;
            if (!y) continue;
            for (uint32_t u = 0; u < P; ++u) {
                const uint32_t m = s_col[u];
                if (!m) continue;
                uint32_t *x = slab + (size_t)u * S + j;
                *x = fp_sub(*x, mulp(y, m), fp);
            }
        }
        if (q == 0 && threadIdx.x == 0) {
            X.panel[KP + nnew] = s_row[t];
            X.panel[2 * KP + nnew] = c;
            X.order[X.state[0] + nnew] = s_row[t];
            X.lead[s_row[t]] = c;
            X.pcol[s_row[t]] = c;
        }
        ++nnew;
        __syncthreads();
    }
    for (uint32_t j = threadIdx.x; j < w; j += PCT)  // the panel back (pivot rows reduced, the rest zero)
        for (uint32_t t = 0; t < P; ++t) X.M[(size_t)s_row[t] * X.ldm + c0 + j] = slab[(size_t)t * S + j];
    if (q == 0 && threadIdx.x == 0) {
        X.state[2] = nnew;
        X.state[0] += nnew;
    }
    cl.sync();  // no block leaves while another may still reach into its shared memory
}

// every other row: r <- r - sum_k r[pc_k] * Q_k over the panel's new pivot rows Q_k; one block per
// row, so a row's multipliers are read before any thread writes the row
__global__ void k_eliminate(const RrefJob *__restrict__ jobs, const uint32_t *__restrict__ bstart, int nj) {
    __shared__ uint32_t m[KP], q[KP], red[32];
    __shared__ int s_any;
    const int jb = job_of_block(bstart, nj);
    const RrefJob &X = jobs[jb];
    const Fp fp = X.fp;
    const uint32_t r = blockIdx.x - bstart[jb], nb = X.nb, nnew = X.state[2];
    if (X.tc || nnew == 0 || X.lead[r] == NOLEAD) return;
    const uint32_t pr = X.pcol[r];
    uint32_t *row = X.M + (size_t)r * X.ldm;
    if (threadIdx.x == 0) s_any = 0;
    __syncthreads();
    if (threadIdx.x < nnew) {
        q[threadIdx.x] = X.panel[KP + threadIdx.x];
        const uint32_t v = q[threadIdx.x] == r ? 0u : row[X.panel[2 * KP + threadIdx.x]];
        m[threadIdx.x] = v;
        if (v) s_any = 1;
    }
    __syncthreads();
    if (!s_any) return;
    uint32_t c = NOLEAD;
    for (uint32_t j = threadIdx.x; j < nb; j += blockDim.x) {
        uint64_t acc = row[j];
        if (fp.small) {  // at most KP raw products below 2^32 each
            for (uint32_t k = 0; k < nnew; ++k)
                if (m[k]) acc += (uint64_t)((fp.p - m[k]) * X.M[(size_t)q[k] * X.ldm + j]);
        } else {
            for (uint32_t k = 0; k < nnew; ++k)
                if (m[k]) acc += fp_mul(fp.p - m[k], X.M[(size_t)q[k] * X.ldm + j], fp);
        }
        const uint32_t x = fp_reduce(acc, fp);
        row[j] = x;
        if (x && c == NOLEAD) c = j;
    }
    if (pr == NOLEAD) {  // a pivot row keeps its leading column; other rows may move or vanish
        c = block_min(c, red);
        if (threadIdx.x == 0) X.lead[r] = c;
    }
}

// The same trailing update on the tensor cores for large D': M <- M - F Q with F[r][k] = M[r][pc_k]
// (zero on the panel's own pivot rows and for k past the new pivots) and Q the new pivot rows.
// Digit planes of F (row r, K index k) and of Q^T (row j, K index k); KP K values, zero past nnew.
template <int L>
__global__ void k_elim_digits(const RrefJob *__restrict__ jobs, int jb) {
    const RrefJob &X = jobs[jb];
    const uint32_t nnew = X.state[2];
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t T = L == 2 ? 32639u : 2139062143u;  // 127 (1 + 256 + ... + 256^{L-1})
    auto put = [&](uint32_t x, uint16_t *dst, uint64_t plane) {
        int v = x <= T ? (int)x : (int)(x - X.fp.p);
#pragma unroll
        for (int l = 0; l < L; ++l) {
            const int a = l + 1 < L ? (int)(((uint32_t)v & 0xFFu) ^ 0x80u) - 0x80 : v;
            if (l + 1 < L) v = (v - a) >> 8;
            dst[(size_t)l * plane] = (uint16_t)(__float_as_uint((float)a) >> 16);
        }
    };
    if (t < X.nC * KP) {  // F: row r, column k
        const uint32_t r = t / KP, k = t % KP;
        uint32_t x = 0;
        if (k < nnew && X.panel[KP + k] != r) x = X.M[(size_t)r * X.ldm + X.panel[2 * KP + k]];
        put(x, X.fa + (size_t)r * X.fkp + k, (uint64_t)X.nC * X.fkp);
    } else if (t < X.nC * KP + X.nb * KP) {  // Q^T: row j, column k
        const uint32_t u = t - X.nC * KP, j = u / KP, k = u % KP;
        const uint32_t x = k < nnew ? X.M[(size_t)X.panel[KP + k] * X.ldm + j] : 0u;
        put(x, X.fb + (size_t)j * X.fkp + k, (uint64_t)X.nb * X.fkp);
    }
}

// leading columns of the rows that are not pivots, after a tensor-core update (block per row)
__global__ void k_leads_np(const RrefJob *__restrict__ jobs, int jb) {
    __shared__ uint32_t red[32];
    const RrefJob &X = jobs[jb];
    const uint32_t r = blockIdx.x;
    if (X.state[2] == 0 || X.lead[r] == NOLEAD || X.pcol[r] != NOLEAD) return;  // uniform per block
    const uint32_t *row = X.M + (size_t)r * X.ldm;
    uint32_t c = NOLEAD;
    for (uint32_t j = threadIdx.x; j < X.nb; j += blockDim.x)
        if (row[j]) { c = j; break; }
    c = block_min(c, red);
    if (threadIdx.x == 0) X.lead[r] = c;
}

// The condition of the round loop, evaluated on the device after each round (one warp): another
// round is needed while some job's last pick left more non-pivot rows than its panel took, and
// fewer than maxrounds rounds have run (every round settles at least one panel of KP rows).
__global__ void k_rref_more(const RrefJob *__restrict__ jobs, int nj, uint32_t *rounds, uint32_t maxrounds,
                            cudaGraphConditionalHandle more_h) {
    bool more = false;
    for (int j = threadIdx.x; j < nj; j += 32) {
        const uint32_t *st = jobs[j].state;
        if (st && st[1] != 0 && st[3] > st[1]) more = true;
    }
    more = __any_sync(0xffffffffu, more);
    if (threadIdx.x == 0) {
        const uint32_t r = *rounds + 1;
        *rounds = r;
        cudaGraphSetConditional(more_h, more && r < maxrounds ? 1u : 0u);
    }
}

// An executable graph and its template; the executable may be destroyed while it is still in
// flight (CUDA then frees it when the launch completes).
struct RoundGraph {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
    RoundGraph() = default;
    RoundGraph(const RoundGraph &) = delete;
    RoundGraph(RoundGraph &&o) noexcept {
        std::swap(g, o.g);
        std::swap(exec, o.exec);
    }
    RoundGraph &operator=(const RoundGraph &) = delete;
    RoundGraph &operator=(RoundGraph &&o) noexcept {
        reset();
        std::swap(g, o.g);
        std::swap(exec, o.exec);
        return *this;
    }
    ~RoundGraph() { reset(); }
    void reset() {
        if (exec) cudaGraphExecDestroy(exec);
        if (g) cudaGraphDestroy(g);
        exec = nullptr;
        g = nullptr;
    }
};

// Loops below this many rounds stay on host launches: recording and instantiating the graph
// costs about as much as launching a few rounds directly.
constexpr uint32_t GRAPH_MIN_ROUNDS = 3;

// Records `body` (which launches one round on the stream it is given and then sets the loop
// condition from the device) as the body of a while-node and instantiates the graph.  The node's
// condition starts at 1 on every launch, so the body runs at least once.  `nodes` receives the
// number of kernels in one round.
template <class F>
RoundGraph record_round_loop(gb_ctx *ctx, F &&body, unsigned &nodes) {
    if (!ctx->capture) GB_CUDA(cudaStreamCreateWithFlags(&ctx->capture, cudaStreamNonBlocking));
    RoundGraph R;
    GB_CUDA(cudaGraphCreate(&R.g, 0));
    cudaGraphConditionalHandle h{};
    GB_CUDA(cudaGraphConditionalHandleCreate(&h, R.g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node{};
    GB_CUDA(cudaGraphAddNode(&node, R.g, nullptr, nullptr, 0, &np));
    GB_CUDA(cudaStreamBeginCaptureToGraph(ctx->capture, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal));
    t_capturing = true;
    t_captured = 0;
    try {
        body(ctx->capture, h);
    } catch (...) {
        t_capturing = false;
        cudaGraph_t x = nullptr;
        cudaStreamEndCapture(ctx->capture, &x);
        throw;
    }
    t_capturing = false;
    nodes = t_captured;
    cudaGraph_t x = nullptr;
    GB_CUDA(cudaStreamEndCapture(ctx->capture, &x));
    GB_CUDA(cudaGraphInstantiate(&R.exec, R.g, 0));
    return R;
}

// the pivot rows in pivot-column order (block per pivot row)
__global__ void k_gather_rref(const RrefJob *__restrict__ jobs, const uint32_t *__restrict__ bstart, int nj) {
    __shared__ uint32_t pos;
    const int jb = job_of_block(bstart, nj);
    const RrefJob &X = jobs[jb];
    const uint32_t e = blockIdx.x - bstart[jb], nb = X.nb;
    const uint32_t r = X.order[e], c = X.pcol[r];
    if (threadIdx.x == 0) {
        uint32_t n = 0;
        for (uint32_t f = 0; f < X.rank; ++f) n += X.pcol[X.order[f]] < c;
        pos = n;
        X.opiv[n] = c;
    }
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < nb; j += blockDim.x) X.out[(size_t)pos * nb + j] = X.M[(size_t)r * X.ldm + j];
}

// ---- reconstruction and the final tails ------------------------------------------------------

struct RowsJob {
    const uint32_t *M;      // rows x nb (rows >= mrows are empty)
    const uint32_t *rpiv;   // echelon pivots (append) or null
    const uint32_t *nonpiv;
    const uint4 *dict;
    const uint4 *lead;      // leading monomial written first (tails) or null
    uint32_t rows, mrows, nb, n, plus;
    uint32_t *cnt;          // this job's range of the concatenated counts
    const uint32_t *oscan;  // range of their exclusive scan (subtract oscan[0])
    uint4 *lm;              // leading monomials of the rows (append)
    const uint32_t *dst_off;  // absolute output offsets (append: the new elements' boff)
    uint4 *omon;            // append: basis monomials
    unsigned long long *okey;  // append: their mono_key
    uint32_t *ocf;
    uint8_t *oexp;          // tails: n-byte exponent vectors
};

// nonzeros of each row (+ plus for the leading term) (block per row)
__global__ void k_count_rows(const RowsJob *__restrict__ jobs, const uint32_t *__restrict__ bstart, int nj) {
    const int jb = job_of_block(bstart, nj);
    const RowsJob &J = jobs[jb];
    const uint32_t r = blockIdx.x - bstart[jb];
    uint32_t c = 0;
    if (r < J.mrows)
        for (uint32_t j = threadIdx.x; j < J.nb; j += blockDim.x) c += J.M[(size_t)r * J.nb + j] != 0;
    for (int d = 16; d; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
    __shared__ uint32_t s[32];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = J.plus;
        for (uint32_t w = 0; w < blockDim.x / 32; ++w) t += s[w];
        J.cnt[r] = t;
        if (J.rpiv) J.lm[r] = J.dict[J.nonpiv[J.rpiv[r]]];
    }
}

// write each row's terms in column order (descending monomials) at its offset (block per row)
__global__ void k_write_rows(const RowsJob *__restrict__ jobs, const uint32_t *__restrict__ bstart, int nj) {
    const int jb = job_of_block(bstart, nj);
    const RowsJob &J = jobs[jb];
    const uint32_t r = blockIdx.x - bstart[jb];
    __shared__ uint32_t base;
    __shared__ uint32_t wsum[32];
    auto put = [&](uint32_t pos, uint4 m, uint32_t c) {
        if (J.omon) {
            J.omon[pos] = m;
            J.okey[pos] = mono_key(m);
        } else {
            const uint32_t w[4] = {m.x, m.y, m.z, m.w};
            for (uint32_t i = 0; i < J.n; ++i) J.oexp[(size_t)pos * J.n + i] = (uint8_t)(w[i >> 2] >> (8 * (i & 3)));
        }
        J.ocf[pos] = c;
    };
    if (threadIdx.x == 0) {
        base = J.dst_off ? J.dst_off[r] : J.oscan[r] - J.oscan[0];
        if (J.lead) {
            put(base, J.lead[r], 1u);
            base += 1;
        }
    }
    __syncthreads();
    if (r >= J.mrows) return;
    const uint32_t *src = J.M + (size_t)r * J.nb;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x / 32;
    for (uint32_t j0 = 0; j0 < J.nb; j0 += blockDim.x) {
        const uint32_t j = j0 + threadIdx.x;
        const uint32_t v = j < J.nb ? src[j] : 0u;
        const unsigned mask = __ballot_sync(0xffffffffu, v != 0);
        if (lane == 0) wsum[warp] = __popc(mask);
        __syncthreads();
        uint32_t before = 0, total = 0;
        for (int w = 0; w < nw; ++w) {
            if (w < warp) before += wsum[w];
            total += wsum[w];
        }
        if (v) put(base + before + __popc(mask & ((1u << lane) - 1u)), J.dict[J.nonpiv[j]], v);
        __syncthreads();
        if (threadIdx.x == 0) base += total;
        __syncthreads();
    }
}

// launch a grouped row kernel: `per_job` blocks per job, plan staged and uploaded with the jobs
template <class JobT>
struct Grouped {
    DBuf<char> d;
    const JobT *jobs = nullptr;
    std::vector<const uint32_t *> plans;
    std::vector<uint32_t> totals;
    void build(gb_ctx *ctx, const std::vector<JobT> &J, const std::vector<std::vector<uint32_t>> &per_job) {
        Stage sg;
        std::vector<size_t> at(per_job.size());
        totals.resize(per_job.size());
        for (size_t k = 0; k < per_job.size(); ++k) totals[k] = plan(sg, per_job[k], at[k]);
        const size_t oj = sg.put(J.data(), sizeof(JobT) * J.size());
        sg.upload(ctx, d);
        jobs = reinterpret_cast<const JobT *>(d.p + oj);
        plans.resize(per_job.size());
        for (size_t k = 0; k < per_job.size(); ++k) plans[k] = reinterpret_cast<const uint32_t *>(d.p + at[k]);
    }
};

// Rows split over clusters when the per-row sweep, not the GPU's width, bounds the time: measured
// on B300 (n=10 workload), 1.8x faster at 9 rows and 1.5x at 81, slower from about 300 rows (a
// cluster barrier per chunk and the multipliers formed in every block), and slower on short sweeps
// (fewer than 2048 pivots).  `rows` counts the non-pivot rows of all sparse matrices of the launch.
bool use_cluster(const RedJob &J, size_t accb, uint64_t rows) {
    const size_t per_block = (size_t)((J.N + CS - 1) / CS) * accb;
    return per_block <= 48 * 1024 && rows <= 160 && J.nA >= 2048;
}

// dynamic shared memory of k_reduce_rows: the device's opt-in limit less the kernel's static part
size_t rows_dyn_smem() {
    int dev = 0, optin = 0;
    GB_CUDA(cudaGetDevice(&dev));
    GB_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa{};
    GB_CUDA(cudaFuncGetAttributes(&fa, reinterpret_cast<const void *>(k_reduce_rows)));
    return (size_t)optin - fa.sharedSizeBytes;
}

// Rows per block of k_reduce_rows for an A32 matrix, or 0 when one row per block is the better
// schedule: with no more rows than SMs one row per block already fills the GPU.  Otherwise enough
// rows per block for about one block per SM, at most RMAX and at most what shared memory holds
// next to a window of WMIN entries.  `rows` counts the non-pivot rows of the launch.
uint32_t rows_per_block(const RedJob &J, uint64_t rows, size_t dyn) {
    const uint64_t nsm = (uint64_t)sm_count(), NS = (J.N + 3u) & ~3u;
    if (rows <= nsm || dyn < 8ull * (WMIN + 8) || J.nA >= ROWS_MAX_PIVOTS) return 0;
    const uint64_t fit = (dyn - 8ull * (WMIN + 8)) / (4 * NS);
    const uint64_t r = std::min<uint64_t>({(rows + nsm - 1) / nsm, (uint64_t)RMAX, fit});
    return r >= 2 ? (uint32_t)r : 0u;
}

// entries of the staging window next to `rpb` accumulator rows (a multiple of 4).
// GB_ROWS_WINDOW=n in the environment caps it at n (n >= 8): a diagnostic that makes chunks span
// several windows.
uint32_t rows_window(const RedJob &J, uint32_t rpb, size_t dyn) {
    const uint64_t NS = (J.N + 3u) & ~3u;
    uint64_t w = ((dyn - 4 * rpb * NS) / 8 - 8) & ~uint64_t(3);
    if (const char *e = std::getenv("GB_ROWS_WINDOW")) {
        const long cap = std::atol(e);
        if (cap >= 8) w = std::min<uint64_t>(w, (uint64_t)cap & ~uint64_t(3));
    }
    return (uint32_t)w;
}

}  // namespace

// the tuned schedule of a bucket, or -1 (the shape rules decide)
static int tuned_choice(const gb_ctx *ctx, uint64_t key) {
    const auto it = ctx->tune.table.find(key);
    return it == ctx->tune.table.end() ? -1 : it->second.choice;
}

// the RREF schedule forced by a tuning run or found in the tuned table (single matrices only),
// else -1: 0 CUDA cores with host rounds, 1 CUDA cores in a graph, 2 tensor cores in a graph
static int rref_schedule(const gb_ctx *ctx, uint32_t p, uint32_t nC, uint32_t nb, int nj) {
    if (ctx->tune.force_rref >= 0) return ctx->tune.force_rref;
    return nj == 1 ? tuned_choice(ctx, tune_key(TUNE_RREF, p, nC, nb, 0)) : -1;
}

// ---- the echelon form of a tall, low-rank D' through a random sketch ----------------------------
//
// RREF(D') is the canonical basis of the row space of D'.  For a random R (rs x nC), S = R D'
// spans the same space whenever rank S = rank D', which holds with high probability once rs
// exceeds the rank; then RREF(S) = RREF(D').  S is one product on the tensor cores, and its
// echelon form works on rs rows instead of nC (at the n=13 workload's largest step, 512 rows
// instead of 6864 for a rank of 429).  The result is then checked exactly: every row v of D' must
// be sum_k v[piv_k] RREF(S)_k, i.e. D' - D'[:, piv] RREF(S) = 0 (one more product and a zero
// test).  A sketch of nearly full rank, or a failed check, falls back to the full echelon form,
// so the result is RREF(D') in every case.
constexpr uint32_t SKETCH_ROWS = 512, SKETCH_MIN_ROWS = 2048;

__global__ void k_sketch_rows(uint64_t n, uint32_t cols, uint32_t p, unsigned long long seed, bool rank1,
                              uint32_t *__restrict__ R) {
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < n; t += (uint64_t)gridDim.x * blockDim.x)
        R[t] = (uint32_t)(splitmix64(seed + (rank1 ? t % cols : t)) % p);
}

__global__ void k_gather_pivot_cols(const uint32_t *__restrict__ D, uint32_t nC, uint32_t nb,
                                    const uint32_t *__restrict__ piv, uint32_t rank, uint32_t *__restrict__ A) {
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < (uint64_t)nC * rank;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i = t / rank, k = t % rank;
        A[t] = D[i * nb + piv[k]];
    }
}

__global__ void k_any_nonzero(const uint32_t *__restrict__ C, uint32_t rows, uint32_t cols, uint64_t ld,
                              uint32_t *__restrict__ flag) {
    bool nz = false;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < (uint64_t)rows * cols;
         t += (uint64_t)gridDim.x * blockDim.x)
        nz |= C[(t / cols) * ld + t % cols] != 0u;
    if (__any_sync(0xffffffffu, nz) && (threadIdx.x & 31) == 0) atomicOr(flag, 1u);
}

static unsigned grid_of(uint64_t items) {
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((items + 255) / 256, 148ull * 16));
}

static uint64_t env_u64(const char *name, uint64_t fallback) {
    const char *v = std::getenv(name);
    return v ? std::strtoull(v, nullptr, 0) : fallback;
}

// true: E->rank, rref, rpiv hold RREF(E->dprime); false: nothing is set (the caller runs the full
// echelon form).  GB_SKETCH_ROWS / GB_SKETCH_RANK1 in the environment are test hooks: fewer sketch
// rows, or a sketch of rank one (whose check must fail on a matrix of larger rank).
static bool echelon_by_sketch(gb_ctx *ctx, gb_echelon *E, const Fp &fp, uint32_t *derr) {
    Arena &ar = ctx->arena;
    cudaStream_t st = ctx->stream;
    const uint32_t nC = E->nC, nb = E->nb;
    const uint32_t rs = (uint32_t)std::min<uint64_t>(env_u64("GB_SKETCH_ROWS", SKETCH_ROWS), nC / 2);
    const uint32_t margin = std::min<uint32_t>(32, rs / 4);
    if (rs < 8) return false;
    const bool rank1 = env_u64("GB_SKETCH_RANK1", 0) != 0;
    DBuf<uint32_t> R;
    R.alloc(ar, (size_t)rs * nC, st);
    k_sketch_rows<<<grid_of((uint64_t)rs * nC), 256, 0, st>>>((uint64_t)rs * nC, nC, fp.p, 0x243F6A8885A308D3ull,
                                                               rank1, R.p);
    counted();
    gb_echelon Es;
    Es.nC = rs;
    Es.nb = nb;
    {
        const uint64_t lds = (nb + 3) / 4 * 4;
        DBuf<uint32_t> S;
        S.alloc(ar, (size_t)rs * lds, st);
        GB_CUDA(cudaMemsetAsync(S.p, 0, 4ull * rs * lds, st));
        matmul_dev(ar, fp, rs, nb, nC, R.p, nC, E->dprime.p, nb, S.p, lds, false, derr, st);
        R.reset();
        Es.dprime.alloc(ar, (size_t)rs * nb, st);
        GB_CUDA(cudaMemcpy2DAsync(Es.dprime.p, 4ull * nb, S.p, 4ull * lds, 4ull * nb, rs, cudaMemcpyDeviceToDevice, st));
    }
    echelon_stage(ctx, {&Es}, {fp}, derr);  // rs < SKETCH_MIN_ROWS rows: the full path
    const uint32_t rank = Es.rank;
    if (rank + margin > rs) return false;   // the sketch may not hold the whole row space
    DBuf<uint32_t> flag;
    flag.alloc(ar, 1, st);
    GB_CUDA(cudaMemsetAsync(flag.p, 0, 4, st));
    if (rank) {
        const uint64_t ldc = (nb + 3) / 4 * 4;
        DBuf<uint32_t> A, C;
        A.alloc(ar, (size_t)nC * rank, st);
        k_gather_pivot_cols<<<grid_of((uint64_t)nC * rank), 256, 0, st>>>(E->dprime.p, nC, nb, Es.rpiv.p, rank, A.p);
        counted();
        C.alloc(ar, (size_t)nC * ldc, st);
        GB_CUDA(cudaMemcpy2DAsync(C.p, 4ull * ldc, E->dprime.p, 4ull * nb, 4ull * nb, nC, cudaMemcpyDeviceToDevice, st));
        matmul_dev(ar, fp, nC, nb, rank, A.p, rank, Es.rref.p, nb, C.p, ldc, true, derr, st);
        k_any_nonzero<<<grid_of((uint64_t)nC * nb), 256, 0, st>>>(C.p, nC, nb, ldc, flag.p);
        counted();
    } else {
        k_any_nonzero<<<grid_of((uint64_t)nC * nb), 256, 0, st>>>(E->dprime.p, nC, nb, nb, flag.p);
        counted();
    }
    uint32_t *h = static_cast<uint32_t *>(ctx_pinned(ctx, 16));
    GB_CUDA(cudaMemcpyAsync(h, flag.p, 4, cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaMemcpyAsync(h + 1, derr, 4, cudaMemcpyDeviceToHost, st));
    ctx_sync(ctx);
    if (h[1]) fail(GB_ETIMEOUT, "sketched echelon form: a bounded wait in the tensor-core kernel gave up");
    if (h[0]) return false;  // some row of D' lies outside the sketch's row space
    E->rank = rank;
    E->rref = std::move(Es.rref);
    E->rpiv = std::move(Es.rpiv);
    E->sketched = 1;
    return true;
}

// RREF of each job's dense matrix Es[j]->dprime (Es[j]->nC x Es[j]->nb, row pitch nb) over F_p
// with fps[j] (Sec. 9.2 panel elimination): sets Es[j]->rank, rref, rpiv.  Bounded waits of the
// tensor-core updates that give up are flagged in derr.
void echelon_stage(gb_ctx *ctx, const std::vector<gb_echelon *> &Es, const std::vector<Fp> &fps,
                   uint32_t *derr) {
    Arena &ar = ctx->arena;
    cudaStream_t st = ctx->stream;
    const int nj = (int)Es.size();
    std::vector<uint32_t> rank(nj, 0);
    // tall D' (many more rows than its rank, as at the large steps): a random sketch first, on
    // request (measured: no faster than the full form once the panel solve runs on a cluster)
    std::vector<uint8_t> done(nj, 0);
    const uint64_t min_rows = env_u64("GB_SKETCH_MIN_ROWS", SKETCH_MIN_ROWS);
    const uint64_t min_entries = min_rows < SKETCH_MIN_ROWS ? 0 : (1ull << 22);
    if (ctx->flags & GB_CTX_SKETCH)
        for (int j = 0; j < nj; ++j)
            if (Es[j]->nC >= min_rows && Es[j]->nb && (uint64_t)Es[j]->nC * Es[j]->nb >= min_entries)
                done[j] = echelon_by_sketch(ctx, Es[j], fps[j], derr) ? 1 : 0;
    // per-job working state, one allocation each
    std::vector<RrefJob> X(nj);
    std::vector<DBuf<uint32_t>> Mw(nj), lead(nj), pcol(nj), order(nj), panel(nj);
    DBuf<uint32_t> states;  // 4 words per job, then the graph's round count; read back in one copy
    states.alloc(ar, 4ull * nj + 4, st);
    GB_CUDA(cudaMemsetAsync(states.p, 0, 16ull * nj + 16, st));
    RoundGraph graph;
    unsigned graph_nodes = 0;
    std::vector<int> live, smem_jobs, cl_jobs, glob_jobs, tc_jobs;
    // panels of rows wider than this are solved by a cluster of blocks (k_panel_rref_cl);
    // GB_PANEL_CLUSTER_MIN_NB in the environment moves the bound (a test hook)
    const uint64_t panel_cluster_min_nb = env_u64("GB_PANEL_CLUSTER_MIN_NB", PANEL_CLUSTER_MIN_NB);
    std::vector<DigitPlanes> FA(nj), FB(nj);
    std::vector<std::unique_ptr<MmPlan>> plans(nj);
    for (int j = 0; j < nj; ++j) {
        const uint32_t nC = Es[j]->nC, nb = Es[j]->nb;
        X[j] = RrefJob{};
        X[j].nC = nC;
        X[j].nb = nb;
        X[j].fp = fps[j];
        if (!nC || !nb || done[j]) continue;
        X[j].ldm = (nb + 3) / 4 * 4;
        Mw[j].alloc(ar, (size_t)nC * X[j].ldm, st);
        lead[j].alloc(ar, nC, st);
        pcol[j].alloc(ar, nC, st);
        order[j].alloc(ar, std::min(nC, nb), st);
        panel[j].alloc(ar, 3 * KP, st);
        GB_CUDA(cudaMemcpy2DAsync(Mw[j].p, 4ull * X[j].ldm, Es[j]->dprime.p, 4ull * nb, 4ull * nb, nC,
                                  cudaMemcpyDeviceToDevice, st));
        // large D': the trailing update of each panel on the tensor cores
        const int sched = rref_schedule(ctx, fps[j].p, nC, nb, nj);
        if ((ctx->flags & GB_CTX_REDUCE_DENSE) || (sched >= 0 ? sched == 2 : (uint64_t)nC * nb >= (1ull << 22))) {
            const uint32_t L = digits_for(fps[j].p);
            FA[j].alloc(ar, L, nC, KP, st);
            FB[j].alloc(ar, L, nb, KP, st);
            GB_CUDA(cudaMemsetAsync(FA[j].p, 0, FA[j].buf.bytes(), st));
            GB_CUDA(cudaMemsetAsync(FB[j].p, 0, FB[j].buf.bytes(), st));
            X[j].tc = 1;
            X[j].fa = FA[j].p;
            X[j].fb = FB[j].p;
            X[j].fkp = FA[j].kpad;
            plans[j] = std::make_unique<MmPlan>(FA[j], FB[j], Mw[j].p, X[j].ldm, nC, nb, fps[j]);
            tc_jobs.push_back(j);
        }
        X[j].M = Mw[j].p;
        X[j].lead = lead[j].p;
        X[j].pcol = pcol[j].p;
        X[j].order = order[j].p;
        X[j].state = states.p + 4 * j;
        X[j].panel = panel[j].p;
        live.push_back(j);
        if (nb >= panel_cluster_min_nb && nb <= PANEL_CLUSTER_MAX_NB) cl_jobs.push_back(j);
        else if (4ull * KP * nb <= 200 * 1024) smem_jobs.push_back(j);
        else glob_jobs.push_back(j);
    }
    if (!live.empty()) {
        std::vector<uint32_t> rows(nj, 0);
        for (int j : live) rows[j] = X[j].nC;
        Grouped<RrefJob> G;
        G.build(ctx, X, {rows});
        DBuf<int> lists;
        lists.alloc(ar, (size_t)nj + 1, st);
        {
            std::vector<int> l(smem_jobs);
            l.insert(l.end(), cl_jobs.begin(), cl_jobs.end());
            l.insert(l.end(), glob_jobs.begin(), glob_jobs.end());
            int *hl = static_cast<int *>(ctx_pinned(ctx, 4ull * (l.size() + 1)));
            std::memcpy(hl, l.data(), 4 * l.size());
            GB_CUDA(cudaMemcpyAsync(lists.p, hl, 4 * l.size(), cudaMemcpyHostToDevice, st));
        }
        size_t pan_bytes = 0;
        for (int j : smem_jobs) pan_bytes = std::max<size_t>(pan_bytes, 4ull * KP * X[j].nb);
        if (!smem_jobs.empty()) opt_in_smem(reinterpret_cast<const void *>(k_panel_rref<true>));
        size_t cl_bytes = 0;
        for (int j : cl_jobs) cl_bytes = std::max<size_t>(cl_bytes, 4ull * KP * ((X[j].nb + PCS - 1) / PCS));
        if (!cl_jobs.empty()) opt_in_smem(reinterpret_cast<const void *>(k_panel_rref_cl));
        // jobs are packed in the job table at their own index; k_pick_panel runs on all of them
        // (a job without rows has no blocks elsewhere and its state stays zero)
        k_leads<<<G.totals[0], 256, 0, st>>>(G.jobs, G.plans[0], nj);
        counted();
        // every round turns each of its rows into a pivot row or a zero row
        uint32_t maxrounds = 1;
        for (int j : live) maxrounds = std::max<uint32_t>(maxrounds, (X[j].nC + KP - 1) / KP + 1);
        // one round: each job picks its next panel, reduces it, and eliminates the panel's
        // pivot columns from all its other rows
        auto round = [&](cudaStream_t s) {
            k_pick_panel<<<nj, 1024, 0, s>>>(G.jobs);
            if (!smem_jobs.empty())
                k_panel_rref<true><<<(unsigned)smem_jobs.size(), PT, pan_bytes, s>>>(G.jobs, lists.p);
            if (!cl_jobs.empty())
                k_panel_rref_cl<<<(unsigned)(PCS * cl_jobs.size()), PCT, cl_bytes, s>>>(G.jobs,
                                                                                      lists.p + smem_jobs.size());
            if (!glob_jobs.empty())
                k_panel_rref<false><<<(unsigned)glob_jobs.size(), PT, 0, s>>>(
                    G.jobs, lists.p + smem_jobs.size() + cl_jobs.size());
            k_eliminate<<<G.totals[0], 256, 0, s>>>(G.jobs, G.plans[0], nj);
            counted(2 + (smem_jobs.empty() ? 0 : 1) + (cl_jobs.empty() ? 0 : 1) + (glob_jobs.empty() ? 0 : 1));
            for (int j : tc_jobs) {
                const unsigned nt = (unsigned)(((size_t)X[j].nC + X[j].nb) * KP);
                if (FA[j].L == 2) k_elim_digits<2><<<(nt + 255) / 256, 256, 0, s>>>(G.jobs, j);
                else k_elim_digits<4><<<(nt + 255) / 256, 256, 0, s>>>(G.jobs, j);
                counted();
                plans[j]->update(0, 0, 0, 0, 0, 0, X[j].nC, X[j].nb, KP, true, derr, s);
                k_leads_np<<<X[j].nC, 256, 0, s>>>(G.jobs, j);
                counted();
            }
        };
        int sched = -1;
        for (int j : live) sched = std::max(sched, rref_schedule(ctx, fps[j].p, X[j].nC, X[j].nb, nj));
        if (!(ctx->flags & GB_CTX_NO_GRAPHS) && (sched >= 0 ? sched >= 1 : maxrounds >= GRAPH_MIN_ROUNDS)) {
            // the whole loop as one graph: the rounds repeat on the device until no job has
            // rows left, with no host round trip between them
            unsigned per_round = 0;
            graph = record_round_loop(ctx, [&](cudaStream_t s, cudaGraphConditionalHandle more) {
                round(s);
                k_rref_more<<<1, 32, 0, s>>>(G.jobs, nj, states.p + 4 * nj, maxrounds, more);
                counted();
            }, per_round);
            GB_CUDA(cudaGraphLaunch(graph.exec, st));
            g_graph_launches.fetch_add(1, std::memory_order_relaxed);
            graph_nodes = per_round;
        } else {
            uint32_t rounds = 0;
            for (;;) {
                const uint32_t group = rounds == 0 ? 2 : 4;
                for (uint32_t g = 0; g < group; ++g) round(st);
                rounds += group;
                uint32_t *h = static_cast<uint32_t *>(ctx_pinned(ctx, 16ull * nj));
                GB_CUDA(cudaMemcpyAsync(h, states.p, 16ull * nj, cudaMemcpyDeviceToHost, st));
                ctx_sync(ctx);
                bool more = false;
                for (int j : live) {
                    const uint32_t *s = h + 4 * j;
                    if (s[1] != 0 && s[3] > s[1]) more = true;
                }
                if (!more || rounds >= maxrounds) break;
            }
        }
        // one more pick confirms that no non-zero non-pivot row is left
        k_pick_panel<<<nj, 1024, 0, st>>>(G.jobs);
        counted();
        uint32_t *h = static_cast<uint32_t *>(ctx_pinned(ctx, 16ull * nj + 16));
        GB_CUDA(cudaMemcpyAsync(h, states.p, 16ull * nj + 16, cudaMemcpyDeviceToHost, st));
        ctx_sync(ctx);
        if (graph.exec) counted(graph_nodes * h[4 * nj]);  // rounds the graph ran
        graph.reset();
        for (int j : live) {
            if (h[4 * j + 1] != 0) fail(GB_EDEVICE, "RREF: rows left after the last round");
            rank[j] = h[4 * j];
        }
        // gather the pivot rows in order
        std::vector<uint32_t> prow(nj, 0);
        for (int j : live) {
            Es[j]->rank = rank[j];
            Es[j]->rref.alloc(ar, (size_t)rank[j] * X[j].nb, st);
            Es[j]->rpiv.alloc(ar, rank[j], st);
            X[j].out = Es[j]->rref.p;
            X[j].opiv = Es[j]->rpiv.p;
            X[j].rank = rank[j];
            prow[j] = rank[j];
        }
        Grouped<RrefJob> G2;
        G2.build(ctx, X, {prow});
        if (G2.totals[0]) {
            k_gather_rref<<<G2.totals[0], 256, 0, st>>>(G2.jobs, G2.plans[0], nj);
            counted();
        }
    }
}

std::vector<std::unique_ptr<gb_echelon>> reduce_rows(const std::vector<gb_macaulay *> &Ms, bool echelon) {
    std::vector<std::unique_ptr<gb_echelon>> Es;
    if (Ms.empty()) return Es;
    gb_ctx *ctx = Ms[0]->sys->ctx;
    Arena &ar = ctx->arena;
    cudaStream_t st = ctx->stream;
    const int nj = (int)Ms.size();
    MmTimer mm_timer;
    mm_timer.ctx = ctx;
    struct TimerScope {
        MmTimer *prev;
        explicit TimerScope(MmTimer *t) : prev(t_mm_timer) { t_mm_timer = t; }
        ~TimerScope() { t_mm_timer = prev; }
    } mm_scope(&mm_timer);
    GB_CUDA(cudaEventRecord(ctx->ev[2], st));
    DBuf<unsigned long long> work;
    work.alloc(ar, 2ull * nj, st);
    GB_CUDA(cudaMemsetAsync(work.p, 0, 16ull * nj, st));
    std::vector<RedJob> R(nj);
    std::vector<DBuf<uint32_t>> Ubuf(nj);
    std::vector<int> mode(nj, A32);
    for (int j = 0; j < nj; ++j) {
        gb_macaulay *Mac = Ms[j];
        gb_system *S = Mac->sys;
        auto E = std::make_unique<gb_echelon>();
        E->mac = Mac;
        E->nC = Mac->nC;
        E->nb = Mac->nb;
        E->dprime.alloc(ar, (size_t)Mac->nC * Mac->nb, st);
        const uint32_t nchunks = std::max<uint32_t>((Mac->nA + CW - 1) / CW, 1);
        Ubuf[j].alloc(ar, (size_t)nchunks * CW * CW, st);
        GB_CUDA(cudaMemsetAsync(Ubuf[j].p, 0, 4ull * nchunks * CW * CW, st));
        RedJob &J = R[j];
        J = RedJob{Mac->row_ptr.p, Mac->col.p, Mac->val.p, Mac->pcols.p, Mac->colpos.p, Mac->nonpiv.p,
                   Ubuf[j].p, E->dprime.p, nullptr, nullptr, work.p + 2 * j, Mac->nA, Mac->nC, Mac->ndict, Mac->nb,
                   S->fp};
        mode[j] = !S->fp.small ? M64 : (Mac->nA < 65536u ? A32 : A64);
        Es.push_back(std::move(E));
    }
    // path of each matrix: dense blocked elimination on the tensor cores (dense.cu) or the sparse
    // row-by-row reduction below
    std::vector<uint8_t> dense(nj, 0);
    {
        size_t room = ar.capacity() > ar.used() ? ar.capacity() - ar.used() : 0;
        for (int j = 0; j < nj; ++j) {
            const RedJob &J = R[j];
            if (!J.nC || !J.nb || !J.nA || (ctx->flags & GB_CTX_REDUCE_SPARSE)) continue;
            // a dense matrix runs its own launch sequence, while the sparse kernels cover every
            // matrix of a batch in one launch: inside a batch only very large matrices go dense
            bool want = dense_pays(J.fp.p, J.N, J.nA, J.nC) && (nj == 1 || J.nA >= 16384);
            const int tuned = nj == 1 ? tuned_choice(ctx, tune_key(TUNE_REDUCE, J.fp.p, J.nA, J.nC, J.nb)) : -1;
            if (ctx->flags & GB_CTX_REDUCE_DENSE) want = true;
            else if (ctx->tune.force_reduce >= 0) want = ctx->tune.force_reduce == 1;
            else if (tuned >= 0) want = tuned == 1;
            const size_t need = dense_bytes(J.fp.p, J.N, J.nA, J.nC);
            if (want && need + (64u << 20) < room) {
                dense[j] = 1;
                room -= need;
            }
        }
    }
    DBuf<uint32_t> derr;
    derr.alloc(ar, 1, st);
    GB_CUDA(cudaMemsetAsync(derr.p, 0, 4, st));
    // accumulators: shared memory per block when N fits, else one global row per block; launch
    // groups by mode and by the shared-memory size class (powers of two)
    std::vector<DBuf<unsigned char>> gbuf(nj);
    std::vector<DBuf<uint32_t>> sbuf(nj);
    uint64_t sparse_rows = 0;
    for (int j = 0; j < nj; ++j)
        if (R[j].nC && R[j].nb && !dense[j]) sparse_rows += R[j].nC;
    std::map<std::pair<int, int>, std::vector<int>> groups;  // (mode, size class or -1) -> jobs
    const size_t rows_dyn = rows_dyn_smem();
    for (int j = 0; j < nj; ++j) {
        if (!R[j].nC || !R[j].nb || dense[j]) continue;
        const size_t accb = mode[j] == A32 ? 4 : 8;
        const size_t bytes = (size_t)R[j].N * accb;
        int cls = -1;
        if (use_cluster(R[j], accb, sparse_rows)) {
            cls = -2;  // rows split over clusters of CS blocks (k_reduce_cl)
            sbuf[j].alloc(ar, (size_t)std::max<uint32_t>(R[j].nA, 1) * (CS + 1), st);
            R[j].split = sbuf[j].p;
        } else if (mode[j] == A32 && (R[j].rpb = rows_per_block(R[j], sparse_rows, rows_dyn)) >= 2) {
            cls = -3;  // several rows per block sharing the staged pivot entries (k_reduce_rows)
            R[j].win = rows_window(R[j], R[j].rpb, rows_dyn);
        } else if (bytes <= 200 * 1024) {
            cls = 0;
            while (((size_t)1024 << cls) < bytes) ++cls;
        } else {
            gbuf[j].alloc(ar, (size_t)R[j].nC * bytes, st);
            R[j].gacc = gbuf[j].p;
        }
        groups[{mode[j], cls}].push_back(j);
    }
    {
        std::vector<uint32_t> tri(nj), inv(nj), spl(nj, 0);
        for (int j = 0; j < nj; ++j) {
            tri[j] = blocks(R[j].nA, 8);
            inv[j] = blocks(((size_t)R[j].nA + CW - 1) / CW, IW);
            if (R[j].split) spl[j] = blocks(R[j].nA, 8);
        }
        std::vector<std::vector<uint32_t>> per{tri, inv, spl};
        for (auto &g : groups) {
            std::vector<uint32_t> rows(nj, 0);
            // blocks, clusters of CS blocks for class -2, blocks of rpb rows for class -3
            for (int j : g.second) rows[j] = g.first.second == -3 ? (R[j].nC + R[j].rpb - 1) / R[j].rpb : R[j].nC;
            per.push_back(rows);
        }
        Grouped<RedJob> G;
        G.build(ctx, R, per);
        if (G.totals[0]) {
            k_build_chunk_tri<<<G.totals[0], 256, 0, st>>>(G.jobs, G.plans[0], nj);
            k_invert_chunk_tri<<<G.totals[1], IW * 32, 0, st>>>(G.jobs, G.plans[1], nj);
            counted(2);
        }
        if (G.totals[2]) {
            k_split<<<G.totals[2], 256, 0, st>>>(G.jobs, G.plans[2], nj);
            counted();
        }
        GB_CUDA(cudaEventRecord(ctx->ev[5], st));
        for (int j = 0; j < nj; ++j) {
            if (!dense[j]) continue;
            const RedJob &J = R[j];
            DenseJob D{};
            D.row_ptr = J.row_ptr;
            D.col = J.col;
            D.val = J.val;
            D.colpos = J.colpos;
            D.pcols = J.pcols;
            D.Uinv = J.U;
            D.N = J.N;
            D.nA = J.nA;
            D.nC = J.nC;
            D.nb = J.nb;
            D.fp = J.fp;
            D.work = J.work;
            reduce_dense(D, J.dprime, ar, derr.p, st);
        }
        size_t gi = 3;
        for (auto &g : groups) {
            const int md = g.first.first, cls = g.first.second;
            if (cls == -3) {
                opt_in_smem(reinterpret_cast<const void *>(k_reduce_rows));
                k_reduce_rows<<<G.totals[gi], RB, rows_dyn, st>>>(G.jobs, G.plans[gi], nj);
                counted();
                ++gi;
                continue;
            }
            if (cls == -2) {
                size_t dyn = 0;
                for (int j : g.second)
                    dyn = std::max<size_t>(dyn, (size_t)((R[j].N + CS - 1) / CS) * (md == A32 ? 4 : 8));
                auto goc = [&](auto kern) {
                    opt_in_smem(reinterpret_cast<const void *>(kern));
                    kern<<<G.totals[gi] * CS, RT, dyn, st>>>(G.jobs, G.plans[gi], nj);
                    counted();
                };
                if (md == A32) goc(k_reduce_cl<A32>);
                else if (md == A64) goc(k_reduce_cl<A64>);
                else goc(k_reduce_cl<M64>);
                ++gi;
                continue;
            }
            const bool smem = cls >= 0;
            size_t dyn = 0;
            if (smem)
                for (int j : g.second) dyn = std::max<size_t>(dyn, (size_t)R[j].N * (md == A32 ? 4 : 8));
            auto go = [&](auto kern) {
                if (smem) opt_in_smem(reinterpret_cast<const void *>(kern));
                kern<<<G.totals[gi], RT, dyn, st>>>(G.jobs, G.plans[gi], nj);
                counted();
            };
            if (md == A32) { if (smem) go(k_reduce<A32, true>); else go(k_reduce<A32, false>); }
            else if (md == A64) { if (smem) go(k_reduce<A64, true>); else go(k_reduce<A64, false>); }
            else { if (smem) go(k_reduce<M64, true>); else go(k_reduce<M64, false>); }
            ++gi;
        }
    }
    GB_CUDA(cudaEventRecord(ctx->ev[3], st));

    if (echelon) {
        std::vector<gb_echelon *> Ep(nj);
        std::vector<Fp> fps(nj);
        for (int j = 0; j < nj; ++j) {
            Ep[j] = Es[j].get();
            fps[j] = R[j].fp;
        }
        echelon_stage(ctx, Ep, fps, derr.p);
    }
    GB_CUDA(cudaEventRecord(ctx->ev[4], st));
    uint64_t *hw = static_cast<uint64_t *>(ctx_pinned(ctx, 16ull * nj + 16));
    GB_CUDA(cudaMemcpyAsync(hw, work.p, 16ull * nj, cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaMemcpyAsync(hw + 2 * nj, derr.p, 4, cudaMemcpyDeviceToHost, st));
    ctx_sync(ctx);
    if (*reinterpret_cast<const uint32_t *>(hw + 2 * nj))
        fail(GB_ETIMEOUT, "dense reduction: a bounded wait in the tensor-core kernel gave up");
    float ms_red = 0.f, ms_rref = 0.f, ms_kern = 0.f;
    GB_CUDA(cudaEventElapsedTime(&ms_red, ctx->ev[2], ctx->ev[3]));
    GB_CUDA(cudaEventElapsedTime(&ms_kern, ctx->ev[5], ctx->ev[3]));
    GB_CUDA(cudaEventElapsedTime(&ms_rref, ctx->ev[3], ctx->ev[4]));
    const double ms_mm = mm_timer.elapsed_ms();
    for (int j = 0; j < nj; ++j) {
        Es[j]->ms_mm = ms_mm;
        Es[j]->mm_flops = mm_timer.flops;
        Es[j]->mm_launches = mm_timer.launches;
        Es[j]->work[0] = hw[2 * j];
        Es[j]->work[1] = hw[2 * j + 1];
        Es[j]->ms_reduce = ms_red;
        Es[j]->ms_rref = ms_rref;
        Es[j]->ms_reduce_kernel = ms_kern;
    }
    return Es;
}

void append_echelon(const std::vector<gb_echelon *> &Es, std::vector<std::vector<Mono>> &lms) {
    lms.assign(Es.size(), {});
    if (Es.empty()) return;
    gb_ctx *ctx = Es[0]->mac->sys->ctx;
    Arena &ar = ctx->arena;
    cudaStream_t st = ctx->stream;
    const int nj = (int)Es.size();
    uint64_t tot = 0;
    std::vector<uint64_t> roff(nj);
    for (int j = 0; j < nj; ++j) {
        roff[j] = tot;
        tot += Es[j]->rank;
    }
    if (!tot) return;
    DBuf<uint32_t> cnt, scan;
    DBuf<uint4> lmd;
    cnt.alloc(ar, tot, st);
    scan.alloc(ar, tot + 1, st);
    lmd.alloc(ar, tot, st);
    std::vector<RowsJob> J(nj);
    std::vector<uint32_t> rows(nj);
    for (int j = 0; j < nj; ++j) {
        gb_echelon *E = Es[j];
        J[j] = RowsJob{E->rref.p, E->rpiv.p, E->mac->nonpiv.p, E->mac->dict.p, nullptr, E->rank, E->rank, E->nb,
                       E->mac->n, 0, cnt.p + roff[j], scan.p + roff[j], lmd.p + roff[j], nullptr, nullptr,
                       nullptr, nullptr};
        rows[j] = E->rank;
    }
    {
        Grouped<RowsJob> G;
        G.build(ctx, J, {rows});
        k_count_rows<<<G.totals[0], 256, 0, st>>>(G.jobs, G.plans[0], nj);
        counted();
    }
    exclusive_scan(ctx, cnt.p, scan.p, tot, st);
    char *h = static_cast<char *>(ctx_pinned(ctx, 4ull * (tot + 1) + 16ull * tot + 64));
    uint32_t *hs = reinterpret_cast<uint32_t *>(h);
    Mono *hl = reinterpret_cast<Mono *>(h + ((4ull * (tot + 1) + 15) & ~15ull));
    GB_CUDA(cudaMemcpyAsync(hs, scan.p, 4ull * (tot + 1), cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaMemcpyAsync(hl, lmd.p, 16ull * tot, cudaMemcpyDeviceToHost, st));
    ctx_sync(ctx);
    // room in every basis, and the new elements' offsets and lengths
    std::vector<uint32_t> hoff_all(tot + 1);
    std::memcpy(hoff_all.data(), hs, 4ull * (tot + 1));
    Stage offs;
    std::vector<size_t> at(nj), at_len(nj);
    for (int j = 0; j < nj; ++j) {
        gb_system *S = Es[j]->mac->sys;
        const uint32_t rank = Es[j]->rank;
        lms[j].assign(hl + roff[j], hl + roff[j] + rank);
        if (!rank) continue;
        const uint32_t b0 = hoff_all[roff[j]];
        const uint64_t add = hoff_all[roff[j] + rank] - b0;
        const uint64_t base = S->nterms;
        if (base + add >= (1ull << 32)) fail(GB_EUNSUPPORTED, "basis above 2^32 terms");
        const size_t ng0 = S->off.size();
        if (base + add > S->bmon.n) {
            S->bmon.grow(ar, std::max<size_t>(base + add, 2 * S->bmon.n), base, st);
            S->bkey.grow(ar, std::max<size_t>(base + add, 2 * S->bkey.n), base, st);
            S->bcf.grow(ar, std::max<size_t>(base + add, 2 * S->bcf.n), base, st);
        }
        if (ng0 + rank > S->boff.n) {
            S->boff.grow(ar, std::max<size_t>(ng0 + rank, 2 * S->boff.n), ng0, st);
            S->blen.grow(ar, std::max<size_t>(ng0 + rank, 2 * S->blen.n), ng0, st);
        }
        std::vector<uint32_t> noff(rank), nlen(rank);
        for (uint32_t e = 0; e < rank; ++e) {
            noff[e] = (uint32_t)(base + hoff_all[roff[j] + e] - b0);
            nlen[e] = hoff_all[roff[j] + e + 1] - hoff_all[roff[j] + e];
        }
        at[j] = offs.put(noff.data(), 4ull * rank);
        at_len[j] = offs.put(nlen.data(), 4ull * rank);
        S->nterms = base + add;
        for (uint32_t e = 0; e < rank; ++e) {
            S->off.push_back(noff[e]);
            S->len.push_back(nlen[e]);
        }
    }
    DBuf<char> d;
    offs.upload(ctx, d);
    for (int j = 0; j < nj; ++j) {
        gb_system *S = Es[j]->mac->sys;
        const uint32_t rank = Es[j]->rank;
        if (!rank) continue;
        const size_t ng0 = S->off.size() - rank;
        GB_CUDA(cudaMemcpyAsync(S->boff.p + ng0, d.p + at[j], 4ull * rank, cudaMemcpyDeviceToDevice, st));
        GB_CUDA(cudaMemcpyAsync(S->blen.p + ng0, d.p + at_len[j], 4ull * rank, cudaMemcpyDeviceToDevice, st));
        J[j].dst_off = S->boff.p + ng0;
        J[j].omon = S->bmon.p;
        J[j].okey = S->bkey.p;
        J[j].ocf = S->bcf.p;
    }
    Grouped<RowsJob> G;
    G.build(ctx, J, {rows});
    k_write_rows<<<G.totals[0], 256, 0, st>>>(G.jobs, G.plans[0], nj);
    counted();
}

void replace_tails(const std::vector<gb_echelon *> &Es, const std::vector<std::vector<uint32_t>> &elems) {
    if (Es.empty()) return;
    gb_ctx *ctx = Es[0]->mac->sys->ctx;
    Arena &ar = ctx->arena;
    cudaStream_t st = ctx->stream;
    const int nj = (int)Es.size();
    const auto tt0 = std::chrono::steady_clock::now();
    auto tms = [&] { return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tt0).count(); };
    // element elems[j][i] becomes LM + (row i of job j's D'), compacted on the device
    uint64_t tot = 0;
    std::vector<uint64_t> roff(nj);
    for (int j = 0; j < nj; ++j) {
        roff[j] = tot;
        tot += elems[j].size();
    }
    if (!tot) {
        for (int j = 0; j < nj; ++j) {
            gb_system *S = Es[j]->mac->sys;
            S->fin_off.assign(1, 0);
            S->fin_exps.reset();
            S->fin_cf.reset();
            S->fin_terms = 0;
        }
        return;
    }
    DBuf<uint32_t> cnt, scan;
    DBuf<uint4> lead;
    cnt.alloc(ar, tot, st);
    scan.alloc(ar, tot + 1, st);
    lead.alloc(ar, tot, st);
    std::vector<uint4> hl(tot);
    for (int j = 0; j < nj; ++j)
        for (size_t i = 0; i < elems[j].size(); ++i) hl[roff[j] + i] = to_u4(Es[j]->mac->sys->lm[elems[j][i]]);
    {
        Stage s;
        const size_t o = s.put(hl.data(), 16ull * tot);
        DBuf<char> d;
        s.upload(ctx, d);
        GB_CUDA(cudaMemcpyAsync(lead.p, d.p + o, 16ull * tot, cudaMemcpyDeviceToDevice, st));
    }
    std::vector<RowsJob> J(nj);
    std::vector<uint32_t> rows(nj);
    for (int j = 0; j < nj; ++j) {
        gb_echelon *E = Es[j];
        J[j] = RowsJob{E->dprime.p, nullptr, E->mac->nonpiv.p, E->mac->dict.p, lead.p + roff[j],
                       (uint32_t)elems[j].size(), E->nC, E->nb, E->mac->n, 1, cnt.p + roff[j], scan.p + roff[j],
                       nullptr, nullptr, nullptr, nullptr, nullptr};
        rows[j] = (uint32_t)elems[j].size();
    }
    {
        Grouped<RowsJob> G;
        G.build(ctx, J, {rows});
        k_count_rows<<<G.totals[0], 256, 0, st>>>(G.jobs, G.plans[0], nj);
        counted();
    }
    exclusive_scan(ctx, cnt.p, scan.p, tot, st);
    std::vector<uint32_t> hs(tot + 1);
    {
        uint32_t *hp = static_cast<uint32_t *>(ctx_pinned(ctx, 4ull * (tot + 1)));
        GB_CUDA(cudaMemcpyAsync(hp, scan.p, 4ull * (tot + 1), cudaMemcpyDeviceToHost, st));
        ctx_sync(ctx);
        std::memcpy(hs.data(), hp, 4ull * (tot + 1));
    }
    const double t_count = tms();
    // each system's terms go to device buffers of its own, which it keeps
    for (int j = 0; j < nj; ++j) {
        gb_system *S = Es[j]->mac->sys;
        const uint32_t b = hs[roff[j]], e = hs[roff[j] + elems[j].size()];
        S->fin_off.resize(elems[j].size() + 1);
        for (size_t i = 0; i <= elems[j].size(); ++i) S->fin_off[i] = hs[roff[j] + i] - b;
        S->fin_terms = e - b;
        S->fin_cf.alloc(ar, e - b, st);
        S->fin_exps.alloc(ar, (size_t)(e - b) * S->n, st);
        J[j].ocf = S->fin_cf.p;
        J[j].oexp = S->fin_exps.p;
    }
    {
        Grouped<RowsJob> G;
        G.build(ctx, J, {rows});
        k_write_rows<<<G.totals[0], 256, 0, st>>>(G.jobs, G.plans[0], nj);
        counted();
    }
    if (trace_on()) {
        ctx_sync(ctx);
        std::fprintf(stderr, "[gb] tails: %llu rows, %u terms; count+scan %.3f ms, write %.3f ms\n",
                     (unsigned long long)tot, hs[tot], t_count, tms() - t_count);
    }
}

// ---- the sparse reduction without device allocation --------------------------------------------
//
// Scratch of gb_reduce_rows_noalloc: pivot-column flags (one word per dictionary column), the
// 32 x 32 chunk triangles (one per 32 pivot rows), the two work counters of k_reduce, an error
// word and the one-job table, carved out of one fixed array that is part of the library image.
// Host code reaches it only through the address cudaGetSymbolAddress returns for the current
// device.
constexpr uint32_t NA_COLPOS = 0;
constexpr uint32_t NA_TRI = GB_NOALLOC_MAX_DICT;
constexpr uint32_t NA_WORK = NA_TRI + GB_NOALLOC_MAX_PIVOTS * CW;  // even: 8-byte aligned
constexpr uint32_t NA_ERR = NA_WORK + 4;
constexpr uint32_t NA_TABLE = NA_WORK + 8;                           // 16-byte aligned
// the one-job table: the job, then the block-start tables {0, blocks} of its three launches
struct NoallocTable {
    RedJob job;
    uint32_t tri_start[2], inv_start[2], red_start[2];
};
constexpr uint32_t NA_WORDS = NA_TABLE + (uint32_t)((sizeof(NoallocTable) + 15) / 4);
static __device__ __align__(256) uint32_t g_noalloc_scratch[NA_WORDS];

// The caller's indices become shared- and scratch-memory addresses in the kernels below, so they
// are checked first, a warp per row: row pointers non-decreasing, columns strictly ascending
// within a row and below N, each pivot row opening at its pivot column, pivot columns strictly
// ascending, non-pivot columns below N.  Any failure sets *err.
__global__ void k_noalloc_check(uint32_t N, uint32_t nA, uint32_t nrows, uint32_t nb,
                                const uint32_t *__restrict__ row_ptr, const uint32_t *__restrict__ col,
                                const uint32_t *__restrict__ pcols, const uint32_t *__restrict__ nonpiv,
                                uint32_t *__restrict__ err) {
    const int lane = threadIdx.x & 31;
    const uint32_t warp0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    bool bad = false;
    for (uint32_t i = warp0; i < nrows; i += nwarps) {
        const uint32_t a = row_ptr[i], b = row_ptr[i + 1];
        if (b < a) { bad = true; continue; }  // the same on every lane
        if (i < nA) {
            const uint32_t pc = pcols[i];
            bad |= pc >= N || a == b || (a < b && col[a] != pc) || (i > 0 && pcols[i - 1] >= pc);
        }
        for (uint32_t q = a + lane; q < b; q += 32) {
            const uint32_t c = col[q];
            bad |= c >= N || (q > a && col[q - 1] >= c);
        }
    }
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < nb; j += gridDim.x * blockDim.x)
        bad |= nonpiv[j] >= N;
    if (bad) atomicOr(err, 1u);
}

// the table arrives as a kernel parameter; after a failed check the job is empty (no pivot rows,
// no rows, no output columns), so the shared kernels below touch nothing
__global__ void k_noalloc_setup(NoallocTable tb, NoallocTable *__restrict__ dst, const uint32_t *__restrict__ err) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        if (*err) tb.job.nA = tb.job.nC = tb.job.nb = 0;
        *dst = tb;
    }
}

__global__ void k_noalloc_mark(uint32_t N, uint32_t nA, const uint32_t *__restrict__ pcols, uint32_t *__restrict__ colpos) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nA && pcols[k] < N) colpos[pcols[k]] = k | 0x80000000u;
}

// after a failed check D' reads 0xFFFFFFFF everywhere: never a residue of a prime below 2^31
__global__ void k_noalloc_poison(size_t n, uint32_t *__restrict__ dprime, const uint32_t *__restrict__ err) {
    if (!*err) return;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
        dprime[t] = 0xFFFFFFFFu;
}

namespace {
uint32_t *noalloc_scratch_for_current_device() {
    static std::mutex mu;
    static uint32_t *addr[64] = {};
    int dev = 0;
    GB_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) fail(GB_EUNSUPPORTED, "device ordinal above 63");
    std::lock_guard<std::mutex> g(mu);
    if (!addr[dev]) {
        void *ptr = nullptr;
        GB_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
        addr[dev] = static_cast<uint32_t *>(ptr);
    }
    return addr[dev];
}
}  // namespace

void reduce_rows_noalloc(uint32_t p, uint32_t N, uint32_t nA, uint32_t nC, uint32_t nb,
                         const uint32_t *row_ptr, const uint32_t *col, const uint32_t *val,
                         const uint32_t *pcols, const uint32_t *nonpiv, uint32_t *dprime,
                         cudaStream_t st) {
    if (p < 3 || p >= (1u << 31) || !is_prime32(p)) fail(GB_EINVAL, "p must be an odd prime below 2^31");
    const Fp fp = make_fp(p);
    const int mode = fp.small ? A32 : M64;
    const uint32_t max_dict = fp.small ? GB_NOALLOC_MAX_DICT : GB_NOALLOC_MAX_DICT / 2;
    if (N > max_dict || nA > GB_NOALLOC_MAX_PIVOTS)
        fail(GB_EINVAL, "gb_reduce_rows_noalloc: ndict above " + std::to_string(max_dict) +
                            " or npivot above " + std::to_string(GB_NOALLOC_MAX_PIVOTS));
    if (nb > N || nA > N) fail(GB_EINVAL, "gb_reduce_rows_noalloc: more pivots or non-pivot columns than columns");
    if (nC > (1u << 31) / (nb ? nb : 1)) fail(GB_EINVAL, "gb_reduce_rows_noalloc: D' above 2^31 entries");
    if (!nC || !nb) return;
    if (!row_ptr || !col || !val || (nA && !pcols) || !nonpiv || !dprime)
        fail(GB_EINVAL, "gb_reduce_rows_noalloc: null device pointer");
    uint32_t *scr = noalloc_scratch_for_current_device();
    uint32_t *colpos = scr + NA_COLPOS, *tri = scr + NA_TRI, *err = scr + NA_ERR;
    unsigned long long *work = reinterpret_cast<unsigned long long *>(scr + NA_WORK);
    const uint32_t nchunks = (nA + CW - 1) / CW;
    // the array keeps the previous call's contents: clear what the kernels expect at zero
    GB_CUDA(cudaMemsetAsync(colpos, 0, 4ull * N, st));
    if (nchunks) GB_CUDA(cudaMemsetAsync(tri, 0, 4ull * nchunks * CW * CW, st));
    GB_CUDA(cudaMemsetAsync(work, 0, 20, st));  // both counters and the error word
    NoallocTable tb{};
    tb.job = RedJob{row_ptr, col, val, pcols, colpos, nonpiv, tri, dprime, nullptr, nullptr, work, nA, nC, N, nb, fp};
    tb.tri_start[1] = blocks(nA, 8);
    tb.inv_start[1] = blocks(nchunks, IW);
    tb.red_start[1] = nC;
    NoallocTable *dtb = reinterpret_cast<NoallocTable *>(scr + NA_TABLE);
    const uint32_t nrows = nA + nC;
    k_noalloc_check<<<std::min<uint32_t>(blocks(nrows, 8), 148 * 8), 256, 0, st>>>(N, nA, nrows, nb, row_ptr, col,
                                                                                  pcols, nonpiv, err);
    k_noalloc_setup<<<1, 32, 0, st>>>(tb, dtb, err);
    counted(2);
    if (nA) {
        k_noalloc_mark<<<blocks(nA, 256), 256, 0, st>>>(N, nA, pcols, colpos);
        k_build_chunk_tri<<<tb.tri_start[1], 256, 0, st>>>(&dtb->job, dtb->tri_start, 1);
        k_invert_chunk_tri<<<tb.inv_start[1], IW * 32, 0, st>>>(&dtb->job, dtb->inv_start, 1);
        counted(3);
    }
    const size_t smem = (size_t)N * (mode == A32 ? 4 : 8);
    if (mode == A32) {
        opt_in_smem(reinterpret_cast<const void *>(k_reduce<A32, true>));
        k_reduce<A32, true><<<nC, RT, smem, st>>>(&dtb->job, dtb->red_start, 1);
    } else {
        opt_in_smem(reinterpret_cast<const void *>(k_reduce<M64, true>));
        k_reduce<M64, true><<<nC, RT, smem, st>>>(&dtb->job, dtb->red_start, 1);
    }
    const size_t nout = (size_t)nC * nb;
    k_noalloc_poison<<<(uint32_t)std::min<size_t>((nout + 255) / 256, 148 * 8), 256, 0, st>>>(nout, dprime, err);
    counted(2);  // like every launch group: a refused launch fails this call
}

}  // namespace gb
