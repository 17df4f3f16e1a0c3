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
#include <cstdlib>

#include "internal.hpp"

namespace gb {

namespace {

constexpr int RT = 256;  // threads per block of the row-reduction kernel

inline unsigned blocks(size_t n, unsigned t) { return (unsigned)((n + t - 1) / t); }

// ---- sparse reduction of the non-pivot rows (PSGE trailing update, Sec. 9.2) -------------------
//
// The pivot columns are taken in chunks of CW = 32 consecutive pivots (pivot rows k..k+31, one
// contiguous CSR segment).  For a non-pivot row v the multipliers of a chunk are the solution of a
// 32 x 32 unit upper-triangular system: f_i = v[c_i] - sum_{j<i} f_j U[j][i], where U[j][i] is the
// entry of pivot row j at pivot column c_i.  One warp per row solves it with shuffles from a shared
// copy of U (prefetched by the other warps while the previous chunk's system is solved); then
// every warp of the block applies v <- v - sum_i f_i (pivot row i) to the accumulators with
// shared-memory atomics (each pivot row's own leading entry included, which leaves v[c_i] = 0).
// A block reduces R non-pivot rows together, so each pivot-row entry read from L2 serves R rows,
// and it synchronises twice per chunk instead of once per pivot column.
//
// Accumulators are lazy (Rem. 8.1), in one of three modes:
//   A32: p < 2^16, each product (p - f) v < 2^32 is Barrett-reduced to [0, p) and added to a 32-bit
//        sum (exact while a column takes fewer than 2^16 updates: the host requires nA < 2^16);
//   A64: p < 2^16, the raw products are added to a 64-bit sum (no reduction per update);
//   M64: p < 2^31, the Montgomery product redc(fR * v) in [0, 2p) is added to a 64-bit sum.
// A32 halves the shared memory per row, which lets more blocks share an SM.  Entries are reduced
// (Barrett) when read.
constexpr int CW = 32;
enum AccMode { A32 = 0, A64 = 1, M64 = 2 };
template <int MODE>
struct AccOf { using type = unsigned long long; };
template <>
struct AccOf<A32> { using type = uint32_t; };

// U[chunk][j][i] for j < i: entry of pivot row chunk*32+j at pivot column pcols[chunk*32+i]
__global__ void k_build_chunk_tri(uint32_t nA, const uint32_t *__restrict__ row_ptr,
                                  const uint32_t *__restrict__ col, const uint32_t *__restrict__ val,
                                  const uint32_t *__restrict__ pcols,
                                  const uint32_t *__restrict__ colpos, uint32_t *__restrict__ U) {
    const uint32_t k = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (k >= nA) return;
    const int lane = threadIdx.x & 31;
    const uint32_t chunk = k / CW, j = k % CW;
    const uint32_t last = pcols[min(chunk * CW + CW, nA) - 1];
    uint32_t *Uc = U + (size_t)chunk * CW * CW + (size_t)j * CW;
    const uint32_t a = row_ptr[k] + 1, b = row_ptr[k + 1];
    for (uint32_t q0 = a; q0 < b; q0 += 32) {
        const uint32_t q = q0 + lane;
        bool past = true;
        if (q < b) {
            const uint32_t c = col[q];
            past = c > last;
            if (!past) {
                const uint32_t cp = colpos[c];
                if ((cp & 0x80000000u) && (cp & 0x7FFFFFFFu) / CW == chunk) Uc[(cp & 0x7FFFFFFFu) % CW] = val[q];
            }
        }
        if (__all_sync(0xffffffffu, past)) break;  // columns ascend: the rest lies past the chunk
    }
}

template <int R, int MODE, bool SMEM>
__global__ void __launch_bounds__(RT) k_reduce(uint32_t nA, uint32_t nC, uint32_t N,
                                              const uint32_t *__restrict__ row_ptr,
                                              const uint32_t *__restrict__ col,
                                              const uint32_t *__restrict__ val,
                                              const uint32_t *__restrict__ pcols,
                                              const uint32_t *__restrict__ U,
                                              const uint32_t *__restrict__ nonpiv, uint32_t nb,
                                              Fp fp, typename AccOf<MODE>::type *__restrict__ gacc,
                                              uint32_t *__restrict__ dprime,
                                              unsigned long long *__restrict__ work) {
    using Acc = typename AccOf<MODE>::type;
    constexpr bool SMALLP = MODE != M64;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint32_t fsh[R][CW];
    __shared__ uint32_t Us[2][CW * CW];
    __shared__ uint32_t rp[CW + 1];
    __shared__ uint32_t s_base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t r0 = blockIdx.x * R;
    const int nr = (int)min((uint32_t)R, nC - r0);
    // base column = smallest leading column of the block's rows
    if (threadIdx.x == 0) {
        uint32_t b = N;
        for (int r = 0; r < nr; ++r) {
            const uint32_t a = row_ptr[nA + r0 + r];
            if (a < row_ptr[nA + r0 + r + 1]) b = min(b, col[a]);
        }
        s_base = b;
    }
    __syncthreads();
    const uint32_t base = s_base, width = N - base;
    Acc *acc = SMEM ? reinterpret_cast<Acc *>(smem_raw) : gacc + (size_t)blockIdx.x * R * N;
    for (uint32_t j = threadIdx.x; j < (uint32_t)R * width; j += RT) acc[j] = 0;
    __syncthreads();
    for (int r = 0; r < nr; ++r) {
        const uint32_t a = row_ptr[nA + r0 + r], b = row_ptr[nA + r0 + r + 1];
        for (uint32_t q = a + threadIdx.x; q < b; q += RT) acc[(size_t)r * width + col[q] - base] = val[q];
    }
    // first chunk holding a pivot column >= base
    uint32_t lo = 0, hi = nA;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (pcols[mid] < base) lo = mid + 1; else hi = mid;
    }
    const uint32_t k0 = (lo / CW) * CW;
    if (k0 < nA)
        for (uint32_t t = threadIdx.x; t < CW * CW; t += RT) Us[0][t] = U[(size_t)(k0 / CW) * CW * CW + t];
    unsigned long long applied = 0, fmas = 0;
    for (uint32_t kc = k0, buf = 0; kc < nA; kc += CW, buf ^= 1) {
        const uint32_t cnt = min((uint32_t)CW, nA - kc);
        __syncthreads();  // the previous chunk's updates (and this chunk's U) are visible
        if (warp < nr) {
            // phase A: multipliers of the chunk for row `warp`
            const Acc *a = acc + (size_t)warp * width;
            uint32_t x = 0;
            if ((uint32_t)lane < cnt) {
                const uint32_t c = pcols[kc + lane];
                if (c >= base) x = MODE == A32 ? fp_reduce32((uint32_t)a[c - base], fp) : fp_reduce(a[c - base], fp);
            }
            const uint32_t *Uc = Us[buf];
            for (uint32_t i = 0; i + 1 < cnt; ++i) {
                const uint32_t fi = __shfl_sync(0xffffffffu, x, i);
                if (fi && (uint32_t)lane > i && (uint32_t)lane < cnt) {
                    const uint32_t u = Uc[i * CW + lane];
                    if (u) x = fp_sub(x, SMALLP ? fp_reduce32(fi * u, fp) : fp_mul(fi, u, fp), fp);
                }
            }
            fsh[warp][lane] = (uint32_t)lane < cnt ? x : 0u;
        } else {
            if (warp < R) fsh[warp][lane] = 0u;
            // the other warps prefetch the next chunk's triangle
            const uint32_t kn = kc + CW;
            if (kn < nA)
                for (uint32_t t = threadIdx.x - 32u * (uint32_t)nr; t < CW * CW; t += RT - 32u * (uint32_t)nr)
                    Us[buf ^ 1][t] = U[(size_t)(kn / CW) * CW * CW + t];
        }
        if (threadIdx.x <= cnt) rp[threadIdx.x] = row_ptr[kc + threadIdx.x];
        __syncthreads();
        // phase B: warp w applies pivot rows w, w + 8, ... of the chunk
        for (uint32_t i = warp; i < cnt; i += RT / 32) {
            uint32_t m[R];
            bool any = false;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const uint32_t f = fsh[r][i];
                m[r] = f ? (SMALLP ? fp.p - f : fp_to_mont(fp.p - f, fp)) : 0u;
                any |= f != 0;
            }
            if (!any) continue;
            const uint32_t a = rp[i], b = rp[i + 1];
            if (lane == 0) {
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if (m[r]) { ++applied; fmas += b - a; }
            }
            for (uint32_t q = a + lane; q < b; q += 64) {
                // two entries per lane in flight
                const bool two = q + 32 < b;
                const uint32_t c0 = col[q] - base, v0 = val[q];
                const uint32_t c1 = two ? col[q + 32] - base : 0u, v1 = two ? val[q + 32] : 0u;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (!m[r]) continue;
                    Acc *ar = acc + (size_t)r * width;
                    if (MODE == A32) {
                        atomicAdd(reinterpret_cast<uint32_t *>(ar + c0), fp_reduce32(m[r] * v0, fp));
                        if (two) atomicAdd(reinterpret_cast<uint32_t *>(ar + c1), fp_reduce32(m[r] * v1, fp));
                    } else if (MODE == A64) {
                        atomicAdd(reinterpret_cast<unsigned long long *>(ar + c0), (unsigned long long)(m[r] * v0));
                        if (two) atomicAdd(reinterpret_cast<unsigned long long *>(ar + c1), (unsigned long long)(m[r] * v1));
                    } else {
                        atomicAdd(reinterpret_cast<unsigned long long *>(ar + c0),
                                  (unsigned long long)fp_redc((uint64_t)m[r] * v0, fp));
                        if (two)
                            atomicAdd(reinterpret_cast<unsigned long long *>(ar + c1),
                                      (unsigned long long)fp_redc((uint64_t)m[r] * v1, fp));
                    }
                }
            }
        }
    }
    __syncthreads();
    if (lane == 0 && (applied || fmas)) {
        atomicAdd(&work[0], applied);
        atomicAdd(&work[1], fmas);
    }
    for (int r = 0; r < nr; ++r) {
        uint32_t *out = dprime + (size_t)(r0 + r) * nb;
        const Acc *a = acc + (size_t)r * width;
        for (uint32_t jj = threadIdx.x; jj < nb; jj += RT) {
            const uint32_t c = nonpiv[jj];
            out[jj] = c < base ? 0u : MODE == A32 ? fp_reduce32((uint32_t)a[c - base], fp) : fp_reduce(a[c - base], fp);
        }
    }
}

// ---- RREF(D'): right-looking Gauss-Jordan by panels of K rows --------------------------------
//
// M starts as a copy of D'.  Each round picks up to K non-zero rows that are not pivots yet, brings
// them to reduced echelon form among themselves in one block (pivots at their leading columns),
// then eliminates the new pivot columns from every other row of M in parallel (a GEMM-shaped
// update), which also keeps the earlier pivot rows reduced.  A pivot row's leading column never
// moves: it is zero left of its pivot, and later pivot rows are zero at it.  When no non-zero
// non-pivot row is left, the pivot rows sorted by pivot column are RREF(D'), which is unique.
constexpr uint32_t KP = 32;       // panel rows
constexpr uint32_t NOLEAD = 0xFFFFFFFFu;

struct Rref {
    uint32_t *M;       // nC x nb working matrix
    uint32_t *lead;    // nC: first non-zero column, NOLEAD for a zero row
    uint32_t *pcol;    // nC: pivot column of a pivot row, NOLEAD otherwise
    uint32_t *order;   // rank: pivot rows in discovery order
    uint32_t *state;   // [0] pivots so far, [1] panel rows, [2] new pivots, [3] rows left
    uint32_t *panel;   // KP panel row ids, then KP new pivot row ids, then KP new pivot columns
    uint32_t nC, nb;
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

// leading columns of every row of M
__global__ void k_leads(Rref X) {
    __shared__ uint32_t red[32];
    const uint32_t r = blockIdx.x;
    const uint32_t *row = X.M + (size_t)r * X.nb;
    uint32_t c = NOLEAD;
    for (uint32_t j = threadIdx.x; j < X.nb; j += blockDim.x)
        if (row[j]) { c = j; break; }
    c = block_min(c, red);
    if (threadIdx.x == 0) {
        X.lead[r] = c;
        X.pcol[r] = NOLEAD;
    }
}

// choose the next panel: the first KP non-zero rows that are not pivots (one block)
__global__ void k_pick_panel(Rref X) {
    __shared__ uint32_t wcnt[32];
    __shared__ uint32_t s_taken;
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

// reduced echelon form of the panel rows among themselves (one block).  With SMEM the panel is
// copied to shared memory, reduced there and written back.
constexpr int PT = 1024;
template <bool SMEM>
__global__ void __launch_bounds__(PT) k_panel_rref(Rref X, Fp fp) {
    extern __shared__ __align__(16) uint32_t pan[];
    __shared__ uint32_t mult[KP], prow[KP], pslot[KP], pc[KP], red[32];
    __shared__ uint32_t s_inv;
    const uint32_t P = X.state[1], nb = X.nb;
    auto rowp = [&](uint32_t t) -> uint32_t * {
        return SMEM ? pan + (size_t)t * nb : X.M + (size_t)X.panel[t] * nb;
    };
    if (SMEM) {
        for (uint32_t t = 0; t < P; ++t) {
            const uint32_t *src = X.M + (size_t)X.panel[t] * nb;
            for (uint32_t j = threadIdx.x; j < nb; j += PT) pan[(size_t)t * nb + j] = src[j];
        }
        __syncthreads();
    }
    uint32_t nnew = 0;
    for (uint32_t t = 0; t < P; ++t) {
        const uint32_t r = X.panel[t];
        uint32_t *row = rowp(t);
        // multipliers: entries at the panel's earlier pivots, negated (pivot rows are RREF
        // among themselves, so each multiplier is read from the unreduced row)
        if (threadIdx.x < nnew) {
            const uint32_t v = row[pc[threadIdx.x]];
            mult[threadIdx.x] = v ? fp.p - v : 0u;
        }
        __syncthreads();
        uint32_t c = NOLEAD;
        for (uint32_t j = threadIdx.x; j < nb; j += PT) {
            uint64_t acc = row[j];
            if (fp.small) {  // raw products < 2^32, at most 32 of them: one reduction per entry
                for (uint32_t k = 0; k < nnew; ++k) acc += (uint64_t)(mult[k] * rowp(pslot[k])[j]);
            } else {
                for (uint32_t k = 0; k < nnew; ++k)
                    if (mult[k]) acc += fp_mul(mult[k], rowp(pslot[k])[j], fp);
            }
            const uint32_t x = nnew ? fp_reduce(acc, fp) : (uint32_t)acc;
            if (nnew) row[j] = x;
            if (x && c == NOLEAD) c = j;
        }
        c = block_min(c, red);
        if (c == NOLEAD) {
            if (threadIdx.x == 0) X.lead[r] = NOLEAD;
            continue;
        }
        if (threadIdx.x == 0) s_inv = fp_inv(row[c], fp);
        __syncthreads();
        const uint32_t inv = s_inv;
        for (uint32_t j = c + threadIdx.x; j < nb; j += PT) row[j] = fp_mul(row[j], inv, fp);
        if (threadIdx.x < nnew) {
            const uint32_t v = rowp(pslot[threadIdx.x])[c];
            mult[threadIdx.x] = v ? fp.p - v : 0u;
        }
        __syncthreads();
        // clear column c from the earlier new rows
        for (uint32_t k = 0; k < nnew; ++k) {
            const uint32_t mk = mult[k];
            if (!mk) continue;
            uint32_t *dst = rowp(pslot[k]);
            for (uint32_t j = c + threadIdx.x; j < nb; j += PT) {
                const uint32_t y = row[j];
                if (y) dst[j] = fp_reduce((uint64_t)dst[j] + (uint64_t)mk * y, fp);
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
        for (uint32_t t = 0; t < P; ++t) {
            uint32_t *dst = X.M + (size_t)X.panel[t] * nb;
            for (uint32_t j = threadIdx.x; j < nb; j += PT) dst[j] = pan[(size_t)t * nb + j];
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

// every other row: r <- r - sum_k r[pc_k] * Q_k over the panel's new pivot rows Q_k; one block per
// row, so a row's multipliers are read before any thread writes the row
__global__ void k_eliminate(Rref X, Fp fp) {
    __shared__ uint32_t m[KP], q[KP], red[32];
    __shared__ int s_any;
    const uint32_t r = blockIdx.x, nb = X.nb, nnew = X.state[2];
    if (nnew == 0 || X.lead[r] == NOLEAD) return;
    const uint32_t pr = X.pcol[r];
    uint32_t *row = X.M + (size_t)r * nb;
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
                if (m[k]) acc += (uint64_t)((fp.p - m[k]) * X.M[(size_t)q[k] * nb + j]);
        } else {
            for (uint32_t k = 0; k < nnew; ++k)
                if (m[k]) acc += fp_mul(fp.p - m[k], X.M[(size_t)q[k] * nb + j], fp);
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

// the pivot rows in pivot-column order
__global__ void k_gather_rref(Rref X, uint32_t rank, uint32_t *__restrict__ out,
                              uint32_t *__restrict__ opiv) {
    const uint32_t e = blockIdx.x, nb = X.nb;
    __shared__ uint32_t pos;
    const uint32_t r = X.order[e], c = X.pcol[r];
    if (threadIdx.x == 0) {
        uint32_t n = 0;
        for (uint32_t f = 0; f < rank; ++f) n += X.pcol[X.order[f]] < c;
        pos = n;
        opiv[n] = c;
    }
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < nb; j += blockDim.x)
        out[(size_t)pos * nb + j] = X.M[(size_t)r * nb + j];
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

// nonzeros of row r of M (rows < mrows; rows beyond are empty), plus one for the leading term
__global__ void k_count_rows_plus(const uint32_t *__restrict__ M, uint32_t rows, uint32_t mrows,
                                  uint32_t nb, uint32_t *__restrict__ cnt) {
    const uint32_t r = blockIdx.x;
    uint32_t c = 0;
    if (r < mrows)
        for (uint32_t j = threadIdx.x; j < nb; j += blockDim.x) c += M[(size_t)r * nb + j] != 0;
    for (int d = 16; d; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
    __shared__ uint32_t s[32];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 1;
        for (uint32_t w = 0; w < blockDim.x / 32; ++w) t += s[w];
        cnt[r] = t;
    }
}

// leading term (coefficient 1) then the nonzeros of row r in column order, exponents as n bytes
__global__ void k_pack_rows(const uint32_t *__restrict__ M, uint32_t rows, uint32_t mrows, uint32_t nb,
                            const uint32_t *__restrict__ nonpiv, const uint4 *__restrict__ dict,
                            const uint4 *__restrict__ lead, const uint32_t *__restrict__ out_off,
                            uint32_t n, uint8_t *__restrict__ oexp, uint32_t *__restrict__ ocf) {
    const uint32_t r = blockIdx.x;
    __shared__ uint32_t base;
    __shared__ uint32_t wsum[32];
    auto put = [&](uint32_t pos, uint4 m, uint32_t c) {
        const uint32_t w[4] = {m.x, m.y, m.z, m.w};
        for (uint32_t i = 0; i < n; ++i) oexp[(size_t)pos * n + i] = (uint8_t)(w[i >> 2] >> (8 * (i & 3)));
        ocf[pos] = c;
    };
    if (threadIdx.x == 0) {
        base = out_off[r];
        put(base, lead[r], 1u);
        base += 1;
    }
    __syncthreads();
    if (r >= mrows) return;
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
        if (v) put(base + before + __popc(mask & ((1u << lane) - 1u)), dict[nonpiv[j]], v);
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
        const bool small = S->fp.small != 0;
        const uint32_t nchunks = (nA + CW - 1) / CW;
        DBuf<uint32_t> U;
        U.alloc(ar, (size_t)std::max(nchunks, 1u) * CW * CW, st);
        GB_CUDA(cudaMemsetAsync(U.p, 0, 4ull * std::max(nchunks, 1u) * CW * CW, st));
        if (nA) {
            k_build_chunk_tri<<<blocks(nA, 8), 256, 0, st>>>(nA, Mac->row_ptr.p, Mac->col.p, Mac->val.p,
                                                            Mac->pcols.p, Mac->colpos.p, U.p);
            counted();
        }
        // accumulator mode and rows per block: the largest R whose blocks all fit in one wave
        const int mode = !small ? M64 : (nA < 65536u ? A32 : A64);
        const size_t accb = mode == A32 ? 4 : 8;
        // rows per block.  Measured on the n=10 dense workload, one row per block (more resident
        // warps) beats sharing each streamed pivot row between 2 or 4 rows; GB_REDUCE_R=2|4
        // selects the shared variants for tuning.
        static const int forced_r = [] {
            const char *e = std::getenv("GB_REDUCE_R");
            return e ? std::atoi(e) : 0;
        }();
        int R = (forced_r == 2 || forced_r == 4) ? forced_r : 1;
        if ((size_t)R * N * accb > 200 * 1024) R = 1;
        const bool use_smem = (size_t)R * N * accb <= 200 * 1024;
        const unsigned grid = (nC + R - 1) / R;
        const size_t smem = use_smem ? (size_t)R * N * accb : 0;
        DBuf<unsigned long long> gacc;
        if (!use_smem) gacc.alloc(ar, (size_t)grid * R * N + 1, st);
        auto launch = [&](auto kern, auto *gp) {
            // static + dynamic shared memory above 48 KB needs the opt-in, whatever the split
            GB_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            kern<<<grid, RT, smem, st>>>(nA, nC, N, Mac->row_ptr.p, Mac->col.p, Mac->val.p, Mac->pcols.p,
                                         U.p, Mac->nonpiv.p, nb, S->fp, gp, E->dprime.p, work.p);
            counted();
        };
        uint32_t *g32 = reinterpret_cast<uint32_t *>(gacc.p);
        unsigned long long *g64 = gacc.p;
#define GB_REDUCE_CASE(RR)                                                                   \
    if (R == RR) {                                                                           \
        if (mode == A32) {                                                                   \
            if (use_smem) launch(k_reduce<RR, A32, true>, g32);                              \
            else launch(k_reduce<RR, A32, false>, g32);                                      \
        } else if (mode == A64) {                                                            \
            if (use_smem) launch(k_reduce<RR, A64, true>, g64);                              \
            else launch(k_reduce<RR, A64, false>, g64);                                      \
        } else {                                                                             \
            if (use_smem) launch(k_reduce<RR, M64, true>, g64);                              \
            else launch(k_reduce<RR, M64, false>, g64);                                      \
        }                                                                                    \
    }
        GB_REDUCE_CASE(1)
        GB_REDUCE_CASE(2)
        GB_REDUCE_CASE(4)
#undef GB_REDUCE_CASE
    }
    GB_CUDA(cudaEventRecord(S->ev[3], st));
    if (echelon && nC && nb) {
        DBuf<uint32_t> Mw, lead, pcol, order, state, panel;
        Mw.alloc(ar, (size_t)nC * nb, st);
        lead.alloc(ar, nC, st);
        pcol.alloc(ar, nC, st);
        order.alloc(ar, std::min(nC, nb), st);
        state.alloc(ar, 4, st);
        panel.alloc(ar, 3 * KP, st);
        GB_CUDA(cudaMemcpyAsync(Mw.p, E->dprime.p, 4ull * nC * nb, cudaMemcpyDeviceToDevice, st));
        GB_CUDA(cudaMemsetAsync(state.p, 0, 16, st));
        Rref X{Mw.p, lead.p, pcol.p, order.p, state.p, panel.p, nC, nb};
        k_leads<<<nC, 256, 0, st>>>(X);
        counted();
        uint32_t *h = static_cast<uint32_t *>(pinned(S, 64));
        const size_t pan_bytes = 4ull * KP * nb;
        const bool pan_smem = pan_bytes <= 200 * 1024;
        if (pan_smem)
            GB_CUDA(cudaFuncSetAttribute(k_panel_rref<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)pan_bytes));
        // rounds are launched in groups; a group's rounds after the last pivot do nothing
        // every round turns each of its rows into a pivot row or a zero row
        const uint32_t maxrounds = (nC + KP - 1) / KP + 1;
        uint32_t rounds = 0;
        for (;;) {
            const uint32_t group = rounds == 0 ? 2 : 4;
            for (uint32_t g = 0; g < group; ++g) {
                k_pick_panel<<<1, 1024, 0, st>>>(X);
                if (pan_smem) k_panel_rref<true><<<1, PT, pan_bytes, st>>>(X, S->fp);
                else k_panel_rref<false><<<1, PT, 0, st>>>(X, S->fp);
                k_eliminate<<<nC, 256, 0, st>>>(X, S->fp);
                counted(3);
            }
            rounds += group;
            GB_CUDA(cudaMemcpyAsync(h, state.p, 16, cudaMemcpyDeviceToHost, st));
            sync(S);
            if (h[1] == 0 || h[3] <= h[1] || rounds >= maxrounds) break;
        }
        // one more pick confirms that no non-zero non-pivot row is left
        k_pick_panel<<<1, 1024, 0, st>>>(X);
        counted();
        GB_CUDA(cudaMemcpyAsync(h, state.p, 16, cudaMemcpyDeviceToHost, st));
        GB_CUDA(cudaMemcpyAsync(h + 4, work.p, 16, cudaMemcpyDeviceToHost, st));
        sync(S);
        if (h[1] != 0) fail(GB_EDEVICE, "RREF: rows left after the last round");
        E->rank = h[0];
        std::memcpy(E->work, h + 4, 16);
        E->rref.alloc(ar, (size_t)E->rank * nb, st);
        E->rpiv.alloc(ar, E->rank, st);
        if (E->rank) {
            k_gather_rref<<<E->rank, 256, 0, st>>>(X, E->rank, E->rref.p, E->rpiv.p);
            counted();
        }
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
    // element elems[i] becomes LM(elems[i]) + (row i of D'), compacted on the device
    Arena &ar = S->ctx->arena;
    cudaStream_t st = S->stream;
    const uint32_t rows = (uint32_t)elems.size(), nb = E->nb, n = S->n;
    gb_macaulay *Mac = E->mac;
    off.assign(1, 0);
    exps.clear();
    cf.clear();
    if (!rows) return;
    DBuf<uint32_t> cnt, doff;
    DBuf<uint4> lead;
    cnt.alloc(ar, rows, st);
    doff.alloc(ar, (size_t)rows + 1, st);
    lead.alloc(ar, rows, st);
    std::vector<uint4> hl(rows);
    for (uint32_t i = 0; i < rows; ++i) hl[i] = to_u4(S->lm[elems[i]]);
    char *h = static_cast<char *>(pinned(S, 20ull * rows + 64));
    std::memcpy(h, hl.data(), 16ull * rows);
    GB_CUDA(cudaMemcpyAsync(lead.p, h, 16ull * rows, cudaMemcpyHostToDevice, st));
    k_count_rows_plus<<<rows, 256, 0, st>>>(E->dprime.p, rows, E->nC, nb, cnt.p);
    counted();
    exclusive_scan(ar, cnt.p, doff.p, rows, st);
    uint32_t *ho = reinterpret_cast<uint32_t *>(h + 16ull * rows);
    GB_CUDA(cudaMemcpyAsync(ho, doff.p, 4ull * (rows + 1), cudaMemcpyDeviceToHost, st));
    sync(S);
    off.assign(ho, ho + rows + 1);
    const uint64_t T = off[rows];
    DBuf<uint8_t> dex;
    DBuf<uint32_t> dcf;
    dex.alloc(ar, T * n, st);
    dcf.alloc(ar, T, st);
    k_pack_rows<<<rows, 256, 0, st>>>(E->dprime.p, rows, E->nC, nb, Mac->nonpiv.p, Mac->dict.p, lead.p,
                                      doff.p, n, dex.p, dcf.p);
    counted();
    exps.resize(T * n);
    cf.resize(T);
    GB_CUDA(cudaMemcpyAsync(exps.data(), dex.p, T * n, cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaMemcpyAsync(cf.data(), dcf.p, 4 * T, cudaMemcpyDeviceToHost, st));
    sync(S);
}

// ---- the sparse reduction without device allocation --------------------------------------------
//
// Scratch of gb_reduce_rows_noalloc: pivot-column flags (one word per dictionary column), the
// 32 x 32 chunk triangles (one per 32 pivot rows) and the two work counters of k_reduce, carved
// out of one fixed array that is part of the library image.  Host code reaches it only through
// the address cudaGetSymbolAddress returns for the current device.
constexpr uint32_t NA_COLPOS = 0;
constexpr uint32_t NA_TRI = GB_NOALLOC_MAX_DICT;
constexpr uint32_t NA_WORK = NA_TRI + GB_NOALLOC_MAX_PIVOTS * CW;  // even: 8-byte aligned
constexpr uint32_t NA_WORDS = NA_WORK + 4;
static __device__ __align__(256) uint32_t g_noalloc_scratch[NA_WORDS];

namespace {
__global__ void k_mark_pivot_cols(uint32_t nA, const uint32_t *__restrict__ pcols,
                                  uint32_t *__restrict__ colpos) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nA) colpos[pcols[k]] = k | 0x80000000u;
}

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
    if (!nC || !nb) return;
    if (!row_ptr || !col || !val || (nA && !pcols) || !nonpiv || !dprime)
        fail(GB_EINVAL, "gb_reduce_rows_noalloc: null device pointer");
    uint32_t *scr = noalloc_scratch_for_current_device();
    uint32_t *colpos = scr + NA_COLPOS, *tri = scr + NA_TRI;
    unsigned long long *work = reinterpret_cast<unsigned long long *>(scr + NA_WORK);
    const uint32_t nchunks = (nA + CW - 1) / CW;
    // the array keeps the previous call's contents: clear what the kernels expect at zero
    GB_CUDA(cudaMemsetAsync(colpos, 0, 4ull * N, st));
    if (nchunks) GB_CUDA(cudaMemsetAsync(tri, 0, 4ull * nchunks * CW * CW, st));
    GB_CUDA(cudaMemsetAsync(work, 0, 16, st));
    if (nA) {
        k_mark_pivot_cols<<<blocks(nA, 256), 256, 0, st>>>(nA, pcols, colpos);
        counted();
        k_build_chunk_tri<<<blocks(nA, 8), 256, 0, st>>>(nA, row_ptr, col, val, pcols, colpos, tri);
        counted();
    }
    const size_t smem = (size_t)N * (mode == A32 ? 4 : 8);
    if (mode == A32) {
        GB_CUDA(cudaFuncSetAttribute(k_reduce<1, A32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_reduce<1, A32, true><<<nC, RT, smem, st>>>(nA, nC, N, row_ptr, col, val, pcols, tri, nonpiv, nb, fp,
                                                     nullptr, dprime, work);
    } else {
        GB_CUDA(cudaFuncSetAttribute(k_reduce<1, M64, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_reduce<1, M64, true><<<nC, RT, smem, st>>>(nA, nC, N, row_ptr, col, val, pcols, tri, nonpiv, nb, fp,
                                                     nullptr, dprime, work);
    }
    counted();
}

}  // namespace gb
