// sp.cu -- symbolic preprocessing SP : batch -> (T, R, Pi) (Def. 5.2) as the two-pass FBSP
// pipeline (the algorithm of Sec. 10), with the one-step reduction closure of Rem. 3.3 run as
// bulk frontier rounds (Sec. 7.2), for many independent jobs (systems) at once.
//
// Keys.  Every monomial of a job has degree <= D (its step degree), so its dense grevlex rank
// (device.cuh) lies in [0, C(n + D, n)).  Ordering of T (Sec. 5.1) is a counting sort: a bitmap
// over the rank space (L2-resident) is marked with atomicOr, and the dictionary column of a rank
// is the number of marked ranks above it (word popcounts + one exclusive scan).
//
// Setification (Sec. 5.1) and the column of every term (the join of Sec. 7.5) go through a hash
// dictionary keyed by the additive monomial key of device.cuh: a basis term carries key(m), a row
// key(t), so a term's key is one 64-bit add, and a slot holds the key, the monomial and (once
// known) its column.  The insert that claims a slot is the "new monomial" test of the closure
// frontier; the dense rank is then computed only for the N distinct monomials, not for every
// term.  Every lookup of the fill compares the stored monomial with the term's; a mismatch (two
// monomials sharing a key) sends the job back through the rank path, in which every term's rank
// marks the bitmap directly and the column is read from its popcount prefix.
//
// Passes (each one launch for all jobs; a job's blocks are found through a prefix table):
//   1. mark the leading monomials of the given rows (they start in Done: no reducer rows for them)
//   2. expand the given rows: every term t*m is marked; unmarked ones join the frontier queue
//   3. closure rounds: for each frontier monomial, the oldest non-redundant g with LM(g) | m gives
//      the reducer row (m / LM(g), g), whose tail is expanded into the next frontier; one
//      read-back of every job's counters per round
//   4. dictionary: popcount scan, columns, dictionary monomials scattered to their columns
//   5. row order: pivot rows by leading column (a scan over the pivot-column flags), then the
//      non-pivot given rows in the order the host fixed
//   6. CSR: count (row lengths) -> exclusive scan (row_ptr) -> fill (col_ind, val); every row
//      writes its own segment [row_ptr[i], row_ptr[i+1]) (the race-freedom theorem of Sec. 11)
// Scans run once over the concatenation of all jobs' arrays; a job reads its prefixes relative
// to the first entry of its own range.
#include <algorithm>
#include <cstddef>
#include <cstdlib>

#include "internal.hpp"

namespace gb {

namespace {

constexpr uint32_t FLAG_PIVOT = 1u, FLAG_REDUCER = 2u, FLAG_TAIL = 4u;
constexpr int WPB = 8;  // warps per block in the warp-per-row kernels

struct Counters {  // device-side counters of one job, read back after each round
    uint32_t q;    // frontier monomials pushed (all rounds)
    uint32_t red;  // reducer rows
    unsigned long long red_nnz;
    uint32_t err;
    uint32_t pad;
};

// one slot of the hash dictionary: 32 bytes, so that a lookup touches one L2 sector
struct alignas(32) HSlot {
    unsigned long long tag;  // 0: empty, else key + 1 (0 mapped to 1)
    uint32_t col;            // dictionary column, once the dictionary is ordered
    uint32_t pad;
    uint4 mon;               // the monomial, written by the thread that claimed the slot
};
static_assert(sizeof(HSlot) == 32 && offsetof(HSlot, col) == 8 && offsetof(HSlot, mon) == 16,
              "the fill reads a slot as two 16-byte words: key, column, pad | monomial");

struct Job {
    // basis of the job's system
    const uint4 *bmon;
    const unsigned long long *bkey;
    const uint32_t *bcf, *boff, *blen;
    // given rows
    const uint4 *gt;
    const uint32_t *gk, *gnp;
    const uint8_t *gf;
    uint32_t ng;
    // keys
    uint32_t *bits;
    const uint32_t *tab;
    int n, sh, tabsz;  // table rows of 2^sh entries
    int deglex;        // the rank table and mono_rank in deglex, else grevlex
    uint32_t W;
    // closure
    const uint32_t *nr_idx;
    const uint4 *nr_lm;
    uint32_t nnr;
    uint4 *qmon;
    uint32_t *qrank;
    uint32_t cap;
    uint4 *red_t;
    uint32_t *red_k, *red_rank, *lm_rank;
    Counters *cnt;
    // hash dictionary (null htab: the rank path)
    HSlot *htab;
    uint32_t hmask, hshift;    // slots - 1, 64 - log2(slots)
    unsigned long long keymask;  // all ones; fewer bits (GB_SP_KEY_MASK) force shared keys in tests
    uint32_t *qslot, *red_slot, *lm_slot;
    // dictionary, rows and CSR (filled in once the counts are known)
    uint32_t N, nA, nrows, nq, nred, nnz;
    uint32_t *wcnt;        // this job's range of the concatenated word counts
    const uint32_t *wpre;  // its range of their exclusive scan (subtract wpre[0])
    uint32_t *is_piv, *src;
    const uint32_t *pidx;  // range of the scan of is_piv (subtract pidx[0])
    uint4 *dict, *row_t;
    uint32_t *row_k, *pcols, *nonpiv, *colpos;
    uint8_t *row_flags;
    uint32_t *lens;
    const uint32_t *lscan;  // range of the scan of lens (subtract lscan[0])
    uint32_t *row_ptr, *col, *val;
};

__device__ __forceinline__ void load_tab(uint32_t *sm, const Job &J) {
    for (int i = threadIdx.x; i < J.tabsz; i += blockDim.x) sm[i] = J.tab[i];
    __syncthreads();
}

__device__ __forceinline__ uint32_t col_of(const Job &J, uint32_t r) {
    const uint32_t w = r >> 5, below = J.bits[w] & ((1u << (r & 31)) - 1u);
    return J.N - 1u - (J.wpre[w] - J.wpre[0] + __popc(below));
}

// mark rank r; true if this call flipped the bit (the monomial is new)
__device__ __forceinline__ bool test_and_set(uint32_t *bits, uint32_t r) {
    const uint32_t w = r >> 5, b = 1u << (r & 31);
    if (bits[w] & b) return false;  // bits only ever get set during a step: a set bit is final
    return !(atomicOr(&bits[w], b) & b);
}

// warp-aggregated append of the lanes' new monomials to the job's frontier queue
__device__ __forceinline__ void push_new(bool isnew, uint4 m, uint32_t r, const Job &J) {
    const unsigned mask = __ballot_sync(0xffffffffu, isnew);
    if (!mask) return;
    const int lane = threadIdx.x & 31, leader = __ffs(mask) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(&J.cnt->q, (uint32_t)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (isnew) {
        const uint32_t pos = base + __popc(mask & ((1u << lane) - 1u));
        if (pos < J.cap) {
            J.qmon[pos] = m;
            J.qrank[pos] = r;
        }
    }
}

constexpr uint32_t ERR_TABLE_FULL = 64u, ERR_KEY_CLASH = 128u;

__device__ __forceinline__ unsigned long long tag_of(unsigned long long key, const Job &J) {
    const unsigned long long t = (key & J.keymask) + 1ull;
    return t ? t : 1ull;
}

__device__ __forceinline__ uint32_t home_slot(unsigned long long tag, const Job &J) {
    return (uint32_t)((tag * 0x9E3779B97F4A7C15ull) >> J.hshift);
}

// claim or find the slot of `tag` (linear probing from slot s, whose tag was read as `cur`; at
// most every slot once).  isnew: this call claimed an empty slot.  A full table sets
// ERR_TABLE_FULL and returns 0xFFFFFFFF.
__device__ __forceinline__ uint32_t h_insert_from(unsigned long long tag, uint32_t s, unsigned long long cur,
                                                  const Job &J, bool &isnew) {
    isnew = false;
    for (uint32_t probe = 0; probe <= J.hmask; ++probe) {
        if (probe) cur = J.htab[s].tag;  // a slot only ever goes from 0 to its final tag
        if (cur == tag) return s;
        if (cur == 0ull) {
            cur = atomicCAS(&J.htab[s].tag, 0ull, tag);
            if (cur == 0ull) {
                isnew = true;
                return s;
            }
            if (cur == tag) return s;
        }
        s = (s + 1u) & J.hmask;
    }
    atomicOr(&J.cnt->err, ERR_TABLE_FULL);
    return 0xFFFFFFFFu;
}

// the slot of a tag inserted by an earlier kernel, or 0xFFFFFFFF
__device__ __forceinline__ uint32_t h_insert(unsigned long long tag, const Job &J, bool &isnew) {
    const uint32_t s = home_slot(tag, J);
    return h_insert_from(tag, s, J.htab[s].tag, J, isnew);
}

__device__ __forceinline__ uint32_t h_find(unsigned long long tag, const Job &J) {
    uint32_t s = home_slot(tag, J);
    for (uint32_t probe = 0; probe <= J.hmask; ++probe) {
        const unsigned long long cur = J.htab[s].tag;
        if (cur == tag) return s;
        if (cur == 0ull) return 0xFFFFFFFFu;
        s = (s + 1u) & J.hmask;
    }
    return 0xFFFFFFFFu;
}

// warp-aggregated append of new monomials and their slots to the job's frontier queue
__device__ __forceinline__ void push_new_slot(bool isnew, uint4 m, uint32_t slot, const Job &J) {
    const unsigned mask = __ballot_sync(0xffffffffu, isnew);
    if (!mask) return;
    const int lane = threadIdx.x & 31, leader = __ffs(mask) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(&J.cnt->q, (uint32_t)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (isnew) {
        const uint32_t pos = base + __popc(mask & ((1u << lane) - 1u));
        if (pos < J.cap) {
            J.qmon[pos] = m;
            J.qslot[pos] = slot;
        }
    }
}

// hash path of expand_terms: a term's key is key(t) + key(m_j); only a term that claims a slot
// loads its monomial (for the slot and the frontier queue).  Four terms per lane in flight.
__device__ __forceinline__ void expand_terms_hash(uint4 t, unsigned long long kt, uint32_t off, uint32_t j0,
                                                  uint32_t len, const Job &J) {
    const int lane = threadIdx.x & 31;
    for (uint32_t jb = j0; jb < len; jb += 4 * 32) {
        // the four terms' home slots are read together (independent loads); a term whose home
        // slot already holds its key -- the common case -- is done
        unsigned long long tg[4], cur[4];
        uint32_t hs[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t j = jb + 32u * u + lane;
            tg[u] = j < len ? tag_of(kt + J.bkey[off + j], J) : 0ull;
            hs[u] = home_slot(tg[u], J);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) cur[u] = tg[u] ? J.htab[hs[u]].tag : 0ull;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t j = jb + 32u * u + lane;
            bool isnew = false;
            uint32_t s = 0;
            uint4 m = make_uint4(0, 0, 0, 0);
            if (tg[u] && cur[u] != tg[u]) {
                s = h_insert_from(tg[u], hs[u], cur[u], J, isnew);
                if (isnew) {
                    m = mono_mul(t, J.bmon[off + j]);
                    J.htab[s].mon = m;
                }
            }
            push_new_slot(isnew, m, s, J);
        }
    }
}

// expand terms [j0, len) of t*g into the bitmap / queue; called by a whole warp
__device__ __forceinline__ void expand_terms(uint4 t, uint32_t off, uint32_t j0, uint32_t len,
                                             const Job &J, const uint32_t *tab) {
    const int lane = threadIdx.x & 31;
    for (uint32_t jb = j0; jb < len; jb += 32) {
        const uint32_t j = jb + lane;
        bool isnew = false;
        uint4 m = make_uint4(0, 0, 0, 0);
        uint32_t r = 0;
        if (j < len) {
            m = mono_mul(t, J.bmon[off + j]);
            r = mono_rank(m, tab, J.n, J.sh, J.deglex != 0);
            isnew = test_and_set(J.bits, r);
        }
        push_new(isnew, m, r, J);
    }
}

// Pass 1: leading monomials of the given rows (tail rows have none); 256 rows per block.
// HASH: the hash-dictionary path (every job of a launch takes the same path)
template <bool HASH>
__global__ void k_mark_given(const Job *__restrict__ jobs, const uint32_t *__restrict__ bstart, int nj) {
    extern __shared__ uint32_t tab[];
    const int jb = job_of_block(bstart, nj);
    const Job &J = jobs[jb];
    load_tab(tab, J);
    const uint32_t i = (blockIdx.x - bstart[jb]) * blockDim.x + threadIdx.x;
    if (i >= J.ng) return;
    if (J.gf[i] & FLAG_TAIL) {
        J.lm_rank[i] = 0xFFFFFFFFu;
        return;
    }
    const uint4 m = mono_mul(J.gt[i], J.bmon[J.boff[J.gk[i]]]);
    const uint32_t r = mono_rank(m, tab, J.n, J.sh, J.deglex != 0);
    atomicOr(&J.bits[r >> 5], 1u << (r & 31));
    J.lm_rank[i] = r;
    if constexpr (HASH) {  // the leading monomials start in the dictionary (Done): never frontier items
        bool isnew = false;
        const uint32_t s = h_insert(tag_of(mono_key(J.gt[i]) + J.bkey[J.boff[J.gk[i]]], J), J, isnew);
        if (isnew) J.htab[s].mon = m;
        J.lm_slot[i] = s;
    }
}

// Pass 2: expand the given rows (warp per row)
template <bool HASH>
__global__ void k_expand_given(const Job *__restrict__ jobs, const uint32_t *__restrict__ bstart, int nj) {
    extern __shared__ uint32_t tab[];
    const int jb = job_of_block(bstart, nj);
    const Job &J = jobs[jb];
    if constexpr (!HASH) load_tab(tab, J);  // the hash path ranks nothing here (no table in shared memory)
    const uint32_t row = (blockIdx.x - bstart[jb]) * WPB + (threadIdx.x >> 5);
    if (row >= J.ng) return;  // whole warp leaves together
    const uint32_t k = J.gk[row];
    const uint32_t j0 = (J.gf[row] & FLAG_TAIL) ? 1u : 0u;
    if constexpr (HASH) expand_terms_hash(J.gt[row], mono_key(J.gt[row]), J.boff[k], j0, J.blen[k], J);
    else expand_terms(J.gt[row], J.boff[k], j0, J.blen[k], J, tab);
}

// Pass 3: one closure round over each job's frontier items [range[2j], range[2j+1]) (warp per item)
template <bool HASH>
__global__ void k_closure(const Job *__restrict__ jobs, const uint32_t *__restrict__ bstart, int nj,
                          const uint32_t *__restrict__ range) {
    extern __shared__ uint32_t tab[];
    const int jb = job_of_block(bstart, nj);
    const Job &J = jobs[jb];
    if constexpr (!HASH) load_tab(tab, J);  // the hash path ranks nothing here (no table in shared memory)
    const uint32_t item = range[2 * jb] + (blockIdx.x - bstart[jb]) * WPB + (threadIdx.x >> 5);
    if (item >= range[2 * jb + 1]) return;
    const int lane = threadIdx.x & 31;
    const uint4 m = J.qmon[item];
    // oldest non-redundant element whose leading monomial divides m (nr_idx ascending)
    int g = -1;
    uint4 lmg = make_uint4(0, 0, 0, 0);
    for (uint32_t cb = 0; cb < J.nnr; cb += 32) {
        const uint32_t idx = cb + lane;
        const bool ok = idx < J.nnr && mono_divides(J.nr_lm[idx], m);
        const unsigned mask = __ballot_sync(0xffffffffu, ok);
        if (mask) {
            const uint32_t hit = cb + __ffs(mask) - 1;
            g = (int)J.nr_idx[hit];
            lmg = J.nr_lm[hit];
            break;
        }
    }
    if (g < 0) return;
    const uint4 t = mono_div(m, lmg);
    const uint32_t len = J.blen[g];
    if (lane == 0) {
        const uint32_t pos = atomicAdd(&J.cnt->red, 1u);
        if (pos < J.cap) {
            J.red_t[pos] = t;
            J.red_k[pos] = (uint32_t)g;
            if constexpr (HASH) J.red_slot[pos] = J.qslot[item];
            else J.red_rank[pos] = J.qrank[item];
        }
        atomicAdd(&J.cnt->red_nnz, (unsigned long long)len);
    }
    if constexpr (HASH) expand_terms_hash(t, mono_key(t), J.boff[g], 1u, len, J);
    else expand_terms(t, J.boff[g], 1u, len, J, tab);
}

// hash path, dictionary: the dense rank of every frontier monomial marks the bitmap (the given
// rows' leading monomials were marked with their ranks in pass 1)
__global__ void k_rank_queue(const Job *__restrict__ jobs, const uint32_t *__restrict__ bstart, int nj) {
    extern __shared__ uint32_t tab[];
    const int jb = job_of_block(bstart, nj);
    const Job &J = jobs[jb];
    if (!J.htab) return;  // the whole block: rank-path jobs marked their bits while expanding
    load_tab(tab, J);
    const uint32_t i = (blockIdx.x - bstart[jb]) * blockDim.x + threadIdx.x;
    if (i >= J.nq) return;
    const uint32_t r = mono_rank(J.qmon[i], tab, J.n, J.sh, J.deglex != 0);
    J.qrank[i] = r;
    atomicOr(&J.bits[r >> 5], 1u << (r & 31));
}

// thread-per-item kernels: 256 items per block, block -> (job, local index i)
#define GB_JOB_ITEM(limit)                                                   \
    const int jb = job_of_block(bstart, nj);                                \
    const Job &J = jobs[jb];                                                \
    const uint32_t i = (blockIdx.x - bstart[jb]) * blockDim.x + threadIdx.x; \
    if (i >= (limit)) return;

__global__ void k_popc(const Job *__restrict__ jobs, const uint32_t *__restrict__ bstart, int nj) {
    GB_JOB_ITEM(J.W)
    J.wcnt[i] = __popc(J.bits[i]);
}

// Pass 4: dictionary monomials to their columns (queue entries, then the given rows' LMs)
__global__ void k_dict_queue(const Job *__restrict__ jobs, const uint32_t *__restrict__ bstart, int nj) {
    GB_JOB_ITEM(J.nq)
    const uint32_t c = col_of(J, J.qrank[i]);
    if (c >= J.N) { atomicOr(&J.cnt->err, 1u); return; }
    J.dict[c] = J.qmon[i];
    if (J.htab) J.htab[J.qslot[i]].col = c;
}

__global__ void k_dict_given(const Job *__restrict__ jobs, const uint32_t *__restrict__ bstart, int nj) {
    GB_JOB_ITEM(J.ng)
    if (!(J.gf[i] & FLAG_PIVOT)) return;
    const uint32_t c = col_of(J, J.lm_rank[i]);
    if (c >= J.N) { atomicOr(&J.cnt->err, 2u); return; }
    J.dict[c] = mono_mul(J.gt[i], J.bmon[J.boff[J.gk[i]]]);
    J.is_piv[c] = 1u;
    J.src[c] = 0x80000000u | i;
    if (J.htab) J.htab[J.lm_slot[i]].col = c;
}

__global__ void k_piv_reducers(const Job *__restrict__ jobs, const uint32_t *__restrict__ bstart, int nj) {
    GB_JOB_ITEM(J.nred)
    const uint32_t c = J.htab ? J.htab[J.red_slot[i]].col : col_of(J, J.red_rank[i]);
    if (c >= J.N) { atomicOr(&J.cnt->err, 4u); return; }
    J.is_piv[c] = 1u;
    J.src[c] = i;
}

// Pass 5a: pivot rows by leading column, and the column maps
__global__ void k_place_pivots(const Job *__restrict__ jobs, const uint32_t *__restrict__ bstart, int nj) {
    GB_JOB_ITEM(J.N)
    const uint32_t c = i;
    const uint32_t pc = J.pidx[c] - J.pidx[0];
    if (J.is_piv[c]) {
        const uint32_t r = pc, s = J.src[c];
        if (r >= J.nA) { atomicOr(&J.cnt->err, 8u); return; }
        if (s & 0x80000000u) {
            const uint32_t g = s & 0x7FFFFFFFu;
            J.row_t[r] = J.gt[g];
            J.row_k[r] = J.gk[g];
            J.row_flags[r] = (uint8_t)(J.gf[g] & (FLAG_PIVOT | FLAG_TAIL));
        } else {
            J.row_t[r] = J.red_t[s];
            J.row_k[r] = J.red_k[s];
            J.row_flags[r] = (uint8_t)(FLAG_PIVOT | FLAG_REDUCER);
        }
        J.pcols[r] = c;
        J.colpos[c] = r | 0x80000000u;
    } else {
        const uint32_t q = c - pc;
        if (q >= J.N - J.nA) { atomicOr(&J.cnt->err, 16u); return; }
        J.nonpiv[q] = c;
        J.colpos[c] = q;
    }
}

// Pass 5b: non-pivot given rows after the nA pivot rows, in the host's order
__global__ void k_place_nonpivots(const Job *__restrict__ jobs, const uint32_t *__restrict__ bstart, int nj) {
    GB_JOB_ITEM(J.ng)
    if (J.gnp[i] == 0xFFFFFFFFu) return;
    const uint32_t r = J.nA + J.gnp[i];
    J.row_t[r] = J.gt[i];
    J.row_k[r] = J.gk[i];
    J.row_flags[r] = (uint8_t)(J.gf[i] & FLAG_TAIL);
}

// Pass 6: count, then the job's own row_ptr from the concatenated scan
__global__ void k_row_len(const Job *__restrict__ jobs, const uint32_t *__restrict__ bstart, int nj) {
    GB_JOB_ITEM(J.nrows)
    J.lens[i] = J.blen[J.row_k[i]] - ((J.row_flags[i] & FLAG_TAIL) ? 1u : 0u);
}

__global__ void k_row_ptr(const Job *__restrict__ jobs, const uint32_t *__restrict__ bstart, int nj) {
    GB_JOB_ITEM(J.nrows + 1)
    J.row_ptr[i] = J.lscan[i] - J.lscan[0];
}

// Pass 6: fill (warp per row)
template <bool HASH>
__global__ void k_fill(const Job *__restrict__ jobs, const uint32_t *__restrict__ bstart, int nj) {
    extern __shared__ uint32_t tab[];
    const int jb = job_of_block(bstart, nj);
    const Job &J = jobs[jb];
    if constexpr (!HASH) load_tab(tab, J);  // the hash path ranks nothing here (no table in shared memory)
    const uint32_t row = (blockIdx.x - bstart[jb]) * WPB + (threadIdx.x >> 5);
    if (row >= J.nrows) return;
    const int lane = threadIdx.x & 31;
    const uint32_t k = J.row_k[row];
    const uint32_t skip = (J.row_flags[row] & FLAG_TAIL) ? 1u : 0u;
    const uint32_t off = J.boff[k] + skip, len = J.blen[k] - skip, s = J.row_ptr[row];
    const uint4 t = J.row_t[row];
    if (s + len > J.nnz) {
        if (lane == 0) atomicOr(&J.cnt->err, 32u);
        return;
    }
    if constexpr (HASH) {
        // hash path: key, slot, and a comparison of the slot's monomial with the term's.  Every
        // load of a lane's two terms is issued before any is used: their keys, monomials and
        // coefficients, then each home slot's 32 bytes (key, column, monomial) in two 16-byte
        // reads; a key or monomial mismatch takes the probing path.  Two terms per lane keep the
        // kernel near 64 registers, so that eight warps per block and four blocks per SM fit.
        constexpr int FH = 2;
        const unsigned long long kt = mono_key(t);
        bool clash = false;
        for (uint32_t j0 = lane; j0 < len; j0 += FH * 32) {
            unsigned long long tg[FH];
            uint32_t v[FH], hs[FH];
            uint4 m[FH], s0[FH], s1[FH];
#pragma unroll
            for (int u = 0; u < FH; ++u) {
                const uint32_t j = j0 + 32u * u;
                tg[u] = 0ull;
                if (j < len) {
                    tg[u] = tag_of(kt + J.bkey[off + j], J);
                    m[u] = mono_mul(t, J.bmon[off + j]);
                    v[u] = J.bcf[off + j];
                }
                hs[u] = home_slot(tg[u], J);
            }
#pragma unroll
            for (int u = 0; u < FH; ++u) {
                if (tg[u]) {
                    const uint4 *sp = reinterpret_cast<const uint4 *>(J.htab + hs[u]);
                    s0[u] = __ldg(sp);
                    s1[u] = __ldg(sp + 1);
                }
            }
#pragma unroll
            for (int u = 0; u < FH; ++u) {
                const uint32_t j = j0 + 32u * u;
                if (j < len) {
                    uint32_t c = 0xFFFFFFFFu;
                    const unsigned long long t0 = ((unsigned long long)s0[u].y << 32) | s0[u].x;
                    uint4 h = s1[u];
                    uint32_t hc = s0[u].z;
                    if (t0 != tg[u]) {  // not in its home slot: probe
                        const uint32_t sl = h_find(tg[u], J);
                        if (sl != 0xFFFFFFFFu) {
                            h = J.htab[sl].mon;
                            hc = J.htab[sl].col;
                        } else {
                            h = make_uint4(~0u, ~0u, ~0u, ~0u);
                        }
                    }
                    if (h.x == m[u].x && h.y == m[u].y && h.z == m[u].z && h.w == m[u].w) c = hc;
                    clash |= c >= J.N;
                    J.col[s + j] = c;
                    J.val[s + j] = v[u];
                }
            }
        }
        if (clash) atomicOr(&J.cnt->err, ERR_KEY_CLASH);
        return;
    }
    // four terms per lane in flight: their ranks and dictionary lookups are independent
    for (uint32_t j0 = lane; j0 < len; j0 += 4 * 32) {
        uint32_t r[4], v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t j = j0 + 32u * u;
            if (j < len) {
                r[u] = mono_rank(mono_mul(t, J.bmon[off + j]), tab, J.n, J.sh, J.deglex != 0);
                v[u] = J.bcf[off + j];
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t j = j0 + 32u * u;
            if (j < len) {
                J.col[s + j] = col_of(J, r[u]);
                J.val[s + j] = v[u];
            }
        }
    }
}

// plan checks: dictionary size, pivot count, nnz and error flags of every job
__global__ void k_check(const Job *__restrict__ jobs, int nj, const uint8_t *__restrict__ live,
                        uint32_t *__restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nj || !live[j]) return;
    const Job &J = jobs[j];
    out[4 * j + 0] = J.wpre[J.W] - J.wpre[0];
    out[4 * j + 1] = J.pidx[J.N] - J.pidx[0];
    out[4 * j + 2] = J.row_ptr[J.nrows];
    out[4 * j + 3] = J.cnt->err;
}

inline unsigned blocks(size_t n, unsigned t) { return (unsigned)((n + t - 1) / t); }

uint64_t binom(uint32_t a, uint32_t b) {
    if (b > a) return 0;
    b = std::min(b, a - b);
    unsigned __int128 r = 1;
    for (uint32_t i = 1; i <= b; ++i) r = r * (a - b + i) / i;
    return r > (unsigned __int128)UINT64_MAX ? UINT64_MAX : (uint64_t)r;
}

// host part of one job
struct SpHost {
    uint32_t D = 0, D1 = 0, sh = 0, W = 0, ng = 0, npiv_given = 0, nnp = 0, tabsz = 0;
    uint64_t space = 0, nnz_given = 0, cap = 0;
    std::vector<uint32_t> tab, np_index;
    std::vector<uint4> gt, nlm;
    std::vector<uint32_t> gk;
    std::vector<uint8_t> gf;
    size_t o_gt = 0, o_gk = 0, o_gf = 0, o_np = 0, o_tab = 0, o_nri = 0, o_nrl = 0;
    DBuf<uint32_t> bits, lm_rank, qrank, red_k, red_rank;
    DBuf<uint4> qmon, red_t;
    // hash dictionary
    bool hash = false;
    uint64_t hcap = 0;
    DBuf<HSlot> htab;
    DBuf<uint32_t> qslot, red_slot, lm_slot;
    Counters hc{};
    uint32_t rounds = 0;
    bool overflow = false;
    bool table_full = false;
};

uint64_t pow2_at_least(uint64_t x) {
    uint64_t c = 1;
    while (c < x) c <<= 1;
    return c;
}

}  // namespace

void symbolic_preprocess(std::vector<SpTask> &tasks) {
    if (tasks.empty()) return;
    gb_ctx *ctx = tasks[0].S->ctx;
    Arena &ar = ctx->arena;
    cudaStream_t st = ctx->stream;
    const int nj = (int)tasks.size();
    GB_CUDA(cudaEventRecord(ctx->ev[0], st));

    std::vector<SpHost> H(nj);
    Stage sg;
    // GB_SP_KEY_MASK=<mask> in the environment keeps only those bits of the hash keys, so that
    // distinct monomials share keys: the fallback to the rank path is then exercised by tests
    unsigned long long keymask = ~0ull;
    if (const char *km = std::getenv("GB_SP_KEY_MASK")) keymask = std::strtoull(km, nullptr, 0);
    // GB_SP_TABLE_SLOTS=<power of two> starts every hash dictionary that small (tests of its growth)
    uint64_t first_slots = 0;
    if (const char *ts = std::getenv("GB_SP_TABLE_SLOTS")) first_slots = std::strtoull(ts, nullptr, 0);
    if (first_slots & (first_slots - 1)) first_slots = 0;
    for (int j = 0; j < nj; ++j) {
        SpTask &T = tasks[j];
        gb_system *S = T.S;
        SpHost &h = H[j];
        const int n = (int)S->n;
        h.ng = (uint32_t)T.rows.size();
        for (const RowSpec &r : T.rows)
            h.D = std::max<uint32_t>(h.D, (uint32_t)(mono_deg(r.t, n) + mono_deg(S->lm[r.k], n)));
        if (h.D > 255) fail(GB_EOVERFLOW, "step degree above 255");
        h.space = binom((uint32_t)n + h.D, (uint32_t)n);
        if (h.space >= (1ull << 32) - 64)
            fail(GB_EUNSUPPORTED, "monomial space C(n+D, n) above 2^32 for the dense monomial keys");
        h.D1 = h.D + 1;
        h.sh = 0;
        while ((1u << h.sh) < h.D1) ++h.sh;
        h.W = (uint32_t)((h.space + 31) / 32);
        h.tab.assign((size_t)n << h.sh, 0);
        for (uint32_t d = 0; d <= h.D; ++d) h.tab[d] = (uint32_t)(d ? binom(n + d - 1, n) : 0);
        for (int i = 1; i < n; ++i)
            for (uint32_t s = 0; s <= h.D; ++s)
                h.tab[((size_t)i << h.sh) + s] =
                    (uint32_t)(S->deglex ? binom(s + (uint32_t)(n - i), (uint32_t)(n - i)) : binom(s + i - 1, i));
        h.tabsz = (uint32_t)h.tab.size();
        h.np_index.assign(h.ng, 0xFFFFFFFFu);
        h.gt.resize(h.ng);
        h.gk.resize(h.ng);
        h.gf.resize(h.ng);
        for (uint32_t i = 0; i < h.ng; ++i) {
            const RowSpec &r = T.rows[i];
            if (r.pivot) ++h.npiv_given;
            else h.np_index[i] = h.nnp++;
            h.nnz_given += S->len[r.k] - r.skip;
            h.gt[i] = to_u4(r.t);
            h.gk[i] = r.k;
            h.gf[i] = (uint8_t)((r.pivot ? FLAG_PIVOT : 0u) | (r.skip ? FLAG_TAIL : 0u));
        }
        h.nlm.resize(T.nonred.size());
        for (size_t i = 0; i < T.nonred.size(); ++i) h.nlm[i] = to_u4(S->lm[T.nonred[i]]);
        h.o_gt = sg.put(h.gt.data(), 16ull * h.ng);
        h.o_gk = sg.put(h.gk.data(), 4ull * h.ng);
        h.o_gf = sg.put(h.gf.data(), h.ng);
        h.o_np = sg.put(h.np_index.data(), 4ull * h.ng);
        h.o_tab = sg.put(h.tab.data(), 4ull * h.tabsz);
        h.o_nri = sg.put(T.nonred.data(), 4ull * T.nonred.size());
        h.o_nrl = sg.put(h.nlm.data(), 16ull * h.nlm.size());
        h.cap = T.cap ? T.cap : std::min<uint64_t>(h.space, std::max<uint64_t>(1u << 14, 2ull * h.nnz_given));
        h.bits.alloc(ar, h.W, st);
        h.lm_rank.alloc(ar, h.ng, st);
        h.qmon.alloc(ar, h.cap, st);
        h.qrank.alloc(ar, h.cap, st);
        h.red_t.alloc(ar, h.cap, st);
        h.red_k.alloc(ar, h.cap, st);
        h.red_rank.alloc(ar, h.cap, st);
        GB_CUDA(cudaMemsetAsync(h.bits.p, 0, 4ull * h.W, st));
        // hash dictionary: at most half full at the expected size (4 x the last step's dictionary)
        h.hash = (ctx->flags & GB_CTX_SP_HASH) && !T.ranks;
        if (h.hash) {
            h.hcap = T.hcap ? T.hcap : first_slots ? first_slots
                            : pow2_at_least(std::min<uint64_t>(2 * h.space + 2,
                                                               std::max<uint64_t>({1u << 14, 4ull * S->last_ndict,
                                                                                   2ull * h.ng})));
            h.htab.alloc(ar, h.hcap, st);
            h.qslot.alloc(ar, h.cap, st);
            h.red_slot.alloc(ar, h.cap, st);
            h.lm_slot.alloc(ar, h.ng, st);
            GB_CUDA(cudaMemsetAsync(h.htab.p, 0, sizeof(HSlot) * h.hcap, st));
        }
    }
    // every job of one call takes the same path, so that each launch is one kernel instantiation
    const bool hash = H[0].hash;
    for (int j = 1; j < nj; ++j)
        if (H[j].hash != hash) fail(GB_EDEVICE, "symbolic preprocessing: jobs of one call on different key paths");
    std::vector<uint32_t> bm(nj), be(nj);
    int max_tab = 1;
    for (int j = 0; j < nj; ++j) {
        bm[j] = blocks(H[j].ng, 256);
        be[j] = blocks(H[j].ng, WPB);
        max_tab = std::max<int>(max_tab, (int)H[j].tabsz);
    }
    size_t o_bm, o_be;
    const uint32_t tbm = plan(sg, bm, o_bm), tbe = plan(sg, be, o_be);
    const size_t o_jobs = sg.put(nullptr, sizeof(Job) * nj);
    DBuf<Counters> cnt;
    cnt.alloc(ar, nj, st);
    GB_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(Counters) * nj, st));
    // the device staging buffer holds the job table, so its address is needed first
    DBuf<char> dstage;
    dstage.alloc(ar, sg.h.size() + 16, st);
    auto dptr = [&](size_t off) { return dstage.p + off; };
    std::vector<Job> jobs(nj);
    for (int j = 0; j < nj; ++j) {
        SpTask &T = tasks[j];
        gb_system *S = T.S;
        SpHost &h = H[j];
        Job &J = jobs[j];
        J = Job{};
        J.bmon = S->bmon.p;
        J.bcf = S->bcf.p;
        J.boff = S->boff.p;
        J.blen = S->blen.p;
        J.gt = reinterpret_cast<const uint4 *>(dptr(h.o_gt));
        J.gk = reinterpret_cast<const uint32_t *>(dptr(h.o_gk));
        J.gf = reinterpret_cast<const uint8_t *>(dptr(h.o_gf));
        J.gnp = reinterpret_cast<const uint32_t *>(dptr(h.o_np));
        J.ng = h.ng;
        J.bits = h.bits.p;
        J.tab = reinterpret_cast<const uint32_t *>(dptr(h.o_tab));
        J.n = (int)S->n;
        J.sh = (int)h.sh;
        J.tabsz = (int)h.tabsz;
        J.deglex = S->deglex ? 1 : 0;
        J.W = h.W;
        J.nr_idx = reinterpret_cast<const uint32_t *>(dptr(h.o_nri));
        J.nr_lm = reinterpret_cast<const uint4 *>(dptr(h.o_nrl));
        J.nnr = (uint32_t)T.nonred.size();
        J.qmon = h.qmon.p;
        J.qrank = h.qrank.p;
        J.cap = (uint32_t)h.cap;
        J.red_t = h.red_t.p;
        J.red_k = h.red_k.p;
        J.red_rank = h.red_rank.p;
        J.lm_rank = h.lm_rank.p;
        J.cnt = cnt.p + j;
        J.bkey = S->bkey.p;
        if (h.hash) {
            J.htab = h.htab.p;
            J.hmask = (uint32_t)(h.hcap - 1);
            uint32_t lg = 0;
            while ((1ull << lg) < h.hcap) ++lg;
            J.hshift = 64u - lg;
            J.qslot = h.qslot.p;
            J.red_slot = h.red_slot.p;
            J.lm_slot = h.lm_slot.p;
            J.keymask = keymask;
        }
    }
    std::memcpy(sg.h.data() + o_jobs, jobs.data(), sizeof(Job) * nj);
    {
        char *hp = static_cast<char *>(ctx_pinned(ctx, sg.h.size() + 16));
        std::memcpy(hp, sg.h.data(), sg.h.size());
        GB_CUDA(cudaMemcpyAsync(dstage.p, hp, sg.h.size(), cudaMemcpyHostToDevice, st));
    }
    const Job *djobs = reinterpret_cast<const Job *>(dptr(o_jobs));
    const size_t tab_smem = 4ull * max_tab;
    if (tbm) {
        if (hash) k_mark_given<true><<<tbm, 256, tab_smem, st>>>(djobs, reinterpret_cast<const uint32_t *>(dptr(o_bm)), nj);
        else k_mark_given<false><<<tbm, 256, tab_smem, st>>>(djobs, reinterpret_cast<const uint32_t *>(dptr(o_bm)), nj);
        counted();
        if (hash) k_expand_given<true><<<tbe, 32 * WPB, 0, st>>>(djobs, reinterpret_cast<const uint32_t *>(dptr(o_be)), nj);
        else k_expand_given<false><<<tbe, 32 * WPB, tab_smem, st>>>(djobs, reinterpret_cast<const uint32_t *>(dptr(o_be)), nj);
        counted();
    }

    // closure rounds: every job's counters come back in one copy per round
    DBuf<uint32_t> dround;  // [2 nj] ranges, then nj + 1 block starts
    dround.alloc(ar, 3ull * nj + 1, st);
    std::vector<uint32_t> f0(nj, 0);
    for (;;) {
        Counters *hc = static_cast<Counters *>(ctx_pinned(ctx, sizeof(Counters) * nj + 16ull * nj + 64));
        GB_CUDA(cudaMemcpyAsync(hc, cnt.p, sizeof(Counters) * nj, cudaMemcpyDeviceToHost, st));
        ctx_sync(ctx);
        std::vector<uint32_t> buf(3ull * nj + 1, 0);
        uint32_t total = 0;
        for (int j = 0; j < nj; ++j) {
            SpHost &h = H[j];
            h.hc = hc[j];
            if (h.hc.q > h.cap || h.hc.red > h.cap) h.overflow = true;
            if (h.hash && ((h.hc.err & ERR_TABLE_FULL) || 2ull * (h.hc.q + h.npiv_given) > h.hcap)) {
                h.overflow = true;  // the table is fuller than half: again with more slots
                h.table_full = true;
            }
            const bool more = tasks[j].closure && !h.overflow && h.hc.q > f0[j] && jobs[j].nnr > 0;
            buf[2 * j] = f0[j];
            buf[2 * j + 1] = more ? h.hc.q : f0[j];
            buf[2 * nj + j] = total;
            if (more) {
                total += blocks(h.hc.q - f0[j], WPB);
                ++h.rounds;
                f0[j] = h.hc.q;
            }
        }
        buf[3 * nj] = total;
        if (!total) break;
        uint32_t *hb = reinterpret_cast<uint32_t *>(hc);  // the counters have been consumed
        std::memcpy(hb, buf.data(), 4 * buf.size());
        GB_CUDA(cudaMemcpyAsync(dround.p, hb, 4 * buf.size(), cudaMemcpyHostToDevice, st));
        if (hash) k_closure<true><<<total, 32 * WPB, 0, st>>>(djobs, dround.p + 2 * nj, nj, dround.p);
        else k_closure<false><<<total, 32 * WPB, tab_smem, st>>>(djobs, dround.p + 2 * nj, nj, dround.p);
        counted();
    }

    // jobs whose queue overflowed start again with room for what they found
    std::vector<SpTask> retry;
    std::vector<int> retry_of;
    for (int j = 0; j < nj; ++j) {
        if (!H[j].overflow) continue;
        SpTask t;
        t.S = tasks[j].S;
        t.rows = tasks[j].rows;
        t.closure = tasks[j].closure;
        t.nonred = tasks[j].nonred;
        t.ranks = tasks[j].ranks;
        const bool queue_full = H[j].hc.q > H[j].cap || H[j].hc.red > H[j].cap;
        if (queue_full && H[j].cap >= H[j].space) fail(GB_EDEVICE, "frontier queue overflow beyond the monomial space");
        t.cap = queue_full ? std::min<uint64_t>(H[j].space, 4ull * std::max<uint64_t>(H[j].hc.q, H[j].hc.red))
                           : H[j].cap;
        if (H[j].table_full) {
            const uint64_t want = pow2_at_least(4ull * (H[j].hc.q + H[j].npiv_given) + 4);
            t.hcap = std::max<uint64_t>(want, 4 * H[j].hcap);
            if (H[j].hcap > 2 * H[j].space + 2) t.ranks = true;  // cannot grow further: exact path
        }
        retry.push_back(std::move(t));
        retry_of.push_back(j);
    }

    // sizes of the plans that did not overflow
    std::vector<int> live;
    std::vector<uint8_t> live_flag(nj, 0);
    uint64_t tw = 0, tN = 0, tr = 0;
    std::vector<uint64_t> woff(nj, 0), noff(nj, 0), roff(nj, 0);
    for (int j = 0; j < nj; ++j) {
        if (H[j].overflow) continue;
        live.push_back(j);
        live_flag[j] = 1;
        SpHost &h = H[j];
        Job &J = jobs[j];
        J.nq = h.hc.q;
        J.nred = h.hc.red;
        J.N = h.npiv_given + J.nq;
        J.nA = J.nred + h.npiv_given;
        J.nrows = h.ng + J.nred;
        const uint64_t nnz = h.nnz_given + h.hc.red_nnz;
        if (nnz >= (1ull << 32)) fail(GB_EUNSUPPORTED, "more than 2^32 nonzeros in one matrix");
        J.nnz = (uint32_t)nnz;
        woff[j] = tw;
        tw += h.W;
        noff[j] = tN;
        tN += J.N;
        roff[j] = tr;
        tr += J.nrows;
    }
    DBuf<uint32_t> wcnt, wpre, ispiv, src, pidx, lens, lscan;
    wcnt.alloc(ar, tw, st);
    wpre.alloc(ar, tw + 1, st);
    ispiv.alloc(ar, tN, st);
    src.alloc(ar, tN, st);
    pidx.alloc(ar, tN + 1, st);
    lens.alloc(ar, tr, st);
    lscan.alloc(ar, tr + 1, st);
    GB_CUDA(cudaMemsetAsync(ispiv.p, 0, 4 * tN, st));
    for (int j : live) {
        SpTask &T = tasks[j];
        Job &J = jobs[j];
        auto M = std::make_unique<gb_macaulay>();
        M->sys = T.S;
        M->n = T.S->n;
        M->degree = H[j].D;
        M->ndict = J.N;
        M->nA = J.nA;
        M->nC = H[j].nnp;
        M->nb = J.N - J.nA;
        M->nrows = J.nrows;
        M->nnz = J.nnz;
        M->closure_rounds = H[j].rounds;
        M->dict.alloc(ar, J.N, st);
        M->row_t.alloc(ar, J.nrows, st);
        M->row_k.alloc(ar, J.nrows, st);
        M->row_flags.alloc(ar, J.nrows, st);
        M->pcols.alloc(ar, J.nA, st);
        M->nonpiv.alloc(ar, M->nb, st);
        M->colpos.alloc(ar, J.N, st);
        M->row_ptr.alloc(ar, (size_t)J.nrows + 1, st);
        M->col.alloc(ar, J.nnz, st);
        M->val.alloc(ar, J.nnz, st);
        J.wcnt = wcnt.p + woff[j];
        J.wpre = wpre.p + woff[j];
        J.is_piv = ispiv.p + noff[j];
        J.src = src.p + noff[j];
        J.pidx = pidx.p + noff[j];
        J.dict = M->dict.p;
        J.row_t = M->row_t.p;
        J.row_k = M->row_k.p;
        J.row_flags = M->row_flags.p;
        J.pcols = M->pcols.p;
        J.nonpiv = M->nonpiv.p;
        J.colpos = M->colpos.p;
        J.lens = lens.p + roff[j];
        J.lscan = lscan.p + roff[j];
        J.row_ptr = M->row_ptr.p;
        J.col = M->col.p;
        J.val = M->val.p;
        T.out = std::move(M);
    }
    if (!live.empty()) {
        // second-stage job table and plans (jobs that overflowed get no blocks)
        Stage s2;
        std::vector<uint32_t> b_w(nj, 0), b_q(nj, 0), b_g(nj, 0), b_r(nj, 0), b_N(nj, 0), b_rows(nj, 0),
            b_rp(nj, 0), b_fill(nj, 0);
        for (int j : live) {
            const Job &J = jobs[j];
            b_w[j] = blocks(J.W, 256);
            b_q[j] = blocks(J.nq, 256);
            b_g[j] = blocks(J.ng, 256);
            b_r[j] = blocks(J.nred, 256);
            b_N[j] = blocks(J.N, 256);
            b_rows[j] = blocks(J.nrows, 256);
            b_rp[j] = blocks((size_t)J.nrows + 1, 256);
            b_fill[j] = blocks(J.nrows, WPB);
        }
        size_t o_w, o_q, o_g, o_r, o_N, o_rows, o_rp, o_fill;
        const uint32_t t_w = plan(s2, b_w, o_w), t_q = plan(s2, b_q, o_q), t_g = plan(s2, b_g, o_g),
                       t_r = plan(s2, b_r, o_r), t_N = plan(s2, b_N, o_N), t_rows = plan(s2, b_rows, o_rows),
                       t_rp = plan(s2, b_rp, o_rp), t_fill = plan(s2, b_fill, o_fill);
        const size_t o_j2 = s2.put(jobs.data(), sizeof(Job) * nj);
        const size_t o_live = s2.put(live_flag.data(), nj);
        DBuf<char> d2;
        s2.upload(ctx, d2);
        const Job *dj = reinterpret_cast<const Job *>(d2.p + o_j2);
        auto P = [&](size_t o) { return reinterpret_cast<const uint32_t *>(d2.p + o); };
        if (t_q) { k_rank_queue<<<t_q, 256, tab_smem, st>>>(dj, P(o_q), nj); counted(); }
        if (t_w) { k_popc<<<t_w, 256, 0, st>>>(dj, P(o_w), nj); counted(); }
        exclusive_scan(ctx, wcnt.p, wpre.p, tw, st);
        if (t_q) { k_dict_queue<<<t_q, 256, 0, st>>>(dj, P(o_q), nj); counted(); }
        if (t_g) { k_dict_given<<<t_g, 256, 0, st>>>(dj, P(o_g), nj); counted(); }
        GB_CUDA(cudaEventRecord(ctx->ev[6], st));  // the dictionary is complete (DictBuild)
        if (t_r) { k_piv_reducers<<<t_r, 256, 0, st>>>(dj, P(o_r), nj); counted(); }
        exclusive_scan(ctx, ispiv.p, pidx.p, tN, st);
        if (t_N) { k_place_pivots<<<t_N, 256, 0, st>>>(dj, P(o_N), nj); counted(); }
        if (t_g) { k_place_nonpivots<<<t_g, 256, 0, st>>>(dj, P(o_g), nj); counted(); }
        if (t_rows) { k_row_len<<<t_rows, 256, 0, st>>>(dj, P(o_rows), nj); counted(); }
        exclusive_scan(ctx, lens.p, lscan.p, tr, st);
        if (t_rp) { k_row_ptr<<<t_rp, 256, 0, st>>>(dj, P(o_rp), nj); counted(); }
        if (t_fill) {
            if (hash) k_fill<true><<<t_fill, 32 * WPB, 0, st>>>(dj, P(o_fill), nj);
            else k_fill<false><<<t_fill, 32 * WPB, tab_smem, st>>>(dj, P(o_fill), nj);
            counted();
        }
        GB_CUDA(cudaEventRecord(ctx->ev[1], st));
        // consistency of every plan with the host's counts (one small read-back)
        DBuf<uint32_t> chk;
        chk.alloc(ar, 4ull * nj, st);
        k_check<<<blocks(nj, 128), 128, 0, st>>>(dj, nj, reinterpret_cast<const uint8_t *>(d2.p + o_live), chk.p);
        counted();
        uint32_t *hchk = static_cast<uint32_t *>(ctx_pinned(ctx, 16ull * nj + 16));
        GB_CUDA(cudaMemcpyAsync(hchk, chk.p, 16ull * nj, cudaMemcpyDeviceToHost, st));
        ctx_sync(ctx);
        float ms = 0.f, ms_dict = 0.f;
        GB_CUDA(cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]));
        GB_CUDA(cudaEventElapsedTime(&ms_dict, ctx->ev[0], ctx->ev[6]));
        for (int j : live) {
            const Job &J = jobs[j];
            const uint32_t *c = hchk + 4 * j;
            if (c[3] == ERR_KEY_CLASH) {
                // two monomials of this step share a hash key: the exact rank path builds it again
                SpTask t;
                t.S = tasks[j].S;
                t.rows = tasks[j].rows;
                t.closure = tasks[j].closure;
                t.nonred = tasks[j].nonred;
                t.ranks = true;
                tasks[j].out.reset();
                retry.push_back(std::move(t));
                retry_of.push_back(j);
                continue;
            }
            if (c[0] != J.N || c[1] != J.nA || c[2] != J.nnz || c[3])
                fail(GB_EDEVICE, "symbolic preprocessing: device counts disagree with the plan: columns " +
                                     std::to_string(c[0]) + "/" + std::to_string(J.N) + ", pivots " +
                                     std::to_string(c[1]) + "/" + std::to_string(J.nA) + ", nnz " +
                                     std::to_string(c[2]) + "/" + std::to_string(J.nnz) + ", flags " +
                                     std::to_string(c[3]));
            tasks[j].out->ms_sp = ms;
            tasks[j].out->ms_dict = ms_dict;
            tasks[j].S->last_ndict = J.N;
        }
    }
    // again, with more room or on the rank path: one call per path
    for (int ranks = 0; ranks < 2; ++ranks) {
        std::vector<SpTask> again;
        std::vector<int> again_of;
        for (size_t i = 0; i < retry.size(); ++i) {
            const bool on_ranks = retry[i].ranks || !(ctx->flags & GB_CTX_SP_HASH);
            if (on_ranks != (ranks == 1)) continue;
            again.push_back(std::move(retry[i]));
            again_of.push_back(retry_of[i]);
        }
        if (again.empty()) continue;
        symbolic_preprocess(again);
        for (size_t i = 0; i < again.size(); ++i) {
            tasks[again_of[i]].out = std::move(again[i].out);
            tasks[again_of[i]].out->sp_redo += 1;
        }
    }
}

namespace {
__global__ void k_basis_keys(const uint4 *__restrict__ mon, unsigned long long *__restrict__ key, uint64_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        key[i] = mono_key(mon[i]);
}
}  // namespace

void basis_keys(const uint4 *mon, unsigned long long *key, uint64_t n, cudaStream_t st) {
    if (!n) return;
    k_basis_keys<<<(unsigned)std::min<uint64_t>((n + 255) / 256, 148 * 8), 256, 0, st>>>(mon, key, n);
    counted();
}

}  // namespace gb
