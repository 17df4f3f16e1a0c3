// device.cuh -- register-level primitives shared by the kernels: F_p arithmetic (Sec. 8) and
// packed monomials with an injective, order-refining key (Sec. 7.3; the key assumption of Sec. 11).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace gb {

// ---------------------------------------------------------------------------------------------
// F_p arithmetic.  Residues are standard representatives in [0, p), p odd, p < 2^31.
//
// Barrett (Sec. 8.3) with k = 64: mu = floor(2^64 / p).  For any x < 2^64,
// q = floor(x * mu / 2^64) satisfies floor(x/p) - 1 <= q <= floor(x/p), so r = x - q p lies in
// [0, 2p) and one predicated subtraction finishes.  This reduces lazily accumulated sums
// (the lazy window of Rem. 8.1) and single products.
//
// Montgomery (Sec. 8.4) with R = 2^32 and p' = -p^{-1} mod R: redc(t) = (t + ((t mod R) p' mod R) p)
// / R is congruent to t R^{-1} and lies in [0, 2p) for t < p R.  The sparse row update multiplies
// every entry of a pivot row by one scalar f; with f converted once to f R mod p, redc(fR * v) is
// f v mod p (up to one p) for a standard v, so the entries never leave standard form.
// ---------------------------------------------------------------------------------------------
struct Fp {
    uint32_t p;
    uint32_t pinv_neg;  // -p^{-1} mod 2^32
    uint64_t mu;        // floor(2^64 / p)
    uint32_t r2;        // R^2 mod p
    uint32_t small;     // 1 when p < 2^16: products of residues fit in 32 bits
    uint32_t mu32;      // floor(2^32 / p), for the 32-bit Barrett reduction (p < 2^16)
    uint32_t pad;
};

#ifdef __CUDACC__
__device__ __forceinline__ uint32_t fp_reduce(uint64_t x, const Fp &f) {
    uint64_t q = __umul64hi(x, f.mu);
    uint64_t r = x - q * (uint64_t)f.p;
    return (uint32_t)(r >= f.p ? r - f.p : r);
}

// x mod p for x < 2^32 and p < 2^16: Barrett with k = 32 (same argument as above, one correction)
__device__ __forceinline__ uint32_t fp_reduce32(uint32_t x, const Fp &f) {
    const uint32_t q = __umulhi(x, f.mu32);
    const uint32_t r = x - q * f.p;
    return r >= f.p ? r - f.p : r;
}

__device__ __forceinline__ uint32_t fp_mul(uint32_t a, uint32_t b, const Fp &f) {
    return fp_reduce((uint64_t)a * b, f);
}

__device__ __forceinline__ uint32_t fp_add(uint32_t a, uint32_t b, const Fp &f) {
    uint32_t s = a + b;
    return s >= f.p ? s - f.p : s;
}

__device__ __forceinline__ uint32_t fp_sub(uint32_t a, uint32_t b, const Fp &f) {
    return a >= b ? a - b : a + f.p - b;
}

// t R^{-1} mod p, in [0, 2p), for t < p * 2^32
__device__ __forceinline__ uint32_t fp_redc(uint64_t t, const Fp &f) {
    uint32_t m = (uint32_t)t * f.pinv_neg;
    return (uint32_t)((t + (uint64_t)m * f.p) >> 32);
}

// a R mod p in [0, p)
__device__ __forceinline__ uint32_t fp_to_mont(uint32_t a, const Fp &f) {
    uint32_t r = fp_redc((uint64_t)a * f.r2, f);
    return r >= f.p ? r - f.p : r;
}

// a^{-1} mod p (0 < a < p, p odd) by the binary extended Euclidean algorithm (Menezes, van
// Oorschot, Vanstone, Handbook of Applied Cryptography, Alg. 14.61 in its modular-inverse form):
// shifts and subtractions on 32-bit values only, about 2 log2(p) iterations, no division.
// Invariants: x1 a = u and x2 a = v (mod p); the loop ends when u or v reaches 1.
__device__ __forceinline__ uint32_t fp_inv(uint32_t a, const Fp &f) {
    const uint32_t p = f.p;
    uint32_t u = a, v = p, x1 = 1, x2 = 0;
    while (u != 1 && v != 1) {
        while (!(u & 1)) {
            u >>= 1;
            x1 = (x1 & 1) ? (uint32_t)(((uint64_t)x1 + p) >> 1) : x1 >> 1;
        }
        while (!(v & 1)) {
            v >>= 1;
            x2 = (x2 & 1) ? (uint32_t)(((uint64_t)x2 + p) >> 1) : x2 >> 1;
        }
        if (u >= v) {
            u -= v;
            x1 = x1 >= x2 ? x1 - x2 : x1 + p - x2;
        } else {
            v -= u;
            x2 = x2 >= x1 ? x2 - x1 : x2 + p - x1;
        }
    }
    return u == 1 ? x1 : x2;
}

// a^{-1} = a^(p-2) mod p (Fermat's little theorem) for p < 2^16: right-to-left square-and-multiply
// with the 32-bit Barrett reduction (every product of two residues is below 2^32).  A straight
// chain of about 30 products: shorter on the GPU than the branching Euclid above for 16-bit p.
__device__ __forceinline__ uint32_t fp_inv_small(uint32_t a, const Fp &f) {
    uint32_t r = 1u, b = a;
    for (uint32_t e = f.p - 2u; e; e >>= 1) {
        if (e & 1u) r = fp_reduce32(r * b, f);
        b = fp_reduce32(b * b, f);
    }
    return r;
}

// ---------------------------------------------------------------------------------------------
// Monomials: n <= 16 exponents of 8 bits packed little-endian in a uint4 (byte i = exponent of
// x_{i+1}).  Multiplication is a bytewise add; the library keeps every exponent and degree below
// 256, so the four 32-bit adds never carry across bytes.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ uint4 mono_mul(uint4 a, uint4 b) {
    return make_uint4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}

__device__ __forceinline__ uint4 mono_div(uint4 b, uint4 a) {  // requires a | b
    return make_uint4(b.x - a.x, b.y - a.y, b.z - a.z, b.w - a.w);
}

__device__ __forceinline__ bool mono_divides(uint4 a, uint4 b) {  // a | b: every byte a_i <= b_i
    return (__vcmpleu4(a.x, b.x) & __vcmpleu4(a.y, b.y) & __vcmpleu4(a.z, b.z) &
            __vcmpleu4(a.w, b.w)) == 0xFFFFFFFFu;
}

__device__ __forceinline__ uint32_t byte_of(uint4 m, int i) {
    uint32_t w = i < 4 ? m.x : i < 8 ? m.y : i < 12 ? m.z : m.w;
    return (w >> (8 * (i & 3))) & 0xFFu;
}

// Dense grevlex rank: the position of x^a among all monomials in n variables, ascending in grevlex
// with x1 > ... > xn.  With S_j = a_1 + ... + a_j and d = S_n:
//     rank(a) = C(n + d - 1, n) + sum_{j=1}^{n-1} C(S_j + j - 1, j).
// C(n + d - 1, n) counts the monomials of degree < d.  Within degree d, a monomial b is smaller
// than a iff at the last index where they differ b has the larger exponent; fixing b_n..b_{j+2} to
// a's and letting b_{j+1} exceed a_{j+1} leaves the first j variables to share a total below S_j,
// which C(S_j + j - 1, j) counts.  The rank is injective and order-preserving (the key assumption
// of Sec. 11),
// so it serves as MonKey, and as a bitmap index in [0, C(n + D, n)) for degrees <= D.
//
// Dense deglex rank (deglex: the first differing exponent decides, the larger one giving the
// larger monomial):
//     rank(a) = C(n + d - 1, n) + sum_{j=1}^{n-1} [C(d - S_{j-1} + n - j, n - j) - C(d - S_j + n - j, n - j)]
// (S_0 = 0).  Within degree d, a monomial b is smaller than a iff at the first index j where they
// differ b_j < a_j; with b_1..b_{j-1} fixed to a's, C(d - S_{j-1} + n - j, n - j) counts the
// completions with b_j >= 0 and C(d - S_j + n - j, n - j) those with b_j >= a_j, so the difference
// counts b_j < a_j (a hockey-stick sum).
//
// tab (shared memory), rows of 2^sh entries: row 0 holds tab[d] = C(n + d - 1, n) for d in [0, D];
// row j = 1..n-1 holds, for s in [0, D] (2^sh > D), tab[(j << sh) + s] = C(s + j - 1, j) (grevlex)
// or C(s + n - j, n - j) (deglex).
// The prefix sums S_j come four at a time from one multiply: byte k of w * 0x01010101 is the sum of
// bytes 0..k of w (no byte carries: every S_j <= D <= 255), and the running total is added to every
// byte of the next word the same way.
__device__ __forceinline__ uint32_t mono_rank(uint4 m, const uint32_t *tab, int n, int sh, bool deglex) {
    const uint32_t p0 = m.x * 0x01010101u;
    const uint32_t p1 = m.y * 0x01010101u + (p0 >> 24) * 0x01010101u;
    const uint32_t p2 = m.z * 0x01010101u + (p1 >> 24) * 0x01010101u;
    const uint32_t p3 = m.w * 0x01010101u + (p2 >> 24) * 0x01010101u;
    const uint32_t d = __dp4a(m.x, 0x01010101u, 0u) + __dp4a(m.y, 0x01010101u, 0u) +
                       __dp4a(m.z, 0x01010101u, 0u) + __dp4a(m.w, 0x01010101u, 0u);
    uint32_t r = 0, prev = 0;  // prev = S_{j-1}
#pragma unroll
    for (int j = 1; j < 16; ++j) {
        if (j >= n) break;
        const uint32_t w = j <= 4 ? p0 : j <= 8 ? p1 : j <= 12 ? p2 : p3;  // S_j is byte j - 1
        const uint32_t sj = (w >> (8 * ((j - 1) & 3))) & 0xFFu;
        if (deglex) {
            r += tab[(j << sh) + d - prev] - tab[(j << sh) + d - sj];
            prev = sj;
        } else {
            r += tab[(j << sh) + sj];
        }
    }
    return r + tab[d];
}

// Linear monomial key for the hash dictionary of symbolic preprocessing:
//     key(a) = sum_i a_i K_i  mod 2^64,   K_i fixed odd 64-bit constants (SplitMix64 outputs).
// It is additive, key(t m) = key(t) + key(m), so the key of a shifted term costs one 64-bit add
// once every basis term carries its own key.  It is not injective: distinct monomials may share
// a key, so every dictionary lookup compares the stored monomial and a mismatch sends the step to
// the exact rank path.  For a fixed pair a != b the differences a_i - b_i are below 2^8 in
// magnitude, so a random K gives key(a) = key(b) with probability at most 2^-56.
static __constant__ unsigned long long MONO_KEY_K[16] = {
    0x63cfc62a2b097593ull, 0xdc0746b419466aedull, 0x08264674f98aa19full, 0x3ca4eb47b26de7adull,
    0xa5b384ad339cfcc3ull, 0x08f720d059892bc5ull, 0xfe6675c92d60f3dfull, 0x1d59c7b9c3a56969ull,
    0xea5685b6014a22c9ull, 0x3935c47ec47e016dull, 0xf72314ef3d87ae57ull, 0xe2c2311ba18cfd93ull,
    0x509d7011d7bc72c9ull, 0x4cd89b9538c27513ull, 0xa4e38806108a16a3ull, 0x5a469fb3420a4217ull};

__device__ __forceinline__ unsigned long long mono_key(uint4 m) {
    const uint32_t w[4] = {m.x, m.y, m.z, m.w};
    unsigned long long h = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) h += (unsigned long long)((w[i >> 2] >> (8 * (i & 3))) & 0xFFu) * MONO_KEY_K[i];
    return h;
}

// SplitMix64 (Steele, Lea, Flood 2014): counter-based pseudo-random words for the random
// combinations of the block Wiedemann path and of the sketched echelon form
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
    unsigned long long z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint32_t mono_deg(uint4 m) {
    return __dp4a(m.x, 0x01010101u, 0u) + __dp4a(m.y, 0x01010101u, 0u) +
           __dp4a(m.z, 0x01010101u, 0u) + __dp4a(m.w, 0x01010101u, 0u);
}

// column of a monomial in the dictionary: the dictionary is the set bits of `bits` (indexed by
// rank) in descending order, word_prefix[w] = set bits in words [0, w)
__device__ __forceinline__ uint32_t rank_to_col(uint32_t r, const uint32_t *bits,
                                                const uint32_t *word_prefix, uint32_t N) {
    uint32_t w = r >> 5, below = bits[w] & ((1u << (r & 31)) - 1u);
    return N - 1u - (word_prefix[w] + __popc(below));
}

// block -> job of a grouped launch: bstart[j] is the first block of job j (non-decreasing, nj
// entries); the largest j with bstart[j] <= blockIdx.x (jobs without blocks are skipped)
__device__ __forceinline__ int job_of_block(const uint32_t *__restrict__ bstart, int nj) {
    int lo = 0, hi = nj - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (bstart[mid] <= blockIdx.x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

#endif  // __CUDACC__

}  // namespace gb
