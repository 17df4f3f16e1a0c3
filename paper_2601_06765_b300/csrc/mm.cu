// mm.cu -- exact dense multiply-accumulate over F_p on the fifth-generation tensor cores:
//     C <- C - A B  (mod p)   or   C <- C + A B  (mod p),
// the GEMM-like block update of the panel-structured elimination (Sec. 9.2) with the modular
// arithmetic of Sec. 8 moved to the epilogue.
//
// Exactness.  A residue x in [0, p) is taken as the representative v = x (x <= T) or x - p
// (x > T), T = 127 (1 + 256 + ... + 256^{L-1}), and written with L balanced base-256 digits
//     v = sum_l a_l 256^l,   a_l in [-128, 127]
// (L = 2 for p < 2^16, L = 4 for p < 2^31; every v lies in the range those digits cover).  A digit
// is an integer of at most 8 significant bits, so it is exact in BF16, and a product of two digits
// (|a b| <= 2^14) is exact in FP32.  For each digit diagonal s the tensor cores accumulate
//     D_s = sum_k sum_{i+j=s} a_i(k) b_j(k)
// in FP32; with c_s <= L products per k, |partial sums| <= K L 2^14 <= 2^23 for K <= 512 / L,
// so every partial sum is an integer the FP32 accumulator holds exactly (with a bit to spare).  The
// epilogue converts each D_s to an integer, pairs adjacent small diagonals in 32 bits, forms
// sum_s D_s (256^s 2^32 mod p) in 64 bits, reduces it once (Montgomery) and adds C, which equals
// (C -/+ A B)[m][n] mod p.  One launch covers K <= 512 / L; longer products are
// split by the host into launches that each update C.
//
// Kernel: persistent, one CTA per SM, each CTA takes a contiguous run of the 128 x (128/L) output
// tiles in row-major tile order.  Every product is one tcgen05.mma (kind::f16, BF16 operands, FP32
// accumulators) of M = 128, N = 128, K = 16: one digit of A against all L digits of B^T side by
// side (128/L rows each), its accumulator window starting at diagonal i, so that A_i B_j lands on
// diagonal i + j.  18 warps:
//   warp 0, lane 0   TMA producer: the digit planes of A for the CTA's current 128-row tile (all of
//                    K, resident in shared memory while the row tile lasts), then per output tile
//                    the K blocks of B^T (all digits in one box) through a ring of slots, and an L2
//                    prefetch of the next tile's C (128-byte swizzle; mbarriers with transaction
//                    counts)
//   warp 1           allocates the tensor memory (two accumulator sets of 2L - 1 diagonals,
//                    alternate tiles) and issues the products from lane 0
//   warps 2-17       epilogue, in EG groups that take alternate tiles (two groups of eight warps
//                    for L = 4, one of sixteen for L = 2; each group covers the four tensor-memory
//                    lane quarters, a thread 16 columns of its row): drains the tile's set as soon
//                    as its products are done (tcgen05.ld of every diagonal, exact conversion,
//                    sum_s D_s (256^s 2^32 mod p) and one Montgomery reduction), zeroes it
//                    (tcgen05.st) and hands it back, so that every product accumulates; then adds
//                    C in the read-modify-write of the group's C buffer in shared memory
//                    (optionally also writing the digit planes of the result's first columns);
//                    one thread of the group issues the TMA store and loads the C tile of the
//                    group's next tile into the freed buffer
// so that one set's products run while the other is drained.  Every wait is bounded; a wait that
// gives up sets an error flag that the host turns into GB_ETIMEOUT, and the CTA still releases its
// tensor memory.  Runs of consecutive launches are programmatic dependent launches (launch_mm).
#include <cuda.h>

#include <algorithm>
#include <cstring>

#include "internal.hpp"

namespace gb {

namespace {

constexpr int MM_BM = 128, MM_BK = 64;  // rows of a C tile, K block (64 BF16 = 128 bytes)
constexpr int MM_MMA_N = 128;           // N of every tcgen05.mma: the L digits of B^T side by side
constexpr int MM_EPI = 16;              // epilogue warps: four per tensor-memory lane quarter
constexpr int MM_THREADS = 32 * (2 + MM_EPI);
constexpr uint32_t MM_SPIN = 1u << 22;  // bounded mbarrier waits

template <int L>
struct MmCfg {
    static constexpr int DIAG = 2 * L - 1;             // digit diagonals
    static constexpr int BN = MM_MMA_N / L;            // columns of a C tile: 32 (L = 4), 64 (L = 2)
    static constexpr int KB = 512 / L / MM_BK;         // K blocks of the longest exact K
    // epilogue groups taking alternate tiles, warps in each (all four lane quarters, WPG / 4 times)
    static constexpr int EG = L == 4 ? 2 : 1;
    static constexpr int WPG = MM_EPI / EG;
    static constexpr int CPT = BN * 4 / WPG;           // columns of each epilogue thread
    static constexpr int DRAIN = DIAG * CPT <= 64 ? CPT : 8;  // columns drained per tensor-memory wait
    static constexpr uint32_t A_BLK = MM_BM * 128;     // bytes of one digit x K block of A
    static constexpr uint32_t A_BYTES = L * KB * A_BLK;
    static constexpr uint32_t B_BLK = MM_MMA_N * 128;  // one K block of B^T: L digits x BN rows
    static constexpr uint32_t C_BOX = MM_BM * 32 * 4;  // one 32-column TMA box of C
    static constexpr int C_BOXES = BN / 32;
    static constexpr uint32_t C_TILE = C_BOXES * C_BOX;
    static constexpr int NCBUF = C_TILE <= 16384u ? 2 : 1;  // C tiles in flight
    static constexpr uint32_t C_BYTES = NCBUF * C_TILE;
    // B^T streams through a ring of K-block slots: as many as fit beside A and C
    static constexpr uint32_t SMEM_MAX = 227u * 1024u;
    static constexpr uint32_t OVERHEAD = 1024 + 512;  // alignment + barriers
    static constexpr int NSLOT = (int)((SMEM_MAX - OVERHEAD - A_BYTES - C_BYTES) / B_BLK);
    static constexpr uint32_t B_BYTES = (uint32_t)NSLOT * B_BLK;
    static constexpr uint32_t SMEM_DATA = A_BYTES + C_BYTES + B_BYTES;
    static constexpr uint32_t SMEM = SMEM_DATA + OVERHEAD;
    // two accumulator sets (tiles alternate), set s at tensor-memory column 256 s; diagonal d of a
    // set at column BN d
    static constexpr uint32_t SET_COLS = 256;
    static constexpr uint32_t TMEM_COLS = 512;
    static_assert(DIAG * BN <= (int)SET_COLS, "tensor memory");
    static_assert(NSLOT >= 2, "shared memory");
};

struct MmParams {
    uint32_t M, N, K;       // the update covers C[cy + m][cx + n], m < M, n < N; K <= 512 / L
    int ax, ay, bx, by;     // TMA coordinates of A (k, m) and of B^T (k, n) at the origin
    int cx, cy;             // TMA coordinates of the update region in C
    uint32_t ntn, items;    // tiles per tile row (BN columns each), tiles in all
    Fp fp;
    uint64_t big;           // 2^31 p, which keeps the accumulated sum positive
    uint32_t rd[7];         // (256^d mod p) 2^32 mod p (C += A B), or (p - 256^d mod p) 2^32 mod p
    uint32_t *err;          // bit 0: a bounded wait gave up
    // optional: the digit planes of the updated entries of the region's first dig_cols columns
    // (a multiple of 16) go to dig (row m, K index n; row pitch dig_kpad, plane pitch dig_plane)
    uint16_t *dig;
    uint64_t dig_kpad, dig_plane;
    uint32_t dig_cols;
};

// ---- PTX wrappers (sm_100 family) ----------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// wait for the phase of the given parity to complete; false when the bound runs out
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (uint32_t i = 0; i < MM_SPIN; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y), "r"(z)
        : "memory");
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
        : "memory");
}
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, uint32_t src, int x, int y) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(src), "r"(x), "r"(y)
                 : "memory");
}
// bring a box of a tensor into L2 (no shared memory, no completion to wait for)
__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap *map, int x, int y) {
    asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// the named barrier of epilogue group g, NT threads (barrier 0 is __syncthreads)
template <int NT>
__device__ __forceinline__ void epi_sync(int g) { asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "n"(NT) : "memory"); }
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
// N consecutive 32-bit columns (N = 8 or 16) of this thread's tensor-memory lane
template <int N>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, uint32_t (&r)[N]) {
    if constexpr (N == 16) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
              "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr));
    } else {
        static_assert(N == 8, "8 or 16 columns");
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                     : "r"(taddr));
    }
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// zeros into N = 8 or 16 consecutive 32-bit columns of this thread's tensor-memory lane
template <int N>
__device__ __forceinline__ void tmem_zero(uint32_t taddr) {
    if constexpr (N == 16) {
        asm volatile(
            "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1};" ::"r"(taddr),
            "r"(0u)
            : "memory");
    } else {
        static_assert(N == 8, "8 or 16 columns");
        asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1};" ::"r"(taddr), "r"(0u)
                     : "memory");
    }
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }


// Shared-memory matrix descriptor of a K-major tile with 128-byte swizzle: rows of 128 bytes,
// 8-row groups 1024 bytes apart (stride byte offset), descriptor version 1, layout type 2.
// The tile base is 1024-byte aligned; a K offset inside the 128-byte row moves the start address.
// Low word: start address >> 4 (bits 0-13), leading byte offset 16 >> 4 (bits 16-29); adding a
// 16-byte-unit offset to it moves the start address (shared addresses stay below 2^18, so the
// 14-bit field never carries).  High word: stride byte offset 1024 >> 4, version, swizzle mode.
__device__ __forceinline__ uint32_t sdesc_lo(uint32_t addr) { return ((addr & 0x3FFFFu) >> 4) | (1u << 16); }
constexpr uint32_t SDESC_HI = (1024u >> 4) | (1u << 14) | (2u << 29);
__device__ __forceinline__ uint64_t sdesc_of(uint32_t lo) { return ((uint64_t)SDESC_HI << 32) | lo; }

// Instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A and B (bits 7-9,
// 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(MM_BM >> 4) << 24);
}

__device__ __forceinline__ int acc_int(uint32_t bits) { return __float2int_rn(__uint_as_float(bits)); }
// The same for |x| <= 2^22 without the conversion unit: x + 1.5 2^23 lies in [2^23, 2^24], where
// FP32 steps by 1, so the sum is exact and its bit pattern minus that of 1.5 2^23 is x (the
// classic round-by-adding-a-magic-constant conversion; 2^24 itself continues the pattern).
__device__ __forceinline__ int acc_int_small(uint32_t bits) {
    return __float_as_int(__fadd_rn(__uint_as_float(bits), 12582912.0f)) - 0x4B400000;
}
// D_lo + 256 D_hi for two diagonals of the small kind whose sum stays below 2^31 in magnitude,
// from the two biased bit patterns: the bias of both, 257 times that of 1.5 2^23, comes off once
// (wrapping 32-bit arithmetic; the true value fits, so the wrapped result is exact)
__device__ __forceinline__ int acc_pair_small(uint32_t lo, uint32_t hi) {
    const uint32_t a = (uint32_t)__float_as_int(__fadd_rn(__uint_as_float(lo), 12582912.0f));
    const uint32_t b = (uint32_t)__float_as_int(__fadd_rn(__uint_as_float(hi), 12582912.0f));
    return (int)(a + (b << 8) - 257u * 0x4B400000u);
}
// Diagonal d sums min(d + 1, 2L - 1 - d) digit products per k, so |D_d| <= that count x (512 / L)
// x 2^14 at the largest K of a launch; where this is at most 2^22 (diagonals 0, 1, 5, 6 for L = 4;
// 0, 2 for L = 2) the conversion above is exact.
template <int L>
__host__ __device__ constexpr bool small_diag(int d) {
    return (long long)(d + 1 < 2 * L - 1 - d ? d + 1 : 2 * L - 1 - d) * (512 / L) * 16384 <= (1ll << 22);
}

// Digit planes: dst[l][r][k] (row pitch kpad, plane pitch rows * kpad) = BF16 bits of the l-th
// balanced base-256 digit of a residue x (representative x or x - p, T as in the header).
template <int L>
__device__ __forceinline__ void digits_of(uint32_t x, uint32_t p, uint32_t (&a)[L]) {
    const uint32_t T = L == 2 ? 32639u : 2139062143u;  // 127 (1 + 256 + ... + 256^{L-1})
    int v = x <= T ? (int)x : (int)(x - p);
#pragma unroll
    for (int l = 0; l < L; ++l) {
        const int d = l + 1 < L ? (int)(((uint32_t)v & 0xFFu) ^ 0x80u) - 0x80 : v;
        if (l + 1 < L) v = (v - d) >> 8;
        a[l] = __float_as_uint((float)d) >> 16;
    }
}

// the planes of 8 consecutive K values of one row: one 16-byte store per plane (dst 16-byte aligned)
template <int L>
__device__ __forceinline__ void put_digits8(const uint32_t (&x)[8], uint32_t p, uint16_t *dst, uint64_t plane) {
    uint32_t w[L][4];
#pragma unroll
    for (int i = 0; i < 8; i += 2) {
        uint32_t a[L], b[L];
        digits_of<L>(x[i], p, a);
        digits_of<L>(x[i + 1], p, b);
#pragma unroll
        for (int l = 0; l < L; ++l) w[l][i / 2] = a[l] | (b[l] << 16);
    }
#pragma unroll
    for (int l = 0; l < L; ++l)
        *reinterpret_cast<uint4 *>(dst + (size_t)l * plane) = make_uint4(w[l][0], w[l][1], w[l][2], w[l][3]);
}

template <int L>
__global__ void __launch_bounds__(MM_THREADS, 1) k_mm(const __grid_constant__ CUtensorMap ta,
                                                     const __grid_constant__ CUtensorMap tb,
                                                     const __grid_constant__ CUtensorMap tc, const MmParams P) {
    using Cfg = MmCfg<L>;
    constexpr int BN = Cfg::BN, CPT = Cfg::CPT;
    extern __shared__ unsigned char mm_smem_raw[];
    const uint32_t raw = smem_u32(mm_smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;  // 1024-byte aligned
    unsigned char *gbase = mm_smem_raw + (base - raw);
    // layout: A (all digits and K blocks of the row tile) | C tiles | ring of B^T slots | barriers
    const uint32_t sA = base, sC = base + Cfg::A_BYTES, sB = sC + Cfg::C_BYTES;
    const uint32_t bars = base + Cfg::SMEM_DATA;
    const uint32_t a_full = bars, a_empty = bars + 8;
    auto r_full = [&](int r) { return bars + 16 + 8u * r; };
    auto r_empty = [&](int r) { return bars + 32 + 8u * r; };
    auto c_full = [&](int c) { return bars + 48 + 8u * c; };
    auto b_full = [&](int s) { return bars + 80 + 8u * s; };
    auto b_empty = [&](int s) { return bars + 80 + 8u * Cfg::NSLOT + 8u * s; };
    const uint32_t tslot = bars + 80 + 16u * Cfg::NSLOT;
    uint32_t *tslot_g = reinterpret_cast<uint32_t *>(gbase + (tslot - base));
    // set when a bounded wait gives up: from then on every wait returns at once and no new copy,
    // product or store is issued, but every role still runs its whole loop, so the epilogue warps
    // keep meeting at their named barrier and the CTA reaches its teardown
    volatile uint32_t *abort_flag = reinterpret_cast<volatile uint32_t *>(gbase + (tslot + 4 - base));
    auto wait = [&](uint32_t bar, uint32_t parity) -> bool {
        if (*abort_flag) return false;
        if (mbar_wait(bar, parity)) return true;
        *abort_flag = 1u;
        atomicOr(P.err, 1u);
        return false;
    };

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t w0 = (uint32_t)((unsigned long long)blockIdx.x * P.items / gridDim.x);
    const uint32_t w1 = (uint32_t)((unsigned long long)(blockIdx.x + 1) * P.items / gridDim.x);
    const int nkb = (int)((P.K + MM_BK - 1) / MM_BK);
    // epilogue thread: row r of the tile is tensor-memory lane r; the WPG warps of an epilogue
    // group cover the four lane quarters WPG / 4 times, column group grp taking columns
    // CPT grp .. CPT grp + CPT - 1
    const int quarter = warp & 3, grp = ((warp - 2) % Cfg::WPG) >> 2;
    const uint32_t r = (uint32_t)(32 * quarter + lane);

    // a launch that follows this one in the stream may start as soon as this grid's CTAs leave
    // (programmatic dependent launch): it runs its prologue, then waits for this grid below
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (threadIdx.x == 0) {
        *abort_flag = 0u;
        mbar_init(a_full, 1);
        mbar_init(a_empty, 1);
        for (int i = 0; i < 2; ++i) {
            mbar_init(r_full(i), 1);
            mbar_init(r_empty(i), Cfg::WPG);  // one arrival per warp of the group that drains it
        }
        for (int c = 0; c < Cfg::NCBUF; ++c) mbar_init(c_full(c), 1);
        static_assert(Cfg::NCBUF <= 4, "barrier space");
        for (int s = 0; s < Cfg::NSLOT; ++s) {
            mbar_init(b_full(s), 1);
            mbar_init(b_empty(s), 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        tmem_alloc(tslot, Cfg::TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t *>(tslot_g);
    const uint32_t trow = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(CPT * grp);
    // Every product accumulates: the epilogue zeroes both accumulator sets here and each set again
    // right after draining it, so no product has to open a diagonal by overwriting it.
    if (warp >= 2) {
        const int eg = (warp - 2) / Cfg::WPG;
#pragma unroll
        for (int set = 0; set < 2; ++set)
            if (Cfg::EG == 1 || set == eg)  // with two groups, group g drains (and zeroes) set g
#pragma unroll
                for (int d = 0; d < Cfg::DIAG; ++d)
#pragma unroll
                    for (int h = 0; h < CPT / Cfg::DRAIN; ++h)
                        tmem_zero<Cfg::DRAIN>(trow + (uint32_t)set * Cfg::SET_COLS + (uint32_t)(BN * d + Cfg::DRAIN * h));
        tmem_wait_st();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // nothing above touches global memory: under a programmatic dependent launch the prologue
    // overlaps the previous grid, and the operands are read only once it has completed and its
    // writes are visible (without such a launch this returns at once)
    asm volatile("griddepcontrol.wait;" ::: "memory");

    if (warp == 0 && lane == 0) {
        // ---- producer.  K block kb of the it-th tile is the g-th block of the ring sequence,
        // g = it nkb + kb, in slot g mod NSLOT, that slot's (g / NSLOT)-th use.
        int arow = -1;
        uint32_t a_loads = 0, g = 0;
        for (uint32_t w = w0, it = 0; w < w1; ++w, ++it) {
            const int mt = (int)(w / P.ntn), nt = (int)(w % P.ntn);
            // the next tile's C goes to L2 now
            if (w + 1 < w1 && !*abort_flag) {
                const int mn = (int)((w + 1) / P.ntn), nn = (int)((w + 1) % P.ntn);
                for (int h = 0; h < Cfg::C_BOXES; ++h)
                    if ((uint32_t)nn * BN + 32u * h < P.N) tma_prefetch_2d(&tc, P.cx + nn * BN + 32 * h, P.cy + mn * MM_BM);
            }
            if (mt != arow) {
                if (!a_loads || wait(a_empty, (a_loads - 1) & 1u)) {
                    mbar_expect_tx(a_full, (uint32_t)(L * nkb) * Cfg::A_BLK);
                    for (int l = 0; l < L; ++l)
                        for (int kb = 0; kb < nkb; ++kb)
                            tma_load_3d(sA + (uint32_t)(l * Cfg::KB + kb) * Cfg::A_BLK, &ta, a_full,
                                        P.ax + kb * MM_BK, P.ay + mt * MM_BM, l);
                }
                ++a_loads;
                arow = mt;
            }
            for (int kb = 0; kb < nkb; ++kb, ++g) {
                const uint32_t s = g % Cfg::NSLOT, use = g / Cfg::NSLOT;
                if (wait(b_empty(s), (use & 1u) ^ 1u)) {
                    // one box of all L digit planes: the slot holds digit 0's BN rows, then digit 1's...
                    mbar_expect_tx(b_full(s), Cfg::B_BLK);
                    tma_load_3d(sB + s * Cfg::B_BLK, &tb, b_full(s), P.bx + kb * MM_BK, P.by + nt * BN, 0);
                }
            }
        }
    } else if (warp == 1) {
        // ---- MMA issuer: the whole warp runs the loop (warp-uniform descriptors), lane 0 issues.
        // For each K step of 16 and each A digit i, one M=128, N=128, K=16 product of A_i with all
        // L digits of B^T at once: its N columns are the products A_i B_j, j = 0..L-1, BN each,
        // and its accumulator window starts at diagonal i, so A_i B_j lands on diagonal i + j.
        // Every product accumulates into a set the epilogue has zeroed.
        int arow = -1;
        uint32_t a_loads = 0;
        const uint32_t a_lo = sdesc_lo(sA), b_lo = sdesc_lo(sB);
        for (uint32_t w = w0, it = 0; w < w1; ++w, ++it) {
            const int mt = (int)(w / P.ntn);
            if (mt != arow) {
                if (a_loads && lane == 0) mma_commit(a_empty);  // A is free once the earlier products are done
                wait(a_full, a_loads & 1u);
                ++a_loads;
                arow = mt;
            }
            const int set = (int)(it & 1u);
            const bool ok = __all_sync(0xffffffffu, wait(r_empty(set), ((it >> 1) & 1u) ^ 1u));
            tc_fence_after();
            const uint32_t tbase = tmem + (uint32_t)set * Cfg::SET_COLS;
#pragma unroll
            for (int kb = 0; kb < Cfg::KB; ++kb) {
                if (kb < nkb) {
                    const uint32_t g = it * (uint32_t)nkb + (uint32_t)kb;
                    const uint32_t s = g % Cfg::NSLOT;
                    const bool have = __all_sync(0xffffffffu, wait(b_full(s), (g / Cfg::NSLOT) & 1u)) && ok;
                    tc_fence_after();
                    if (have && !*abort_flag && lane == 0) {
                        // descriptor start addresses move in 16-byte units; apart from the slot's
                        // base every offset below is a compile-time constant
                        const uint32_t bs = b_lo + ((s * Cfg::B_BLK) >> 4);
#pragma unroll
                        for (int kk = 0; kk < MM_BK / 16; ++kk) {
#pragma unroll
                            for (int i = 0; i < L; ++i) {
                                const uint64_t ad = sdesc_of(a_lo + (((uint32_t)(i * Cfg::KB + kb) * Cfg::A_BLK + kk * 32) >> 4));
                                const uint32_t bd = bs + ((kk * 32) >> 4);
                                mma_bf16(tbase + (uint32_t)(BN * i), ad, sdesc_of(bd), idesc(MM_MMA_N), 1u);
                            }
                        }
                    }
                    __syncwarp();
                    if (lane == 0) mma_commit(b_empty(s));  // the slot may be refilled once these are done
                }
            }
            __syncwarp();
            if (lane == 0) mma_commit(r_full(set));  // the set's accumulators are ready
            __syncwarp();
        }
    } else if (warp >= 2) {
        // ---- epilogue.  EG groups of warps take alternate tiles (group eg the CTA's tiles
        // it = eg mod EG), so that one group drains a set while the other is still busy with the
        // C tile of the tile before.  In each group one thread (the storer) also moves C: it
        // loads the C tile of the group's next tile into the group's buffer as soon as the store
        // that last used the buffer has read it, so the producer's stream of B blocks never waits
        // on the epilogue.
        const int eg = (warp - 2) / Cfg::WPG;
        const bool storer = (warp - 2) % Cfg::WPG == 0 && lane == 0;
        auto load_c = [&](uint32_t itc) {  // C tile of the CTA's itc-th tile into buffer itc mod NCBUF
            const uint32_t wc = w0 + itc;
            if (wc >= w1 || *abort_flag) return;
            const int mc = (int)(wc / P.ntn), nc = (int)(wc % P.ntn);
            const int boxes = Cfg::C_BOXES == 2 && P.N - (uint32_t)nc * BN > 32u ? 2 : 1;
            const uint32_t cbuf = itc % Cfg::NCBUF;
            mbar_expect_tx(c_full(cbuf), (uint32_t)boxes * Cfg::C_BOX);
            for (int h = 0; h < boxes; ++h)
                tma_load_2d(sC + cbuf * Cfg::C_TILE + (uint32_t)h * Cfg::C_BOX, &tc, c_full(cbuf), P.cx + nc * BN + 32 * h,
                            P.cy + mc * MM_BM);
        };
        if (storer) {
            if (Cfg::EG == 1)
                for (uint32_t i = 0; i < (uint32_t)Cfg::NCBUF; ++i) load_c(i);
            else
                load_c((uint32_t)eg);
        }
        const uint32_t col0 = (uint32_t)(CPT * grp);                // first column in the tile
        const uint32_t box = col0 / 32, chunk0 = (col0 % 32) / 4;  // its 32-column box, 16-byte chunk
        const Fp fp = P.fp;
        for (uint32_t w = w0 + (uint32_t)eg, it = (uint32_t)eg; w < w1; w += Cfg::EG, it += Cfg::EG) {
            const int mt = (int)(w / P.ntn), nt = (int)(w % P.ntn);
            const int set = (int)(it & 1u);
            // value = sum_d D_d 256^d (mod p).  rd[d] = (-/+ 256^d) 2^32 mod p in [0, p), the sign
            // that of the update, so acc = big + sum D_d rd[d] is -/+ value 2^32 (mod p), and one
            // Montgomery reduction of acc (big = 2^31 p) gives -/+ value.  Adjacent diagonals pair
            // up in 32 bits first:
            //   L = 4 (K <= 128): E_0 = D_0 + 256 D_1, |E_0| <= 2^21 + 2^30; E_5 = D_5 + 256 D_6,
            //                     |E_5| <= 2^22 + 2^29; acc = big + E_0 rd0 + D_2 rd2 + D_3 rd3
            //                     + D_4 rd4 + E_5 rd5, |acc - big| < p (2^30 + 2^29 + 2^25);
            //   L = 2 (K <= 256): E_1 = D_1 + 256 D_2, |E_1| <= 2^23 + 2^30; acc = big + D_0 rd0
            //                     + E_1 rd1, |acc - big| < p (2^30 + 2^24).
            // So 0 < acc < 2^32 p, the range of the reduction, whose result u (in [0, 2p)) is
            // brought to [0, p) by "u - p if u >= p", min(u, u - p) in unsigned arithmetic.  Every
            // product is signed 32 x 32 -> 64 bits (rd < p < 2^31).
            uint32_t u[CPT];
            wait(r_full(set), (it >> 1) & 1u);
            tc_fence_after();
            const uint32_t tb = trow + (uint32_t)set * Cfg::SET_COLS;
#pragma unroll
            for (int h = 0; h < CPT / Cfg::DRAIN; ++h) {
                // every diagonal's load of DRAIN columns in flight at once, one wait: the drain pays
                // one tensor-memory latency per DRAIN columns instead of one per diagonal
                constexpr int NW = Cfg::DRAIN;
                uint32_t v[Cfg::DIAG][NW];
#pragma unroll
                for (int d = 0; d < Cfg::DIAG; ++d) tmem_ld<NW>(tb + (uint32_t)(BN * d + NW * h), v[d]);
                tmem_wait_ld();
#pragma unroll
                for (int d = 0; d < Cfg::DIAG; ++d) tmem_zero<NW>(tb + (uint32_t)(BN * d + NW * h));
                const long long big = (long long)P.big;
#pragma unroll
                for (int j = 0; j < NW; ++j) {
                    long long acc;
                    if constexpr (L == 4) {
                        static_assert(small_diag<4>(0) && small_diag<4>(1) && small_diag<4>(5) && small_diag<4>(6),
                                      "paired diagonals");
                        acc = big + (long long)acc_pair_small(v[0][j], v[1][j]) * (int)P.rd[0] +
                              (long long)acc_int(v[2][j]) * (int)P.rd[2] + (long long)acc_int(v[3][j]) * (int)P.rd[3] +
                              (long long)acc_int(v[4][j]) * (int)P.rd[4] +
                              (long long)acc_pair_small(v[5][j], v[6][j]) * (int)P.rd[5];
                    } else {
                        static_assert(L == 2 && small_diag<2>(0) && small_diag<2>(2), "paired diagonals");
                        // E_1 = D_1 + 256 D_2: D_1 is converted exactly, D_2 through the bias
                        const int e1 = acc_int(v[1][j]) + 256 * acc_int_small(v[2][j]);
                        acc = big + (long long)acc_int_small(v[0][j]) * (int)P.rd[0] + (long long)e1 * (int)P.rd[1];
                    }
                    const uint64_t t = (uint64_t)acc;
                    const uint32_t m = (uint32_t)t * fp.pinv_neg;
                    const uint32_t x = (uint32_t)((t + (uint64_t)m * fp.p) >> 32);
                    u[NW * h + j] = min(x, x - fp.p);
                }
            }
            // the set is drained and zeroed: hand it back
            tmem_wait_st();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(r_empty(set));
            if (Cfg::EG == 1 && Cfg::NCBUF >= 2 && storer && it > 0) {
                bulk_wait_read0();  // the previous tile's store has read its buffer: a later tile's C
                load_c(it + Cfg::NCBUF - 1);
            }
            const uint32_t cb = it % Cfg::NCBUF;
            const bool have_c = wait(c_full(cb), (it / Cfg::NCBUF) & 1u);
            // row r of the thread's box: 128 bytes, 16-byte chunk j at chunk position j ^ (r mod 8)
            unsigned char *crow = gbase + (sC - base) + cb * Cfg::C_TILE + box * Cfg::C_BOX + r * 128u;
            if (have_c) {
#pragma unroll
                for (int jj = 0; jj < CPT / 4; ++jj) {
                    const uint32_t j = chunk0 + (uint32_t)jj;
                    uint4 *q = reinterpret_cast<uint4 *>(crow + 16u * (j ^ (r & 7u)));
                    uint4 c = *q;
                    uint32_t *cw = reinterpret_cast<uint32_t *>(&c);
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const uint32_t s = cw[e] + u[4 * jj + e];  // C -/+ value, both in [0, p)
                        cw[e] = min(s, s - fp.p);
                    }
                    *q = c;
                }
                // the digit planes of the first dig_cols columns, from the updated entries just
                // written (a thread's CPT columns are all in or all out: dig_cols is a multiple of 16)
                const uint32_t dc = (uint32_t)nt * BN + col0, dr = (uint32_t)mt * MM_BM + r;
                if (dc < P.dig_cols && dr < P.M) {
                    uint16_t *dst = P.dig + (size_t)dr * P.dig_kpad + dc;
#pragma unroll 1
                    for (int q8 = 0; q8 < CPT / 8; ++q8) {
                        const uint32_t j = chunk0 + 2u * (uint32_t)q8;
                        const uint4 a = *reinterpret_cast<const uint4 *>(crow + 16u * (j ^ (r & 7u)));
                        const uint4 b = *reinterpret_cast<const uint4 *>(crow + 16u * ((j + 1) ^ (r & 7u)));
                        const uint32_t x8[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
                        put_digits8<L>(x8, fp.p, dst + 8 * q8, P.dig_plane);
                    }
                }
            }
            fence_async_smem();
            epi_sync<32 * Cfg::WPG>(eg);
            if (storer) {
                const int boxes = Cfg::C_BOXES == 2 && P.N - (uint32_t)nt * BN > 32u ? 2 : 1;
                if (!*abort_flag)
                    for (int h = 0; h < boxes; ++h)
                        tma_store_2d(&tc, sC + cb * Cfg::C_TILE + (uint32_t)h * Cfg::C_BOX, P.cx + nt * BN + 32 * h,
                                     P.cy + mt * MM_BM);
                bulk_commit();
                if (Cfg::EG == 2 || Cfg::NCBUF == 1) {
                    bulk_wait_read0();  // the buffer is free again: the group's next C tile
                    load_c(it + Cfg::EG);
                }
            }
        }
        if (storer) bulk_wait_all();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem, Cfg::TMEM_COLS);
    }
}

// rows of a row-major source (src[r * rs + k]): thread per (row, 8 K values), the whole padded
// row written (zeros past K); the loads are 16-byte vectors when vec (rs % 4 == 0, src 16-byte
// aligned)
template <int L>
__global__ void k_digits(const uint32_t *__restrict__ src, uint64_t rs, uint32_t R, uint32_t K,
                         uint16_t *__restrict__ dst, uint64_t kpad, uint64_t plane, uint32_t p, int vec) {
    const uint64_t groups = kpad / 8, total = (uint64_t)R * groups;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t r = (uint32_t)(t / groups), k0 = (uint32_t)(t % groups) * 8u;
        const uint32_t *row = src + (size_t)r * rs;
        uint32_t x[8];
        if (vec && k0 + 8 <= K) {
            const uint4 a = *reinterpret_cast<const uint4 *>(row + k0), b = *reinterpret_cast<const uint4 *>(row + k0 + 4);
            x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w; x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
        } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) x[i] = k0 + i < K ? row[k0 + i] : 0u;
        }
        put_digits8<L>(x, p, dst + (size_t)r * kpad + k0, plane);
    }
}

// The same planes when the source is row-major in K (src[k * ks + r], the columns of B as rows of
// B^T): 64 x 64 tiles through shared memory, read along r and written along k, 8 K values (16
// bytes per plane) a thread, a warp covering four rows' 128-byte segments.  The whole padded row
// is written (zeros past K).
template <int L>
__global__ void k_digits_t(const uint32_t *__restrict__ src, uint64_t ks, uint32_t R, uint32_t K,
                           uint16_t *__restrict__ dst, uint64_t kpad, uint64_t plane, uint32_t p) {
    __shared__ uint32_t tile[64][65];
    const uint32_t r0 = blockIdx.x * 64, k0 = blockIdx.y * 64;
    for (uint32_t i = threadIdx.x; i < 64 * 64; i += blockDim.x) {
        const uint32_t kk = i / 64, rr = i % 64, k = k0 + kk, r = r0 + rr;
        tile[kk][rr] = (k < K && r < R) ? src[(size_t)k * ks + r] : 0u;
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < 64 * 8; i += blockDim.x) {
        const uint32_t rr = i / 8, kg = i % 8, r = r0 + rr;
        if (r >= R || k0 + 8 * kg >= kpad) continue;
        uint32_t x[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = tile[8 * kg + j][rr];
        put_digits8<L>(x, p, dst + (size_t)r * kpad + k0 + 8 * kg, plane);
    }
}

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_tiled() {
    static EncodeTiled fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        GB_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q));
        if (q != cudaDriverEntryPointSuccess || !f) fail(GB_EDEVICE, "cuTensorMapEncodeTiled is not available");
        return reinterpret_cast<EncodeTiled>(f);
    }();
    return fn;
}

void encode(CUtensorMap *m, CUtensorMapDataType t, cuuint32_t rank, void *base, const cuuint64_t *dims,
            const cuuint64_t *strides, const cuuint32_t *box) {
    std::memset(m, 0, sizeof(*m));
    const cuuint32_t es[3] = {1, 1, 1};
    const CUresult r = encode_tiled()(m, t, rank, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                      CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) fail(GB_EDEVICE, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
}

// digit planes [L][rows][kpad] (BF16), box of 64 K values x box_rows rows x 1 digit
CUtensorMap digit_map(const DigitPlanes &D, uint32_t box_rows, uint32_t box_digits) {
    if (D.kpad % 8 || (reinterpret_cast<uintptr_t>(D.p) & 15))
        fail(GB_EDEVICE, "digit planes: row pitch or base not 16-byte aligned");
    CUtensorMap m;
    const cuuint64_t dims[3] = {D.K, D.rows, D.L};
    const cuuint64_t strides[2] = {2ull * D.kpad, 2ull * D.kpad * D.rows};
    const cuuint32_t box[3] = {(cuuint32_t)MM_BK, box_rows, box_digits};
    encode(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, D.p, dims, strides, box);
    return m;
}

}  // namespace

int sm_count() {
    static int n[64] = {};
    int dev = 0;
    GB_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) fail(GB_EUNSUPPORTED, "device ordinal above 63");
    if (!n[dev]) GB_CUDA(cudaDeviceGetAttribute(&n[dev], cudaDevAttrMultiProcessorCount, dev));
    return n[dev];
}

uint32_t digits_for(uint32_t p) { return p < 65536u ? 2u : 4u; }
uint32_t mm_kmax(uint32_t p) { return 512u / digits_for(p); }

void DigitPlanes::alloc(Arena &ar, uint32_t L_, uint64_t rows_, uint64_t K_, cudaStream_t st) {
    L = L_;
    rows = rows_;
    K = K_;
    kpad = (K + 63) / 64 * 64;
    buf.alloc(ar, (size_t)L * rows * kpad, st);
    p = buf.p;
}

void to_digits(const uint32_t *src, uint64_t rs, uint64_t ks, const DigitPlanes &D, uint32_t p, cudaStream_t st) {
    if (!D.rows || !D.K) return;
    const uint64_t plane = D.rows * D.kpad;
    if (rs == 1 && ks != 1) {  // K-strided source: transpose through shared memory
        if ((D.kpad + 63) / 64 > 65535u) fail(GB_EUNSUPPORTED, "digit planes: K too large for one launch");
        const dim3 grid((unsigned)((D.rows + 63) / 64), (unsigned)((D.kpad + 63) / 64));
        if (D.L == 2) k_digits_t<2><<<grid, 256, 0, st>>>(src, ks, (uint32_t)D.rows, (uint32_t)D.K, D.p, D.kpad, plane, p);
        else k_digits_t<4><<<grid, 256, 0, st>>>(src, ks, (uint32_t)D.rows, (uint32_t)D.K, D.p, D.kpad, plane, p);
        counted();
        return;
    }
    if (ks != 1) fail(GB_EUNSUPPORTED, "digit planes: the source must be contiguous in K or in rows");
    const int vec = rs % 4 == 0 && (reinterpret_cast<uintptr_t>(src) & 15) == 0;
    const uint64_t items = D.rows * (D.kpad / 8);
    const unsigned grid = (unsigned)std::min<uint64_t>((items + 255) / 256, 65535u * 16u);
    if (D.L == 2) k_digits<2><<<grid, 256, 0, st>>>(src, rs, (uint32_t)D.rows, (uint32_t)D.K, D.p, D.kpad, plane, p, vec);
    else k_digits<4><<<grid, 256, 0, st>>>(src, rs, (uint32_t)D.rows, (uint32_t)D.K, D.p, D.kpad, plane, p, vec);
    counted();
}

// Tensor maps of one operand set (A digit planes, B^T digit planes, C) for any number of
// updates over sub-ranges of them: the maps are encoded once, each launch passes its offsets.
struct MmPlan::Maps {
    CUtensorMap ta, tb, tc;
};

// One k_mm launch.  With pdl (and outside stream capture) it is a programmatic dependent launch:
// it may begin (its prologue: barriers, tensor memory, the zeroing of the accumulators) while the
// previous kernel of the stream finishes, and waits for that kernel (griddepcontrol.wait) before
// its first global access.  Otherwise it is an ordinary launch.
template <int L>
void launch_mm(unsigned grid, cudaStream_t st, const CUtensorMap &ta, const CUtensorMap &tb, const CUtensorMap &tc,
               const MmParams &P, bool pdl) {
    opt_in_smem(reinterpret_cast<const void *>(k_mm<L>));
    if (!pdl || t_capturing) {
        k_mm<L><<<grid, MM_THREADS, MmCfg<L>::SMEM, st>>>(ta, tb, tc, P);
        return;
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(MM_THREADS);
    cfg.dynamicSmemBytes = MmCfg<L>::SMEM;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    GB_CUDA(cudaLaunchKernelEx(&cfg, k_mm<L>, ta, tb, tc, P));
}

MmPlan::MmPlan(const DigitPlanes &A_, const DigitPlanes &B_, uint32_t *C_, uint64_t ldc_, uint32_t crows,
               uint32_t ccols, const Fp &fp_)
    : A(&A_), B(&B_), C(C_), ldc(ldc_), rows(crows), cols(ccols), fp(fp_), maps(new Maps) {
    const uint32_t L = digits_for(fp.p);
    if (A->L != L || B->L != L) fail(GB_EDEVICE, "mm plan: digit count does not match p");
    if (ldc % 4 || (reinterpret_cast<uintptr_t>(C) & 15)) fail(GB_EDEVICE, "mm plan: C rows not 16-byte aligned");
    maps->ta = digit_map(*A, MM_BM, 1);
    maps->tb = digit_map(*B, MM_MMA_N / L, L);  // all digits of a tile's rows in one box
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {4ull * ldc};
    const cuuint32_t box[2] = {32u, (cuuint32_t)MM_BM};  // 128 bytes: the 128-byte swizzle span
    encode(&maps->tc, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, C, dims, strides, box);
    // raised here, before any launch, so that launches recorded into a graph find it set
    opt_in_smem(L == 2 ? reinterpret_cast<const void *>(k_mm<2>) : reinterpret_cast<const void *>(k_mm<4>));
}

MmPlan::~MmPlan() { delete maps; }

// C[cy + m][cx + n] <- C -/+ sum_k A[ay + m][ax + k] B^T[by + n][bx + k] mod p for m < M, n < N,
// k < K <= mm_kmax(p).  A ragged last tile of the update region (N not a multiple of the tile
// width, M not a multiple of 128) must end the C tensor of the plan on that side, where the TMA
// store clips it; cx must be a multiple of 4.
void MmPlan::update(uint32_t ax, uint32_t ay, uint32_t bx, uint32_t by, uint32_t cx, uint32_t cy, uint32_t M,
                    uint32_t N, uint32_t K, bool sub, uint32_t *err, cudaStream_t st, const DigitPlanes *dig,
                    uint32_t dig_cols, bool pdl) const {
    if (!M || !N || !K) return;
    if (K > mm_kmax(fp.p)) fail(GB_EDEVICE, "mm_update: K above the exact accumulation bound");
    if (ax % 8 || bx % 8) fail(GB_EDEVICE, "mm_update: K offsets must be multiples of 8 (16-byte TMA rule)");
    // the kernel reads whole 64-wide K blocks: a ragged K must end where one operand's planes end
    // (the TMA fills the rest of that operand's block with zeros, so the other operand's extra
    // values, which must be finite, multiply zeros)
    if (K % MM_BK && ax + K != A->K && bx + K != B->K) fail(GB_EDEVICE, "mm_update: ragged K inside both planes");
    if (ax + K > A->K || bx + K > B->K || ay + M > A->rows || by + N > B->rows)
        fail(GB_EDEVICE, "mm_update: operand range outside the digit planes");
    const uint32_t bn = MM_MMA_N / A->L;
    if (cx % 4 || cx + N > cols || cy + M > rows || (N % bn && cx + N != cols) || (M % MM_BM && cy + M != rows))
        fail(GB_EDEVICE, "mm_update: a ragged C region does not end the tensor");
    MmParams P{};
    P.M = M;
    P.N = N;
    P.K = K;
    P.ax = (int)ax;
    P.ay = (int)ay;
    P.bx = (int)bx;
    P.by = (int)by;
    P.cx = (int)cx;
    P.cy = (int)cy;
    P.ntn = (N + bn - 1) / bn;
    const uint64_t items = (uint64_t)((M + MM_BM - 1) / MM_BM) * P.ntn;
    if (items >= (1ull << 31)) fail(GB_EUNSUPPORTED, "mm_update: too many tiles for one launch");
    P.items = (uint32_t)items;
    P.fp = fp;
    P.big = (uint64_t)fp.p << 31;
    for (uint32_t d = 0, x = 1; d < 7; ++d, x = (uint32_t)((uint64_t)x * 256 % fp.p)) {
        const uint32_t y = sub && x ? fp.p - x : x;     // -/+ 256^d mod p
        P.rd[d] = (uint32_t)(((uint64_t)y << 32) % fp.p);  // in Montgomery form
    }
    P.err = err;
    if (dig && dig_cols) {
        if (dig->L != A->L || dig->rows < M || dig_cols % 16 || dig_cols > N || dig_cols > dig->kpad)
            fail(GB_EDEVICE, "mm_update: digit planes of the result do not fit");
        P.dig = dig->p;
        P.dig_kpad = dig->kpad;
        P.dig_plane = dig->rows * dig->kpad;
        P.dig_cols = dig_cols;
    }
    const unsigned grid = (unsigned)std::min<uint64_t>(items, (uint64_t)sm_count());
    MmTimer *T = t_capturing ? nullptr : t_mm_timer;
    cudaEvent_t e1 = nullptr;
    if (T) {
        if (!T->span_end) {
            std::vector<cudaEvent_t> &pool = T->ctx->mm_ev;
            while (pool.size() < T->used + 2) {
                cudaEvent_t e;
                GB_CUDA(cudaEventCreate(&e));
                pool.push_back(e);
            }
            GB_CUDA(cudaEventRecord(pool[T->used], st));
            e1 = pool[T->used + 1];
            T->used += 2;
        }
        T->flops += 2.0 * A->L * A->L * (double)M * N * K;
        T->launches++;
    }
    if (A->L == 2) launch_mm<2>(grid, st, maps->ta, maps->tb, maps->tc, P, pdl);
    else launch_mm<4>(grid, st, maps->ta, maps->tb, maps->tc, P, pdl);
    counted();
    if (e1) GB_CUDA(cudaEventRecord(e1, st));
}

thread_local MmTimer *t_mm_timer = nullptr;

void matmul_dev(Arena &ar, const Fp &fp, uint32_t m, uint32_t n, uint32_t k, const uint32_t *A, uint64_t lda,
                const uint32_t *B, uint64_t ldb, uint32_t *C, uint64_t ldc, bool subtract, uint32_t *err,
                cudaStream_t st) {
    if (!m || !n || !k) return;
    const uint32_t L = digits_for(fp.p);
    DigitPlanes DA, DB;
    DA.alloc(ar, L, m, k, st);
    DB.alloc(ar, L, n, k, st);
    to_digits(A, lda, 1, DA, fp.p, st);
    to_digits(B, 1, ldb, DB, fp.p, st);  // B^T: row j holds column j of B
    // the kernel moves C tiles by TMA: rows must start on 16-byte boundaries, else C is staged
    DBuf<uint32_t> Cs;
    uint32_t *Cw = C;
    uint64_t ldw = ldc;
    if (ldc % 4 || (reinterpret_cast<uintptr_t>(C) & 15)) {
        ldw = (n + 3) / 4 * 4;
        Cs.alloc(ar, (size_t)m * ldw, st);
        Cw = Cs.p;
        GB_CUDA(cudaMemcpy2DAsync(Cw, 4 * ldw, C, 4 * ldc, 4ull * n, m, cudaMemcpyDeviceToDevice, st));
    }
    const uint32_t kmax = mm_kmax(fp.p);
    const MmPlan plan(DA, DB, Cw, ldw, m, n, fp);
    for (uint32_t k0 = 0; k0 < k; k0 += kmax)
        plan.update(k0, 0, k0, 0, 0, 0, m, n, std::min(kmax, k - k0), subtract, err, st, nullptr, 0, true);
    if (Cw != C) GB_CUDA(cudaMemcpy2DAsync(C, 4 * ldc, Cw, 4 * ldw, 4ull * n, m, cudaMemcpyDeviceToDevice, st));
}

void MmTimer::begin_span(cudaStream_t st) {
    if (t_capturing || span_end) return;
    std::vector<cudaEvent_t> &pool = ctx->mm_ev;
    while (pool.size() < used + 2) {
        cudaEvent_t e;
        GB_CUDA(cudaEventCreate(&e));
        pool.push_back(e);
    }
    GB_CUDA(cudaEventRecord(pool[used], st));
    span_end = pool[used + 1];
    used += 2;
}

void MmTimer::end_span(cudaStream_t st) {
    if (!span_end) return;
    GB_CUDA(cudaEventRecord(span_end, st));
    span_end = nullptr;
}

double MmTimer::elapsed_ms() const {
    double ms = 0.0;
    for (size_t i = 0; i + 1 < used; i += 2) {
        float x = 0.f;
        GB_CUDA(cudaEventElapsedTime(&x, ctx->mm_ev[i], ctx->mm_ev[i + 1]));
        ms += x;
    }
    return ms;
}

}  // namespace gb
