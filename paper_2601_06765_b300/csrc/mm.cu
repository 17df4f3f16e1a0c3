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
// so every partial sum is an integer the FP32 accumulator holds exactly (with a bit to spare).  The epilogue converts
// each D_s to an integer and forms sum_s D_s 256^s mod p (Horner, one Barrett reduction per
// digit), which equals (A B)[m][n] mod p.  One launch covers K <= 512 / L; longer products are
// split by the host into launches that each update C.
//
// Kernel (one 128 x 64 tile of C per CTA, 6 warps):
//   warp 0, lane 0   TMA producer: digit planes of A (128 x 64 per digit) and B^T (64 x 64 per
//                    digit) for each 64-wide K block into a ring of shared-memory stages
//                    (128-byte swizzle), mbarrier with transaction count
//   warp 1           allocates the tensor memory; lane 0 issues tcgen05.mma (kind::f16, BF16
//                    operands, FP32 accumulators, M = 128, N = 64, K = 16) for every digit pair
//                    into the accumulator of its diagonal, and commits to the stage's "empty"
//                    barrier and finally to the "accumulators full" barrier
//   warps 2-5        epilogue: tcgen05.ld of the thread's row of every diagonal, exact
//                    conversion, Horner mod p, read-modify-write of C
// Every wait is bounded; a wait that gives up sets an error flag that the host turns into
// GB_ETIMEOUT, and the CTA still releases its tensor memory.
#include <cuda.h>

#include <algorithm>
#include <cstring>

#include "internal.hpp"

namespace gb {

namespace {

constexpr int MM_BM = 128, MM_BN = 64, MM_BK = 64;  // tile of C, K block (64 BF16 = 128 bytes)
constexpr int MM_THREADS = 192;
constexpr uint32_t MM_SPIN = 1u << 22;               // bounded mbarrier waits

template <int L>
struct MmCfg {
    static constexpr int DIAG = 2 * L - 1;                              // digit diagonals
    static constexpr uint32_t A_TILE = MM_BM * MM_BK * 2;               // bytes per digit
    static constexpr uint32_t B_TILE = MM_BN * MM_BK * 2;
    static constexpr uint32_t STAGE = L * (A_TILE + B_TILE);
    static constexpr int STAGES = L == 2 ? 4 : 2;
    static constexpr uint32_t TMEM_COLS = DIAG * MM_BN <= 256 ? 256 : 512;
    static constexpr uint32_t SMEM = STAGES * STAGE + 1024 + 256;       // + alignment + barriers
};

struct MmParams {
    uint32_t M, N, K;       // C is M x N; the product runs over K
    int ax, ay, bx, by;     // TMA coordinates of the first K block of A (k, m) and of B^T (k, n)
    uint32_t *C;            // element (m, n) at C[m * ldc + n]
    uint64_t ldc;
    Fp fp;
    uint64_t big;           // a multiple of p above 2^48, added before each Barrett reduction
    int sub;                // 1: C -= A B, 0: C += A B
    uint32_t *err;          // bit 0: a bounded wait gave up
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
// 16 consecutive 32-bit columns of this thread's tensor-memory lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major tile with 128-byte swizzle: rows of 128 bytes,
// 8-row groups 1024 bytes apart (stride byte offset), descriptor version 1, layout type 2.
// The tile base is 1024-byte aligned; a K offset inside the 128-byte row moves the start address.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A and B (bits 7-9,
// 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(MM_BN >> 3) << 17) |
                           ((uint32_t)(MM_BM >> 4) << 24);

// signed value (|x| < 2^62 - big) mod p
__device__ __forceinline__ uint32_t mod_signed(long long x, const MmParams &P) {
    return fp_reduce((uint64_t)(x + (long long)P.big), P.fp);
}

template <int L>
__global__ void __launch_bounds__(MM_THREADS, 1) k_mm(const __grid_constant__ CUtensorMap ta,
                                                     const __grid_constant__ CUtensorMap tb, const MmParams P) {
    using Cfg = MmCfg<L>;
    extern __shared__ unsigned char mm_smem_raw[];
    const uint32_t raw = smem_u32(mm_smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;  // stage buffers, 1024-byte aligned
    unsigned char *gbase = mm_smem_raw + (base - raw);
    const uint32_t bars = base + Cfg::STAGES * Cfg::STAGE;  // full[S], empty[S], accfull, tmem slot
    auto full = [&](int s) { return bars + 8u * s; };
    auto empty = [&](int s) { return bars + 8u * (Cfg::STAGES + s); };
    const uint32_t accfull = bars + 8u * (2 * Cfg::STAGES);
    const uint32_t tslot = accfull + 8u;
    uint32_t *tslot_g = reinterpret_cast<uint32_t *>(gbase + (tslot - base));

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t m0 = blockIdx.y * MM_BM, n0 = blockIdx.x * MM_BN;
    const int nkb = (int)((P.K + MM_BK - 1) / MM_BK);

    if (threadIdx.x == 0) {
        for (int s = 0; s < Cfg::STAGES; ++s) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        mbar_init(accfull, 1);
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

    if (warp == 0 && lane == 0) {
        // producer
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % Cfg::STAGES;
            const uint32_t ph = (uint32_t)(kb / Cfg::STAGES) & 1u;
            if (!mbar_wait(empty(s), ph ^ 1u)) {
                atomicOr(P.err, 1u);
                break;
            }
            const uint32_t st = base + s * Cfg::STAGE;
            mbar_expect_tx(full(s), Cfg::STAGE);
            for (int l = 0; l < L; ++l) {
                tma_load_3d(st + l * Cfg::A_TILE, &ta, full(s), P.ax + kb * MM_BK, P.ay + (int)m0, l);
                tma_load_3d(st + L * Cfg::A_TILE + l * Cfg::B_TILE, &tb, full(s), P.bx + kb * MM_BK, P.by + (int)n0, l);
            }
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        uint32_t started = 0;  // diagonals written at least once
        bool ok = true;
        for (int kb = 0; kb < nkb && ok; ++kb) {
            const int s = kb % Cfg::STAGES;
            const uint32_t ph = (uint32_t)(kb / Cfg::STAGES) & 1u;
            if (!mbar_wait(full(s), ph)) {
                atomicOr(P.err, 1u);
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t st = base + s * Cfg::STAGE;
#pragma unroll
            for (int kk = 0; kk < MM_BK / 16; ++kk) {
#pragma unroll
                for (int i = 0; i < L; ++i) {
#pragma unroll
                    for (int j = 0; j < L; ++j) {
                        const int d = i + j;
                        const uint64_t ad = sdesc(st + i * Cfg::A_TILE + kk * 32);
                        const uint64_t bd = sdesc(st + L * Cfg::A_TILE + j * Cfg::B_TILE + kk * 32);
                        mma_bf16(tmem + (uint32_t)(d * MM_BN), ad, bd, IDESC, (started >> d) & 1u);
                        started |= 1u << d;
                    }
                }
            }
            mma_commit(empty(s));  // the stage is free once these products are done
        }
        mma_commit(accfull);
    } else if (warp >= 2) {
        // epilogue: row r of the tile is tensor-memory lane r
        const int sub = warp & 3;
        const uint32_t r = (uint32_t)(32 * sub + lane);
        const uint32_t m = m0 + r;
        const bool ok = mbar_wait(accfull, 0);
        if (!ok && lane == 0) atomicOr(P.err, 1u);
        tc_fence_after();
        const uint32_t trow = tmem + ((uint32_t)(32 * sub) << 16);
#pragma unroll 1
        for (int g = 0; g < MM_BN / 16; ++g) {
            uint32_t acc[16];
            uint32_t v[16];
            // Horner over the diagonals, highest first
            tmem_ld16(trow + (uint32_t)((Cfg::DIAG - 1) * MM_BN + 16 * g), v);
            tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[j] = mod_signed((long long)__float2int_rn(__uint_as_float(v[j])), P);
#pragma unroll 1
            for (int d = Cfg::DIAG - 2; d >= 0; --d) {
                tmem_ld16(trow + (uint32_t)(d * MM_BN + 16 * g), v);
                tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    acc[j] = mod_signed(((long long)acc[j] << 8) + (long long)__float2int_rn(__uint_as_float(v[j])), P);
            }
            if (ok && m < P.M) {
                uint32_t *crow = P.C + (size_t)m * P.ldc;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const uint32_t n = n0 + 16 * g + j;
                    if (n < P.N) {
                        const uint32_t c = crow[n], s = acc[j];
                        crow[n] = P.sub ? (c >= s ? c - s : c + P.fp.p - s) : fp_add(c, s, P.fp);
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem, Cfg::TMEM_COLS);
    }
}

// Digit planes: dst[l][r][k] (row pitch kpad, plane pitch rows * kpad) = BF16 bits of the l-th
// balanced base-256 digit of the residue at src[r * rs + k * ks], for r < R, k < K.
template <int L>
__global__ void k_digits(const uint32_t *__restrict__ src, uint64_t rs, uint64_t ks, uint32_t R, uint32_t K,
                         uint16_t *__restrict__ dst, uint64_t kpad, uint64_t plane, uint32_t p) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    for (uint32_t r = blockIdx.y; r < R; r += gridDim.y) {
        const uint32_t x = src[(size_t)r * rs + (size_t)k * ks];
        const uint32_t T = L == 2 ? 32639u : 2139062143u;  // 127 (1 + 256 + ... + 256^{L-1})
        int v = x <= T ? (int)x : (int)(x - p);
#pragma unroll
        for (int l = 0; l < L; ++l) {
            const int a = l + 1 < L ? (int)(((uint32_t)v & 0xFFu) ^ 0x80u) - 0x80 : v;
            if (l + 1 < L) v = (v - a) >> 8;
            dst[(size_t)l * plane + (size_t)r * kpad + k] = (uint16_t)(__float_as_uint((float)a) >> 16);
        }
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

}  // namespace

uint32_t digits_for(uint32_t p) { return p < 65536u ? 2u : 4u; }
uint32_t mm_kmax(uint32_t p) { return 512u / digits_for(p); }

// Tensor map of digit planes [L][rows][kpad] (BF16), box of 64 K values x box_rows rows x 1 digit.
CUtensorMap digit_map(const DigitPlanes &D, uint32_t box_rows) {
    if (D.kpad % 8 || (reinterpret_cast<uintptr_t>(D.p) & 15))
        fail(GB_EDEVICE, "digit planes: row pitch or base not 16-byte aligned");
    CUtensorMap m;
    std::memset(&m, 0, sizeof(m));
    const cuuint64_t dims[3] = {D.K, D.rows, D.L};
    const cuuint64_t strides[2] = {2ull * D.kpad, 2ull * D.kpad * D.rows};
    const cuuint32_t box[3] = {(cuuint32_t)MM_BK, box_rows, 1};
    const cuuint32_t es[3] = {1, 1, 1};
    const CUresult r = encode_tiled()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, D.p, dims, strides, box, es,
                                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) fail(GB_EDEVICE, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
    return m;
}

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
    const dim3 grid((unsigned)((D.K + 255) / 256), (unsigned)std::min<uint64_t>(D.rows, 65535));
    const uint64_t plane = D.rows * D.kpad;
    if (D.L == 2) k_digits<2><<<grid, 256, 0, st>>>(src, rs, ks, (uint32_t)D.rows, (uint32_t)D.K, D.p, D.kpad, plane, p);
    else k_digits<4><<<grid, 256, 0, st>>>(src, rs, ks, (uint32_t)D.rows, (uint32_t)D.K, D.p, D.kpad, plane, p);
    counted();
}

// C[M x N] (row pitch ldc) <- C -/+ A B mod p, A given by digit planes of A (rows m, K-major,
// starting at row ay and K offset ax), B by digit planes of B^T (rows n, K-major, starting at row
// by and K offset bx); K <= mm_kmax(p).  err: a device word that collects the error flags.
void mm_update(const DigitPlanes &A, uint32_t ax, uint32_t ay, const DigitPlanes &B, uint32_t bx, uint32_t by,
               uint32_t M, uint32_t N, uint32_t K, uint32_t *C, uint64_t ldc, const Fp &fp, bool sub, uint32_t *err,
               cudaStream_t st) {
    if (!M || !N || !K) return;
    const uint32_t L = digits_for(fp.p);
    if (A.L != L || B.L != L) fail(GB_EDEVICE, "mm_update: digit count does not match p");
    if (K > mm_kmax(fp.p)) fail(GB_EDEVICE, "mm_update: K above the exact accumulation bound");
    if (ax % 8 || bx % 8) fail(GB_EDEVICE, "mm_update: K offsets must be multiples of 8 (16-byte TMA rule)");
    // the kernel reads whole 64-wide K blocks: a ragged K must end where the planes end (the TMA
    // then fills the rest of the block with zeros)
    if (K % MM_BK && (ax + K != A.K || bx + K != B.K)) fail(GB_EDEVICE, "mm_update: ragged K inside the planes");
    if (ax + K > A.K || bx + K > B.K || ay + M > A.rows || by + N > B.rows)
        fail(GB_EDEVICE, "mm_update: operand range outside the digit planes");
    const CUtensorMap ta = digit_map(A, MM_BM), tb = digit_map(B, MM_BN);
    MmParams P{};
    P.M = M;
    P.N = N;
    P.K = K;
    P.ax = (int)ax;
    P.ay = (int)ay;
    P.bx = (int)bx;
    P.by = (int)by;
    P.C = C;
    P.ldc = ldc;
    P.fp = fp;
    P.big = ((1ull << 50) / fp.p + 1) * fp.p;
    P.sub = sub ? 1 : 0;
    P.err = err;
    const dim3 grid((N + MM_BN - 1) / MM_BN, (M + MM_BM - 1) / MM_BM);
    if (grid.y > 65535u) fail(GB_EUNSUPPORTED, "mm_update: M too large for one launch");
    if (L == 2) {
        opt_in_smem(reinterpret_cast<const void *>(k_mm<2>));
        k_mm<2><<<grid, MM_THREADS, MmCfg<2>::SMEM, st>>>(ta, tb, P);
    } else {
        opt_in_smem(reinterpret_cast<const void *>(k_mm<4>));
        k_mm<4><<<grid, MM_THREADS, MmCfg<4>::SMEM, st>>>(ta, tb, P);
    }
    counted();
}

}  // namespace gb
