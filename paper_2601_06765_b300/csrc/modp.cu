// modp.cu -- gb_modp_apply: the register-level F_p primitives of device.cuh applied elementwise to
// device arrays, so that each one can be checked on its own against plain integer arithmetic:
// Barrett reduction (Sec. 8.3), Montgomery reduction and domain conversion (Sec. 8.4), the two
// inverses, the lazy accumulation windows of the sparse reduction (Rem. 8.1), and chains of
// multiply-adds kept in registers (Barrett against Montgomery: the modular inner loop timed by the
// microbenchmarks of Sec. 12.2).  The kernels
// call exactly the functions the reduction kernels call, with the Fp constants of make_fp.
#include "internal.hpp"

namespace gb {

namespace {

__global__ void k_modp_apply(int op, Fp fp, uint64_t n, uint32_t window, const uint32_t *__restrict__ a,
                             const uint32_t *__restrict__ b, const uint32_t *__restrict__ c,
                             uint32_t *__restrict__ out) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t r = 0;
        switch (op) {
        case GB_MODP_REDUCE64: r = fp_reduce(((uint64_t)a[i] << 32) | b[i], fp); break;
        case GB_MODP_REDUCE32: r = fp_reduce32(a[i], fp); break;
        case GB_MODP_MULADD: r = fp_reduce((uint64_t)a[i] * b[i] + c[i], fp); break;
        case GB_MODP_REDC: r = fp_redc(((uint64_t)a[i] << 32) | b[i], fp); break;
        case GB_MODP_TO_MONT: r = fp_to_mont(a[i], fp); break;
        case GB_MODP_MONT_MUL: r = fp_redc((uint64_t)fp_to_mont(a[i], fp) * b[i], fp); break;
        case GB_MODP_INV: r = fp_inv(a[i], fp); break;
        case GB_MODP_INV_SMALL: r = fp_inv_small(a[i], fp); break;
        case GB_MODP_LAZY32: {
            // the A32 accumulator of the sparse reduction: a start residue, then reduced products
            // added in 32 bits with no reduction in between, reduced once at the end
            uint32_t acc = c[i];
            const uint64_t j0 = i * window;
            for (uint32_t j = 0; j < window; ++j) acc += fp_reduce32(a[j0 + j] * b[j0 + j], fp);
            r = fp_reduce32(acc, fp);
            break;
        }
        case GB_MODP_LAZY_MONT: {
            // the M64 accumulator: a start residue, then redc((a R mod p) * b) terms (each below 2p)
            // added in 64 bits, reduced once at the end
            uint64_t acc = c[i];
            const uint64_t j0 = i * window;
            for (uint32_t j = 0; j < window; ++j)
                acc += fp_redc((uint64_t)fp_to_mont(a[j0 + j], fp) * b[j0 + j], fp);
            r = fp_reduce(acc, fp);
            break;
        }
        case GB_MODP_CHAIN_BARRETT: {
            uint32_t x = a[i];
            const uint32_t m = b[i], d = c[i];
            for (uint32_t j = 0; j < window; ++j) x = fp_reduce((uint64_t)x * m + d, fp);
            r = x;
            break;
        }
        case GB_MODP_CHAIN_MONT: {
            uint32_t x = a[i];
            const uint32_t m = fp_to_mont(b[i], fp), d = c[i];
            for (uint32_t j = 0; j < window; ++j) {
                uint32_t y = fp_redc((uint64_t)x * m, fp);  // x b mod p, in [0, 2p)
                y = y >= fp.p ? y - fp.p : y;
                x = fp_add(y, d, fp);
            }
            r = x;
            break;
        }
        default: break;
        }
        out[i] = r;
    }
}

}  // namespace

void modp_apply(int op, uint32_t p, uint64_t n, uint32_t window, const uint32_t *a, const uint32_t *b,
                const uint32_t *c, uint32_t *out, cudaStream_t st) {
    if (p < 3 || p >= (1u << 31) || !is_prime32(p)) fail(GB_EINVAL, "p must be an odd prime below 2^31");
    if (op < GB_MODP_REDUCE64 || op > GB_MODP_CHAIN_MONT) fail(GB_EINVAL, "gb_modp_apply: unknown operation");
    const bool small_only = op == GB_MODP_REDUCE32 || op == GB_MODP_INV_SMALL || op == GB_MODP_LAZY32;
    if (small_only && p >= 65536u) fail(GB_EINVAL, "gb_modp_apply: this operation needs p < 2^16");
    const bool windowed = op == GB_MODP_LAZY32 || op == GB_MODP_LAZY_MONT;
    const bool chain = op == GB_MODP_CHAIN_BARRETT || op == GB_MODP_CHAIN_MONT;
    if ((windowed || chain) && (window == 0 || (op == GB_MODP_LAZY32 && window >= 65536u)))
        fail(GB_EINVAL, "gb_modp_apply: window must be in [1, 2^16) for the 32-bit sum, >= 1 otherwise");
    if (!n) return;
    const bool needs_b = op == GB_MODP_REDUCE64 || op == GB_MODP_MULADD || op == GB_MODP_REDC ||
                         op == GB_MODP_MONT_MUL || windowed || chain;
    const bool needs_c = op == GB_MODP_MULADD || windowed || chain;
    if (!a || !out || (needs_b && !b) || (needs_c && !c)) fail(GB_EINVAL, "gb_modp_apply: null device pointer");
    const unsigned grid = (unsigned)std::min<uint64_t>((n + 255) / 256, 148ull * 16);
    k_modp_apply<<<grid, 256, 0, st>>>(op, make_fp(p), n, window, a, b, c, out);
    counted();
}

}  // namespace gb
