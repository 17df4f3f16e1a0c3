// sig.cu -- the admissibility filter of signature-constrained row selection (Sec. 14, "GPU-facing
// reformulation"; Thm. signature-sound): candidate rows carry packed signature keys, the predicate
// is evaluated over that metadata in bulk, and the survivors are compacted by a scan, so that no
// signature logic enters the kernels that build or reduce the matrix.
//
// A block of candidates is (generator i, shift degree e): candidate j is the signature x^a e_i with
// x^a the j-th monomial of degree e in descending term order.  The F5 criterion rejects it when x^a
// is a leading monomial of the degree-e part of the ideal of the earlier generators; that set is
// a bitmap over the same positions j (bit j of word j / 32), so the predicate is one bit test.  A
// survivor's packed key is (i << 40) | (e << 32) | j: sorted keys are signatures in increasing
// index, then in the order of the candidate list.
#include "internal.hpp"

namespace gb {

namespace {

constexpr int ST = 256;

unsigned grid_for(uint64_t n) {
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((n + ST - 1) / ST, 148ull * 8));
}

// flag[j] = 1 when candidate j is admissible (forbidden may be null: every candidate is)
__global__ void k_sig_admissible(uint32_t ncand, const uint32_t *__restrict__ forbidden, uint32_t *__restrict__ flag) {
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < ncand; j += gridDim.x * blockDim.x)
        flag[j] = forbidden ? ((forbidden[j >> 5] >> (j & 31u)) & 1u) ^ 1u : 1u;
}

// the admissible candidates' keys at their scanned positions (stream compaction)
__global__ void k_sig_compact(uint32_t ncand, unsigned long long head, const uint32_t *__restrict__ flag,
                              const uint32_t *__restrict__ pos, unsigned long long *__restrict__ keys) {
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < ncand; j += gridDim.x * blockDim.x)
        if (flag[j]) keys[pos[j]] = head | j;
}

}  // namespace

uint32_t sig_filter(gb_ctx *ctx, uint32_t index, uint32_t e, uint32_t ncand, const uint32_t *forbidden,
                    unsigned long long *keys) {
    if (index >= (1u << 24) || e > 255) fail(GB_EINVAL, "signature key: index below 2^24 and degree below 256");
    if (!ncand) return 0;
    Arena &ar = ctx->arena;
    cudaStream_t st = ctx->stream;
    DBuf<uint32_t> flag, pos;
    flag.alloc(ar, ncand, st);
    pos.alloc(ar, (size_t)ncand + 1, st);
    k_sig_admissible<<<grid_for(ncand), ST, 0, st>>>(ncand, forbidden, flag.p);
    counted();
    exclusive_scan(ctx, flag.p, pos.p, ncand, st);
    const unsigned long long head = ((unsigned long long)index << 40) | ((unsigned long long)e << 32);
    k_sig_compact<<<grid_for(ncand), ST, 0, st>>>(ncand, head, flag.p, pos.p, keys);
    counted();
    uint32_t *h = static_cast<uint32_t *>(ctx_pinned(ctx, 16));
    GB_CUDA(cudaMemcpyAsync(h, pos.p + ncand, 4, cudaMemcpyDeviceToHost, st));
    ctx_sync(ctx);
    return h[0];
}

}  // namespace gb
