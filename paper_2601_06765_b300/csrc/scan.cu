// scan.cu -- exclusive prefix sums of u32 arrays: the "plan" step of count -> plan -> fill
// (Sec. 7.1; the FBSP algorithm of Sec. 10).  Tiles of 256 x ITEMS values per block: per-thread
// serial sums, a warp-shuffle scan of the thread sums, then tile offsets from a recursive scan of
// tile totals.  ITEMS (4, 8 or 16) is chosen per size bucket by the autotuner, 8 without it.
#include <algorithm>

#include "internal.hpp"

namespace gb {

constexpr int SCAN_T = 256;

// ITEMS consecutive values per thread, SCAN_T * ITEMS per tile
template <int ITEMS>
__global__ void __launch_bounds__(SCAN_T) k_scan_tiles(const uint32_t *__restrict__ in,
                                                      uint32_t *__restrict__ out,
                                                      uint32_t *__restrict__ tile_sums, size_t n) {
    constexpr int TILE = SCAN_T * ITEMS;
    __shared__ uint32_t warp_sums[SCAN_T / 32];
    const size_t base = (size_t)blockIdx.x * TILE + (size_t)threadIdx.x * ITEMS;
    uint32_t v[ITEMS], sum = 0;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        v[i] = base + i < n ? in[base + i] : 0u;
        sum += v[i];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t y = lane < SCAN_T / 32 ? warp_sums[lane] : 0u;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint32_t z = __shfl_up_sync(0xffffffffu, y, d);
            if (lane >= d) y += z;
        }
        if (lane < SCAN_T / 32) warp_sums[lane] = y;
    }
    __syncthreads();
    uint32_t run = x - sum + (warp ? warp_sums[warp - 1] : 0u);
    if (threadIdx.x == SCAN_T - 1) tile_sums[blockIdx.x] = run + sum;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
}

template <int ITEMS>
__global__ void __launch_bounds__(SCAN_T) k_scan_add(uint32_t *__restrict__ out,
                                                    const uint32_t *__restrict__ tile_prefix,
                                                    size_t n) {
    constexpr int TILE = SCAN_T * ITEMS;
    const size_t base = (size_t)blockIdx.x * TILE;
    const uint32_t add = tile_prefix[blockIdx.x];
    for (int i = threadIdx.x; i < TILE; i += SCAN_T)
        if (base + i < n) out[base + i] += add;
}

__global__ void k_copy_u32(uint32_t *dst, const uint32_t *src) { *dst = *src; }

namespace {

template <int ITEMS>
void scan_with(gb_ctx *ctx, const uint32_t *in, uint32_t *out, size_t n, cudaStream_t s) {
    constexpr size_t TILE = (size_t)SCAN_T * ITEMS;
    const size_t tiles = n ? (n + TILE - 1) / TILE : 1;
    if (tiles == 1) {
        k_scan_tiles<ITEMS><<<1, SCAN_T, 0, s>>>(in, out, out + n, n);
        counted();
        return;
    }
    DBuf<uint32_t> sums, pref;
    sums.alloc(ctx->arena, tiles, s);
    pref.alloc(ctx->arena, tiles + 1, s);
    k_scan_tiles<ITEMS><<<(unsigned)tiles, SCAN_T, 0, s>>>(in, out, sums.p, n);
    counted();
    exclusive_scan(ctx, sums.p, pref.p, tiles, s);
    k_scan_add<ITEMS><<<(unsigned)tiles, SCAN_T, 0, s>>>(out, pref.p, n);
    counted();
    k_copy_u32<<<1, 1, 0, s>>>(out + n, pref.p + tiles);
    counted();
}

}  // namespace

// values per thread of each candidate tile (TUNE_SCAN choice 0, 1, 2); without a tuned bucket, 8
constexpr int SCAN_ITEMS_OF[3] = {4, 8, 16};

void exclusive_scan_items(gb_ctx *ctx, int items, const uint32_t *in, uint32_t *out, size_t n, cudaStream_t s) {
    if (items == 4) scan_with<4>(ctx, in, out, n, s);
    else if (items == 16) scan_with<16>(ctx, in, out, n, s);
    else scan_with<8>(ctx, in, out, n, s);
}

void exclusive_scan(gb_ctx *ctx, const uint32_t *in, uint32_t *out, size_t n, cudaStream_t s) {
    int items = 8;
    const auto it = ctx->tune.table.find(tune_key(TUNE_SCAN, 0, (uint32_t)std::min<size_t>(n, UINT32_MAX - 1), 0, 0));
    if (it != ctx->tune.table.end() && it->second.choice < 3) items = SCAN_ITEMS_OF[it->second.choice];
    exclusive_scan_items(ctx, items, in, out, n, s);
}

}  // namespace gb
