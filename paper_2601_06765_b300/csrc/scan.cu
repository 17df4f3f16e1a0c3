// scan.cu -- exclusive prefix sums of u32 arrays: the "plan" step of count -> plan -> fill
// (Sec. 7.1; the FBSP algorithm of Sec. 10).  Tiles of 2048 values per 256-thread block:
// per-thread serial sums, a warp-shuffle scan of the thread sums, then tile offsets from a
// recursive scan of tile totals.
#include "internal.hpp"

namespace gb {

constexpr int SCAN_T = 256, SCAN_ITEMS = 8, SCAN_TILE = SCAN_T * SCAN_ITEMS;

__global__ void __launch_bounds__(SCAN_T) k_scan_tiles(const uint32_t *__restrict__ in,
                                                      uint32_t *__restrict__ out,
                                                      uint32_t *__restrict__ tile_sums, size_t n) {
    __shared__ uint32_t warp_sums[SCAN_T / 32];
    const size_t base = (size_t)blockIdx.x * SCAN_TILE + (size_t)threadIdx.x * SCAN_ITEMS;
    uint32_t v[SCAN_ITEMS], sum = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
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
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
}

__global__ void __launch_bounds__(SCAN_T) k_scan_add(uint32_t *__restrict__ out,
                                                    const uint32_t *__restrict__ tile_prefix,
                                                    size_t n) {
    const size_t base = (size_t)blockIdx.x * SCAN_TILE;
    const uint32_t add = tile_prefix[blockIdx.x];
    for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_T)
        if (base + i < n) out[base + i] += add;
}

__global__ void k_copy_u32(uint32_t *dst, const uint32_t *src) { *dst = *src; }

void exclusive_scan(Arena &ar, const uint32_t *in, uint32_t *out, size_t n, cudaStream_t s) {
    const size_t tiles = n ? (n + SCAN_TILE - 1) / SCAN_TILE : 1;
    if (tiles == 1) {
        k_scan_tiles<<<1, SCAN_T, 0, s>>>(in, out, out + n, n);
        counted();
        GB_CUDA(cudaGetLastError());
        return;
    }
    DBuf<uint32_t> sums, pref;
    sums.alloc(ar, tiles, s);
    pref.alloc(ar, tiles + 1, s);
    k_scan_tiles<<<(unsigned)tiles, SCAN_T, 0, s>>>(in, out, sums.p, n);
    counted();
    GB_CUDA(cudaGetLastError());
    exclusive_scan(ar, sums.p, pref.p, tiles, s);
    k_scan_add<<<(unsigned)tiles, SCAN_T, 0, s>>>(out, pref.p, n);
    counted();
    k_copy_u32<<<1, 1, 0, s>>>(out + n, pref.p + tiles);
    counted();
    GB_CUDA(cudaGetLastError());
}

}  // namespace gb
