// scan_dev.cuh -- the 1024-thread block exclusive scan shared by the
// device-wide scan (sort.cu) and the spawn kernels (qed.cu), which rank
// their own block's event flags against the scanned block sums.
#pragma once
#include <cstdint>

namespace pic {

constexpr int kScanItems = 4096;  // per scan block (1024 threads x 4; the spawn kernels: 256 x 16)

// exclusive scan of one value per thread over a block of NT threads (a
// multiple of 32, at most 1024); sh: 32 words of shared memory; total: the
// block's sum (on every thread)
template <int NT>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *sh, uint32_t &total)
{
    static_assert(NT % 32 == 0 && NT <= 1024, "whole warps, at most 32");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t s = lane < NT / 32 ? sh[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        sh[lane] = s;
    }
    __syncthreads();
    total = sh[NT / 32 - 1];
    uint32_t before = warp ? sh[warp - 1] : 0u;
    uint32_t r = before + x - v;
    __syncthreads();
    return r;
}

__device__ __forceinline__ uint32_t block_excl_scan_1024(uint32_t v, uint32_t *sh, uint32_t &total)
{
    return block_excl_scan<1024>(v, sh, total);
}

}  // namespace pic
