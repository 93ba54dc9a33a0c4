// scan_dev.cuh -- the 1024-thread block exclusive scan shared by the
// device-wide scan (sort.cu) and the spawn kernels (qed.cu), which rank
// their own block's event flags against the scanned block sums.
#pragma once
#include <cstdint>

namespace pic {

constexpr int kScanItems = 4096;  // per scan block (1024 threads x 4)

// exclusive scan of one value per thread over a block of 1024 threads; sh:
// 32 words of shared memory; total: the block's sum (on every thread)
__device__ __forceinline__ uint32_t block_excl_scan_1024(uint32_t v, uint32_t *sh, uint32_t &total)
{
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
        uint32_t s = sh[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        sh[lane] = s;
    }
    __syncthreads();
    total = sh[31];
    uint32_t before = warp ? sh[warp - 1] : 0u;
    uint32_t r = before + x - v;
    __syncthreads();
    return r;
}

}  // namespace pic
