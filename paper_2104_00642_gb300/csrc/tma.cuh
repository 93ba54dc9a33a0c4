// tma.cuh -- tensor-memory-accelerator (TMA) copies into shared memory with
// an mbarrier, written as inline PTX (sm_90 and later, here sm_103a).
//
// Device: mbarrier init / expect-tx / bounded parity wait, a 3D tiled bulk
// tensor load.  Host: the tensor map of the field array (entry point taken
// from the driver at run time, so the library does not link libcuda).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace pic {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// order this thread's earlier generic shared-memory accesses before a
// following async-proxy (TMA) write to the same memory
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// one tile of a 3D tensor: coordinates (x, y, z) of the tile's first element,
// x fastest; x * element size must be a multiple of 16 bytes
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// one tile of a 4D tensor (x fastest; x * element size a multiple of 16 bytes)
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int x, int y, int z, int w,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar))
        : "memory");
}

// wait for the barrier phase with the given parity; gives up after
// max_tries polls (each poll may suspend the thread for a short while) and
// returns false then
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int max_tries)
{
    const uint32_t a = smem_u32(bar);
    for (int i = 0; i < max_tries; i++) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 4-byte asynchronous global -> shared copy (no register round trip), and
// the wait for all of this thread's copies
__device__ __forceinline__ void cp_async4(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Host: tensor map of `ncomp` float arrays of ext[1] rows x ext[0] floats
// (row pitch `pitch` floats, component stride `vol` floats), tiles of
// box[0] x box[1] x box[2]; out-of-range elements read as zero.  Returns
// false when the driver refuses the description.
bool tma_encode_field_map(CUtensorMap *map, const float *base, int ext0, int ext1, long long pitch, long long vol,
                          int ncomp, const int *box);
// the same for 3D arrays: ext[3] (x fastest), strides sy, sz and vol in floats,
// tiles box[0..3] (x, y, z, component)
bool tma_encode_field_map3(CUtensorMap *map, const float *base, const int *ext, long long sy, long long sz,
                           long long vol, int ncomp, const int *box);

}  // namespace pic
