// umma.cuh -- fifth-generation tensor-core (tcgen05) building blocks written
// as inline PTX for sm_100-family GPUs (here sm_103a): tensor-memory (TMEM)
// allocation, shared-memory matrix descriptors, the instruction descriptor of
// a BF16 x BF16 -> FP32 MMA, the MMA itself, its completion on an mbarrier,
// and the TMEM -> register load of the accumulator.
//
// Operand layout used throughout: both operands K-major without swizzle, in
// core matrices of 8 rows x 16 bytes (8 BF16 values along K) stored as 128
// contiguous bytes; core matrices adjacent along K are kUmmaLbo bytes apart,
// 8-row groups kUmmaSbo bytes apart (a row of 64 BF16 values spans the eight
// K groups of one 1 KB row group).  Element (row, k) of such a tile sits at
//   (row / 8) * kUmmaSbo + (k / 8) * kUmmaLbo + (row % 8) * 16 + (k % 8) * 2.
#pragma once
#include <cstdint>

#include "tma.cuh"

namespace pic {

constexpr int kUmmaLbo = 128;   // bytes between core matrices adjacent along K
constexpr int kUmmaSbo = 1024;  // bytes between 8-row groups (64 K values per row)

__host__ __device__ constexpr int umma_offset(int row, int k)
{
    return (row >> 3) * kUmmaSbo + (k >> 3) * kUmmaLbo + (row & 7) * 16 + (k & 7) * 2;
}

// shared-memory matrix descriptor: start address, leading (K) and stride
// (8-row group) byte offsets, all in 16-byte units; descriptor version 1;
// base offset 0; no swizzle
__device__ __forceinline__ uint64_t umma_smem_desc(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((kUmmaLbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((kUmmaSbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor of kind::f16 with BF16 A and B, FP32 accumulator,
// both operands K-major, shape M x N (M in {64, 128}, N a multiple of 16)
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N)
{
    return (1u << 4)                          // accumulator format: F32
           | (1u << 7)                        // A format: BF16
           | (1u << 10)                       // B format: BF16
           | ((uint32_t)(N >> 3) << 17)       // N / 8
           | ((uint32_t)(M >> 4) << 24);      // M / 16
}

// D[tmem] (+)= A[smem] . B[smem]^T for one K = 16 slice, issued by one thread
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                          bool accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"((uint32_t)accumulate)
        : "memory");
}

// arrive once on the mbarrier when this thread's MMAs issued so far complete
__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// whole warp: allocate `ncols` TMEM columns (a power of two >= 32); the base
// address is written to *slot (shared memory)
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

// whole warp: free the columns again
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// whole warp: 32 consecutive FP32 columns of the warp's 32 TMEM lanes (lane
// i of the warp gets TMEM lane 32 (warp % 4) + i), then wait for the load
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
}

}  // namespace pic
