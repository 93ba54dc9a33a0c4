// mlp_tc.cuh -- the surrogate network evaluated by a whole CTA of 128
// threads on the fifth-generation tensor cores: thread t supplies row t of a
// 128-row tile, the two 64 x 64 hidden layers are tcgen05 MMAs (M = 128,
// N = 64, four K = 16 slices) issued by one thread with the accumulator in
// 64 columns of tensor memory, and every warp reads its 32 rows back with
// tcgen05.ld.  The input layer, SiLU, the BF16 rounding of the activations
// and the 64 -> 2 head are those of mlp_forward_rows (mlp.cuh), so the two
// evaluations differ only in the order of the FP32 accumulation.
#pragma once
#include "mlp.cuh"
#include "umma.cuh"

namespace pic {

constexpr int kMlpTcRows = 128;  // rows per evaluation = threads per CTA
constexpr int kMlpTcCols = 64;   // TMEM columns (FP32 accumulator, N = 64)

struct MlpTcSmem {
    alignas(1024) uint8_t A[kMlpTcRows * kMlpH * 2];  // activations (UMMA layout)
    alignas(1024) uint8_t B1[kMlpH * kMlpH * 2];      // W1, rows = output features (UMMA layout)
    alignas(1024) uint8_t B2[kMlpH * kMlpH * 2];
    float W0[kMlpH * 2], b0[kMlpH], b1[kMlpH], b2[kMlpH], W3[2 * kMlpH], b3[4];
    uint64_t bar;
    uint32_t tmem;
};

// whole CTA: copy the network from its device image into the UMMA layout,
// allocate the TMEM accumulator (warp 0) and set up the barrier
__device__ __forceinline__ void mlp_tc_setup(MlpTcSmem &S, const MlpImage *img)
{
    for (int q = threadIdx.x; q < 2 * kMlpH * (kMlpH / 2); q += blockDim.x) {
        const int l = q / (kMlpH * kMlpH / 2), r = q - l * (kMlpH * kMlpH / 2);
        const int n = r / (kMlpH / 2), kp = r - n * (kMlpH / 2);
        const uint32_t w = (l ? img->W2 : img->W1)[n * kMlpPitch + kp];
        *reinterpret_cast<uint32_t *>((l ? S.B2 : S.B1) + umma_offset(n, 2 * kp)) = w;
    }
    for (int q = threadIdx.x; q < kMlpH * 2; q += blockDim.x) {
        S.W0[q] = img->W0[q];
        S.W3[q] = img->W3[q];
    }
    for (int q = threadIdx.x; q < kMlpH; q += blockDim.x) {
        S.b0[q] = img->b0[q];
        S.b1[q] = img->b1[q];
        S.b2[q] = img->b2[q];
    }
    if (threadIdx.x < 4) S.b3[threadIdx.x] = img->b3[threadIdx.x];
    if (threadIdx.x == 0) mbar_init(&S.bar, 1);
    if (threadIdx.x < 32) tmem_alloc(&S.tmem, kMlpTcCols);
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
}

// whole CTA, after the last evaluation
__device__ __forceinline__ void mlp_tc_teardown(MlpTcSmem &S)
{
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (threadIdx.x < 32) tmem_dealloc(S.tmem, kMlpTcCols);
}

// this thread's 64 activations f(acc + bias), rounded to BF16, into row
// threadIdx.x of the A tile
template <typename Fn2>
__device__ __forceinline__ void mlp_tc_put_row(MlpTcSmem &S, const float (&acc)[kMlpH], Fn2 f2)
{
    uint8_t *row = S.A + umma_offset(threadIdx.x, 0);
#pragma unroll
    for (int j = 0; j < kMlpH / 8; j++) {
        uint4 v;
        v.x = f2(acc[8 * j + 0], acc[8 * j + 1]);
        v.y = f2(acc[8 * j + 2], acc[8 * j + 3]);
        v.z = f2(acc[8 * j + 4], acc[8 * j + 5]);
        v.w = f2(acc[8 * j + 6], acc[8 * j + 7]);
        *reinterpret_cast<uint4 *>(row + j * kUmmaLbo) = v;
    }
}

// one hidden layer: TMEM = A . W^T (thread 0 issues, all wait), then this
// thread's row back into registers.  Returns false (in every thread) if
// the MMAs did not complete within the poll limit.
__device__ __forceinline__ bool mlp_tc_layer(MlpTcSmem &S, const uint8_t *B, uint32_t &phase, float (&acc)[kMlpH])
{
    fence_proxy_async_smem();  // the generic-proxy writes of A before the MMA reads it
    tmem_fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
        tmem_fence_after();
        const uint32_t a0 = smem_u32(S.A), b0 = smem_u32(B);
        constexpr uint32_t idesc = umma_idesc_bf16(kMlpTcRows, kMlpH);
#pragma unroll
        for (int s = 0; s < kMlpH / 16; s++)
            umma_bf16(S.tmem, umma_smem_desc(a0 + s * 2 * kUmmaLbo), umma_smem_desc(b0 + s * 2 * kUmmaLbo), idesc,
                      s > 0);
        umma_commit(&S.bar);
    }
    const bool done = mbar_wait(&S.bar, phase, 1 << 20);
    if (__syncthreads_or(!done)) return false;
    phase ^= 1u;
    tmem_fence_after();
    const uint32_t taddr = S.tmem + ((uint32_t)(32 * (threadIdx.x >> 5)) << 16);
    float v[32];
    tmem_ld32(taddr, v);
#pragma unroll
    for (int i = 0; i < 32; i++) acc[i] = v[i];
    tmem_ld32(taddr + 32, v);
#pragma unroll
    for (int i = 0; i < 32; i++) acc[32 + i] = v[i];
    return true;
}

// Whole CTA (blockDim.x == 128): row threadIdx.x has inputs (x0, x1) (any
// values where the result is unused) and gets outputs (y0, y1).  Returns
// false in every thread on a timeout of the tensor cores.
__device__ __forceinline__ bool mlp_eval_cta(MlpTcSmem &S, uint32_t &phase, float x0, float x1, float &y0, float &y1)
{
    float acc[kMlpH];
#pragma unroll
    for (int c = 0; c < kMlpH; c++) acc[c] = fmaf(S.W0[2 * c + 1], x1, fmaf(S.W0[2 * c], x0, S.b0[c]));
    auto act = [](float a, float b) { return silu2_bf16(a, b); };
    mlp_tc_put_row(S, acc, act);
    if (!mlp_tc_layer(S, S.B1, phase, acc)) return false;
#pragma unroll
    for (int c = 0; c < kMlpH; c++) acc[c] += S.b1[c];
    mlp_tc_put_row(S, acc, act);
    if (!mlp_tc_layer(S, S.B2, phase, acc)) return false;
    float p0 = S.b3[0], p1 = S.b3[1];
#pragma unroll
    for (int c = 0; c < kMlpH; c++) {
        const float a = silu(acc[c] + S.b2[c]);
        p0 = fmaf(a, S.W3[c], p0);
        p1 = fmaf(a, S.W3[kMlpH + c], p1);
    }
    y0 = p0;
    y1 = p1;
    return true;
}

}  // namespace pic
