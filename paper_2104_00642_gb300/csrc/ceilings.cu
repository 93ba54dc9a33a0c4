// ceilings.cu -- throughput ceilings of the instruction mixes the push
// kernels are made of, measured on the GPU they run on: FP32 FMA, FP64 FMA,
// shared-memory integer atomics (conflict-free, as the lane-strided deposit
// issues them, and with all 32 lanes on one word), and the warp reduction
// the warp-aggregated deposit uses.  Each kernel runs a fixed number of
// independent chains per thread on a grid of 8 CTAs of 256 threads per SM
// and is timed with CUDA events; the results are per second for the whole
// GPU.  Loops have compile-time trip counts; nothing waits on anything.
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/pic.h"
#include "pic_internal.cuh"

namespace pic {

constexpr int kCeilIters = 4096;
constexpr int kCeilChains = 8;

template <typename R>
__global__ void __launch_bounds__(256) k_ceil_fma(R seed, R *sink)
{
    R a[kCeilChains];
#pragma unroll
    for (int c = 0; c < kCeilChains; c++) a[c] = seed + R(threadIdx.x + c);
    const R m = R(0.999999), k = R(1e-7);
    for (int i = 0; i < kCeilIters; i++) {
#pragma unroll
        for (int c = 0; c < kCeilChains; c++) a[c] = fma(a[c], m, k);
    }
    R s = 0;
#pragma unroll
    for (int c = 0; c < kCeilChains; c++) s += a[c];
    if (s == R(-1.2345)) sink[threadIdx.x] = s;  // never true: keeps the chains live
}

// MODE 0: lane l adds to word l (32 banks, no conflict); MODE 1: every lane
// of the warp adds to one word; MODE 2: the warp reduction of the
// aggregated deposit (__reduce_add_sync over a group mask), then one atomic
// per group, for groups of 8 lanes
template <int MODE>
__global__ void __launch_bounds__(256) k_ceil_atom(int seed, int *sink)
{
    __shared__ int box[256 * kCeilChains];
    for (int q = threadIdx.x; q < 256 * kCeilChains; q += blockDim.x) box[q] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned grp = 0xFFu << (lane & ~7);
    int v = seed + lane;
    for (int i = 0; i < kCeilIters / 8; i++) {
#pragma unroll
        for (int c = 0; c < kCeilChains; c++) {
            int *w = box + (warp * kCeilChains + c) * 32;
            if (MODE == 0) atomicAdd(w + lane, v);
            else if (MODE == 1) atomicAdd(w, v);
            else {
                const int s = __reduce_add_sync(grp, v);
                if ((lane & 7) == 0) atomicAdd(w + lane, s);
            }
            v += 1;
        }
    }
    __syncthreads();
    if (box[threadIdx.x] == -12345) sink[threadIdx.x] = v;
}

}  // namespace pic

using namespace pic;

extern "C" int pic_measure_ceilings(double *out)
{
    if (!out) return PIC_ERR_ARG;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PIC_ERR_CUDA;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int grid = 8 * nsm, block = 256;
    void *sink = nullptr;
    if (cudaMalloc(&sink, 4096) != cudaSuccess) return PIC_ERR_NOMEM;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const double threads = (double)grid * block;
    auto timed = [&](auto launch, double ops_per_thread) {
        launch();  // warm-up
        cudaEventRecord(a);
        for (int r = 0; r < 5; r++) launch();
        cudaEventRecord(b);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        return 5.0 * threads * ops_per_thread / (ms * 1e-3);
    };
    const double fmas = (double)kCeilIters * kCeilChains;
    const double atoms = (double)(kCeilIters / 8) * kCeilChains;
    out[0] = 2.0 * timed([&] { k_ceil_fma<float><<<grid, block>>>(1.0f, (float *)sink); }, fmas);    // FP32 flop/s
    out[1] = 2.0 * timed([&] { k_ceil_fma<double><<<grid, block>>>(1.0, (double *)sink); }, fmas);   // FP64 flop/s
    out[2] = timed([&] { k_ceil_atom<0><<<grid, block>>>(1, (int *)sink); }, atoms);  // lane atomics/s, no conflict
    out[3] = timed([&] { k_ceil_atom<1><<<grid, block>>>(1, (int *)sink); }, atoms);  // lane atomics/s, one word per warp
    out[4] = timed([&] { k_ceil_atom<2><<<grid, block>>>(1, (int *)sink); }, atoms);  // lane values/s through reduce + atomic
    const cudaError_t e = cudaGetLastError();
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(sink);
    return e == cudaSuccess ? PIC_OK : PIC_ERR_CUDA;
}
