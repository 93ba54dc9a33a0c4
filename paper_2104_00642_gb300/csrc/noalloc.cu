// noalloc.cu -- FP64 field energy of caller-owned device arrays without any
// device allocation.
//
// Who needs it: callers that cannot call cudaMalloc -- code that runs where
// the CUDA allocator is off limits to it, such as a plugin living inside a
// host application that owns every device allocation through its own pool,
// or a real-time loop that must not allocate once it runs.  They cannot
// create a pic_sim (pic_create allocates), but they can still reduce their
// own field arrays with the library's fixed-order FP64 reduction.
//
// How: the reduction is the same two-pass fixed tree as the diagnostics
// (per-block partial sums, then one block summing them in index order), but
// its scratch -- the per-block partials -- is a file-scope static device
// array of a fixed size instead of memory from cudaMalloc.  That array exists
// once on every GPU that loads the library and is held until the process
// exits.  Host code may not use its name as a device address, so the first
// call on a device looks its address up with cudaGetSymbolAddress (with that
// device current) and caches it.  The address belongs to the CUDA context it
// was looked up in: after cudaDeviceReset the next context may load the
// module elsewhere, so the cache remembers the context's unique identifier
// and looks the address up again when the current context is another one.
#include <cuda.h>

#include <cstdio>
#include <mutex>
#include <string>

#include "../../include/pic.h"
#include "pic_internal.cuh"

namespace pic {
void set_global_error(const std::string &msg);  // defined in capi.cu
}

namespace {

constexpr int kNaThreads = 256;
constexpr int kNaItems = 64;                              // elements per thread
constexpr int kNaMaxBlocks = 4096;                        // partial sums held
constexpr long long kNaBlockElems = (long long)kNaThreads * kNaItems;
constexpr long long kNaMaxN = kNaMaxBlocks * kNaBlockElems;  // 67,108,864 elements per array
constexpr int kNaMaxDevices = 64;

// the scratch: two partial sums (E^2, B^2) per block
static __device__ __align__(256) double g_noalloc_partials[2 * kNaMaxBlocks];

struct Six {
    const double *p[6];
};

__device__ __forceinline__ double na_warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// each block sums its kNaBlockElems elements of the six arrays (fixed
// strided order, fixed shuffle tree) into partial[2b], partial[2b+1]
__global__ void __launch_bounds__(kNaThreads) k_na_partials(Six f, long long n, double *partial)
{
    double e2 = 0.0, b2 = 0.0;
    long long base = (long long)blockIdx.x * kNaBlockElems + threadIdx.x;
    for (int q = 0; q < kNaItems; q++) {
        long long i = base + (long long)q * kNaThreads;
        if (i >= n) break;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            double e = f.p[c][i], b = f.p[3 + c][i];
            e2 += e * e;
            b2 += b * b;
        }
    }
    __shared__ double sh[2][kNaThreads / 32];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    e2 = na_warp_sum(e2);
    b2 = na_warp_sum(b2);
    if (lane == 0) {
        sh[0][warp] = e2;
        sh[1][warp] = b2;
    }
    __syncthreads();
    if (warp == 0) {
        double x = lane < kNaThreads / 32 ? sh[0][lane] : 0.0;
        double y = lane < kNaThreads / 32 ? sh[1][lane] : 0.0;
        x = na_warp_sum(x);
        y = na_warp_sum(y);
        if (lane == 0) {
            partial[2 * blockIdx.x] = x;
            partial[2 * blockIdx.x + 1] = y;
        }
    }
}

// one block: out[0] = dV/2 sum_b partial[2b], out[1] = dV/2 sum_b partial[2b+1]
__global__ void __launch_bounds__(kNaThreads) k_na_final(const double *partial, int nb, double half_dV, double *out)
{
    double x = 0.0, y = 0.0;
    for (int b = threadIdx.x; b < nb; b += kNaThreads) {
        x += partial[2 * b];
        y += partial[2 * b + 1];
    }
    __shared__ double sh[2][kNaThreads / 32];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    x = na_warp_sum(x);
    y = na_warp_sum(y);
    if (lane == 0) {
        sh[0][warp] = x;
        sh[1][warp] = y;
    }
    __syncthreads();
    if (warp == 0) {
        x = lane < kNaThreads / 32 ? sh[0][lane] : 0.0;
        y = lane < kNaThreads / 32 ? sh[1][lane] : 0.0;
        x = na_warp_sum(x);
        y = na_warp_sum(y);
        if (lane == 0) {
            out[0] = half_dV * x;
            out[1] = half_dV * y;
        }
    }
}

std::mutex g_na_mutex;
void *g_na_addr[kNaMaxDevices] = {};
unsigned long long g_na_ctx[kNaMaxDevices] = {};  // identifier of the context g_na_addr belongs to

// unique identifier of the current CUDA context (driver entry points, so the
// library needs no link to the driver library); false if there is no current
// context or the driver does not offer the calls
bool na_current_context(unsigned long long *id)
{
    using GetCurrent = CUresult (*)(CUcontext *);
    using GetId = CUresult (*)(CUcontext, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(p);
    });
    CUcontext ctx = nullptr;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
    return get_id(ctx, id) == CUDA_SUCCESS;
}

int na_fail(int code, const char *msg)
{
    pic::set_global_error(msg);
    return code;
}

}  // namespace

extern "C" int pic_field_energy_noalloc(const double *const dev_fields[6], int64_t n, double dV, double *dev_out2,
                                        void *stream)
{
    if (!dev_fields || !dev_out2) return na_fail(PIC_ERR_ARG, "pic_field_energy_noalloc: null pointer");
    for (int c = 0; c < 6; c++)
        if (!dev_fields[c]) return na_fail(PIC_ERR_ARG, "pic_field_energy_noalloc: null field pointer");
    if (n < 0 || n > kNaMaxN) {
        char buf[160];
        snprintf(buf, sizeof buf, "pic_field_energy_noalloc: n = %lld outside [0, %lld] (size of the static scratch)",
                 (long long)n, kNaMaxN);
        return na_fail(PIC_ERR_ARG, buf);
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kNaMaxDevices)
        return na_fail(PIC_ERR_CUDA, "pic_field_energy_noalloc: no current CUDA device");
    void *scratch = nullptr;
    {
        // set-up, once per device (and again in a new context of that device)
        // with that device current: the device address of the static scratch
        // array
        std::lock_guard<std::mutex> lk(g_na_mutex);
        unsigned long long ctx = 0;
        const bool known = na_current_context(&ctx);
        if (!g_na_addr[dev] || !known || g_na_ctx[dev] != ctx) {
            void *addr = nullptr;
            e = cudaGetSymbolAddress(&addr, g_noalloc_partials);
            if (e != cudaSuccess) {
                g_na_addr[dev] = nullptr;
                std::string m = std::string("pic_field_energy_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
                return na_fail(PIC_ERR_CUDA, m.c_str());
            }
            // the look-up made the device's primary context current if none was
            unsigned long long now = 0;
            g_na_addr[dev] = addr;
            g_na_ctx[dev] = na_current_context(&now) ? now : 0;
        }
        scratch = g_na_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    int nb = (int)((n + kNaBlockElems - 1) / kNaBlockElems);
    Six f;
    for (int c = 0; c < 6; c++) f.p[c] = dev_fields[c];
    if (nb > 0) k_na_partials<<<nb, kNaThreads, 0, st>>>(f, n, (double *)scratch);
    k_na_final<<<1, kNaThreads, 0, st>>>((const double *)scratch, nb, 0.5 * dV, dev_out2);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        std::string m = std::string("pic_field_energy_noalloc: ") + cudaGetErrorString(e);
        return na_fail(PIC_ERR_CUDA, m.c_str());
    }
    return PIC_OK;
}
