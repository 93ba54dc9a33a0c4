// mlp_tc.cu -- batched evaluation of the surrogate network on the
// fifth-generation tensor cores (tcgen05, accumulators in tensor memory):
// persistent CTAs of 128 threads, one 128-row tile per pass.
#include <algorithm>

#include "mlp_host.cuh"
#include "mlp_tc.cuh"
#include "pic_internal.cuh"

namespace pic {

namespace {

__global__ void __launch_bounds__(kMlpTcRows) k_mlp_eval_tc(const MlpImage *img, long long n,
                                                             const float *__restrict__ X, float *__restrict__ Y,
                                                             int *err)
{
    extern __shared__ unsigned char smem_raw[];
    MlpTcSmem &S = *reinterpret_cast<MlpTcSmem *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    mlp_tc_setup(S, img);
    uint32_t phase = 0;
    const long long ntiles = (n + kMlpTcRows - 1) / kMlpTcRows;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long i = tile * kMlpTcRows + threadIdx.x;
        const bool ok = i < n;
        float y0 = 0.f, y1 = 0.f;
        if (!mlp_eval_cta(S, phase, ok ? X[2 * i] : 0.f, ok ? X[2 * i + 1] : 0.f, y0, y1)) {
            // the tensor cores did not answer: flag it, give the MMAs in
            // flight a last bounded wait, free the tensor memory, stop
            if (threadIdx.x == 0) atomicOr(err, ERR_TIMEOUT);
            mbar_wait(&S.bar, phase, 1 << 20);
            break;
        }
        if (ok) {
            Y[2 * i] = y0;
            Y[2 * i + 1] = y1;
        }
    }
    mlp_tc_teardown(S);
}

}  // namespace

size_t mlp_tc_smem_bytes() { return sizeof(MlpTcSmem) + 1024; }

void launch_mlp_eval_tc(const MlpImage *img, long long n, const float *X, float *Y, int *err, cudaStream_t st)
{
    if (n <= 0) return;
    static bool attr = false;
    const int smem = (int)mlp_tc_smem_bytes();
    if (!attr) {
        cudaFuncSetAttribute(k_mlp_eval_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        attr = true;
    }
    static int nsm = 0;
    if (!nsm) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    }
    // 4 CTAs of 36 KB per SM: 256 of the 512 TMEM columns
    const long long tiles = (n + kMlpTcRows - 1) / kMlpTcRows;
    const int grid = (int)std::min<long long>(tiles, 4ll * nsm);
    note_launch();
    k_mlp_eval_tc<<<grid, kMlpTcRows, smem, st>>>(img, n, X, Y, err);
}

}  // namespace pic
