// mlp_host.cuh -- host side of the surrogate network (mlp.cu).
#pragma once
#include <cuda_runtime.h>

#include "mlp.cuh"
#include "qed.cuh"

namespace pic {

// one network: FP32 master parameters with Adam moments and the gradient
// (packed order), and the BF16 device image the kernels read
struct MlpNet {
    MlpImage *img = nullptr;
    float *P = nullptr, *M = nullptr, *V = nullptr, *G = nullptr;
    MlpNorm nrm{};
    bool ready = false;
};

// training scratch for a batch of B rows (B a multiple of 128)
struct MlpScratch {
    long long B = 0;
    float *X = nullptr, *T = nullptr, *Y = nullptr;  // [B][2]
    MlpZ Z{}, D{};                                   // [B][64] each
    float *loss = nullptr;                           // [0] this iteration, [1] the last one
    int *it = nullptr;                               // iteration counter
    double *acc = nullptr;                           // validation accumulators (kMlpValAcc)
    float *partials = nullptr;                       // per-block / per-warp gradient partials
};

// validation grid: kMlpValRows x kMlpValRows cell midpoints in (ln chi, r);
// accumulators: max |d ln G|, max |d s|, sum d s^2, (unused), then per chi
// row the sums of the network's and the tables' energy fractions
constexpr int kMlpValRows = 256;
constexpr int kMlpValAcc = 4 + 2 * kMlpValRows;

// floats of gradient partials a batch of B rows needs (mlp_partial_floats)
size_t mlp_partial_floats(long long B);

struct MlpAdam {
    long long iters;
    double lr0, lr_final;
    float beta1, beta2, eps;
};

// (both staged images stay below the 48 KB default dynamic shared memory)
static_assert(kMlpTrainStageBytes <= 48 * 1024, "no opt-in needed");
void launch_mlp_image(const float *P, MlpImage *img, cudaStream_t st);
void launch_mlp_forward(const MlpImage *img, long long B, const float *X, const MlpZ &Z, float *Y, cudaStream_t st);
// backward pass, weight gradients and their fixed-order reduction into grad
// (overwritten) and *loss (overwritten); partials: mlp_partial_floats(B)
void launch_mlp_backward(const MlpImage *img, long long B, const float *X, const float *Tg, const float *Y,
                         const MlpZ &Z, const MlpZ &D, float *partials, float *grad, float w_rate, float *loss,
                         cudaStream_t st);
void mlp_train_iteration(MlpNet &net, MlpScratch &S, const QedTables &T, int p, const uint32_t *key,
                         const MlpAdam &a, float w_rate, cudaStream_t st);
void launch_mlp_eval(const MlpImage *img, long long n, const float *X, float *Y, cudaStream_t st);
// the same evaluation on the tcgen05 tensor cores (mlp_tc.cu); a timeout of
// the tensor cores sets ERR_TIMEOUT in *err
void launch_mlp_eval_tc(const MlpImage *img, long long n, const float *X, float *Y, int *err, cudaStream_t st);
size_t mlp_tc_smem_bytes();
void launch_qed_eval_surr(const MlpImage *img, const MlpNorm &nrm, const QedTables &T, bool f64, int p, long long n,
                          const double *chi, const double *r, double *out, cudaStream_t st);
void launch_mlp_validate(const MlpImage *img, const MlpNorm &nrm, const QedTables &T, int p, int nc, int nr,
                         double *acc, cudaStream_t st);

}  // namespace pic
