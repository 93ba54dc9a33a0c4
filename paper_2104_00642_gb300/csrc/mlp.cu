// mlp.cu -- training and evaluation kernels of the surrogate network that
// stands in for the QED tables (Sec. IV, Eqs. (23)/(24)).
//
// Training (one Adam step per iteration, all on the device, captured once
// as a CUDA graph and replayed):
//   data   : Philox (x0, r) samples, targets from the FP64 tables
//   fwd    : per warp 32 rows, mma.sync BF16 hidden layers, stores Z1..Z3
//   bwd    : per warp: dY, head gradients, deltas D3 -> D2 -> D1 through
//            the transposed weights on the tensor cores
//   wgrad  : dW_l = sum_rows D_{l+1} (x) bf16(a_l) in FP32, db_l = sum D
//   adam   : FP32 master update, BF16 image rewrite, gradient zeroed
//   tick   : iteration counter, loss latch
// Loss L = (1/B) sum_rows [(y0 - s)^2 + w (y1 - l)^2].
#include <cmath>

#include "mlp_host.cuh"
#include "qed.cuh"

namespace pic {

namespace {

__device__ __forceinline__ float bf16_round(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// write parameter i (packed order) into the image
__device__ __forceinline__ void image_put(MlpImage *img, int i, float v)
{
    if (i < kOffB0) {
        img->W0[i - kOffW0] = bf16_round(v);
    } else if (i < kOffW1) {
        img->b0[i - kOffB0] = v;
    } else if (i < kOffB1 || (i >= kOffW2 && i < kOffB2)) {
        const bool two = i >= kOffW2;
        const int q = i - (two ? kOffW2 : kOffW1), n = q / kMlpH, k = q % kMlpH;
        __nv_bfloat16 *W = reinterpret_cast<__nv_bfloat16 *>(two ? img->W2 : img->W1);
        __nv_bfloat16 *WT = reinterpret_cast<__nv_bfloat16 *>(two ? img->W2T : img->W1T);
        const __nv_bfloat16 b = __float2bfloat16_rn(v);
        W[n * 2 * kMlpPitch + k] = b;
        WT[k * 2 * kMlpPitch + n] = b;
    } else if (i < kOffW2) {
        img->b1[i - kOffB1] = v;
    } else if (i < kOffW3) {
        img->b2[i - kOffB2] = v;
    } else if (i < kOffB3) {
        img->W3[i - kOffW3] = bf16_round(v);
    } else {
        img->b3[i - kOffB3] = v;
    }
}

__global__ void k_mlp_image(const float *__restrict__ P, MlpImage *img)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kMlpNParams) image_put(img, i, P[i]);
}

// training samples: x0 uniform in [-1, 1] (ln chi uniform over the range),
// r uniform as the Monte Carlo draws it; targets from the FP64 tables
__global__ void k_mlp_data(QedTables T, int p, MlpNorm nrm, uint32_t k0, uint32_t k1, const int *it, long long B,
                           float *__restrict__ X, float *__restrict__ Y)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B) return;
    uint32_t w[4];
    philox4x32_10((uint32_t)i, (uint32_t)(i >> 32), (uint32_t)*it, QP_TRAIN + p, k0, k1, w);
    const float x0 = (float)(2.0 * uniform24(w[0]) - 1.0);
    // emission: half the rows take r uniform, half r = 1 - (1 - t)^2 with t
    // uniform (uniform in the network's r coordinate), so that the hard end of
    // the spectrum (r -> 1), which carries most of the emitted energy, is
    // sampled as densely as the soft end
    const double t = uniform24(w[1]);
    const double r = p == QED_RAD && (w[2] & 1u) ? 1.0 - (1.0 - t) * (1.0 - t) : t;
    const double lnchi = ((double)x0 - nrm.x0b) / nrm.x0a, chi = exp(lnchi);
    const double rr = p == QED_PAIR ? fmin(r, 1.0 - r) : r;
    const double s = cbrt(qed_sample<double>(T, p, chi, rr));
    const double lg = qed_lnG_table<double>(T, p, (lnchi - T.lnchi0) / T.dlnchi);
    X[2 * i] = x0;
    X[2 * i + 1] = (float)mlp_rcoord(p, r);
    Y[2 * i] = (float)s;
    Y[2 * i + 1] = (float)((lg - nrm.mu) / nrm.sd);
}

// rows of this thread's quad group: rr = 16 (r >> 1) + 8 (r & 1) + g
__device__ __forceinline__ long long quad_row(long long row0, int r, int g) { return row0 + 16 * (r >> 1) + 8 * (r & 1) + g; }

__global__ void __launch_bounds__(128) k_mlp_fwd(const MlpImage *img, long long B, const float *__restrict__ X,
                                                 MlpZ Z, float *__restrict__ Y)
{
    extern __shared__ __align__(16) unsigned char smem[];
    mlp_stage(smem, img, kMlpStageBytes);
    __syncthreads();
    const MlpImage &S = *reinterpret_cast<const MlpImage *>(smem);
    const long long row0 = ((long long)blockIdx.x * 4 + (threadIdx.x >> 5)) * 32;
    if (row0 >= B) return;  // B is a multiple of 32: whole warps
    const int g = (threadIdx.x & 31) >> 2, t = threadIdx.x & 3;
    float x[4][2], y[4][2];
#pragma unroll
    for (int r = 0; r < 4; r++) {
        const long long row = quad_row(row0, r, g);
        x[r][0] = X[2 * row];
        x[r][1] = X[2 * row + 1];
    }
    mlp_forward_rows<true>(S, x, y, Z, row0);
    if (t == 0)
#pragma unroll
        for (int r = 0; r < 4; r++) {
            const long long row = quad_row(row0, r, g);
            Y[2 * row] = y[r][0];
            Y[2 * row + 1] = y[r][1];
        }
}

// head: per-warp partials of dW3 (128), db3 (2) and the loss (1)
constexpr int kHeadPartial = 2 * kMlpH + 3;

__global__ void __launch_bounds__(128) k_mlp_bwd(const MlpImage *img, long long B, const float *__restrict__ Tg,
                                                 const float *__restrict__ Y, MlpZ Z, MlpZ D, float *__restrict__ head,
                                                 float w_rate)
{
    extern __shared__ __align__(16) unsigned char smem[];
    mlp_stage(smem, img, kMlpTrainStageBytes);
    __syncthreads();
    const MlpImage &S = *reinterpret_cast<const MlpImage *>(smem);
    const long long row0 = ((long long)blockIdx.x * 4 + (threadIdx.x >> 5)) * 32;
    if (row0 >= B) return;
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const float invB = 1.0f / (float)B;
    float dy[4][2], lsum = 0.f;
#pragma unroll
    for (int r = 0; r < 4; r++) {
        const long long row = quad_row(row0, r, g);
#pragma unroll
        for (int o = 0; o < 2; o++) {
            const float e = Y[2 * row + o] - Tg[2 * row + o], w = o ? w_rate : 1.0f;
            dy[r][o] = 2.0f * w * e * invB;
            lsum += w * e * e * invB;
        }
    }
    // head: D3 = (dy W3) * silu'(z3); dW3 = sum dy a3; db3 = sum dy
    float d[2][8][4], gw[2][16];
#pragma unroll
    for (int q = 0; q < 16; q++) gw[0][q] = gw[1][q] = 0.f;
#pragma unroll
    for (int m = 0; m < 2; m++)
#pragma unroll
        for (int nt = 0; nt < 8; nt++)
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int r = 2 * m + h, c = 8 * nt + 2 * t;
                const long long row = quad_row(row0, r, g);
                const float2 z = *reinterpret_cast<const float2 *>(&Z.z[2][row * kMlpH + c]);
                const float zz[2] = {z.x, z.y};
#pragma unroll
                for (int e = 0; e < 2; e++) {
                    const float a = silu(zz[e]);
                    const float da = dy[r][0] * S.W3[c + e] + dy[r][1] * S.W3[kMlpH + c + e];
                    d[m][nt][2 * h + e] = da * dsilu(zz[e]);
                    gw[0][2 * nt + e] = fmaf(dy[r][0], a, gw[0][2 * nt + e]);
                    gw[1][2 * nt + e] = fmaf(dy[r][1], a, gw[1][2 * nt + e]);
                }
                *reinterpret_cast<float2 *>(&D.z[2][row * kMlpH + c]) = make_float2(d[m][nt][2 * h], d[m][nt][2 * h + 1]);
            }
    // this warp's partial sums of the head gradient and the loss (summed over
    // warps in a fixed order by k_mlp_reduce: training is deterministic)
    float *ph = head + (row0 / 32) * kHeadPartial;
#pragma unroll
    for (int o = 0; o < 2; o++)
#pragma unroll
        for (int q = 0; q < 16; q++) {
            float v = gw[o][q];
            v += __shfl_xor_sync(0xffffffffu, v, 4);
            v += __shfl_xor_sync(0xffffffffu, v, 8);
            v += __shfl_xor_sync(0xffffffffu, v, 16);
            if (g == 0) ph[o * kMlpH + 8 * (q >> 1) + 2 * t + (q & 1)] = v;
        }
    // db3 and the loss: the quad's lanes hold the same rows; count lane t == 0
#pragma unroll
    for (int o = 0; o < 2; o++) {
        float v = t == 0 ? dy[0][o] + dy[1][o] + dy[2][o] + dy[3][o] : 0.f;
#pragma unroll
        for (int sh = 16; sh > 0; sh >>= 1) v += __shfl_xor_sync(0xffffffffu, v, sh);
        if (lane == 0) ph[2 * kMlpH + o] = v;
    }
    lsum = t == 0 ? lsum : 0.f;
#pragma unroll
    for (int sh = 16; sh > 0; sh >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, sh);
    if (lane == 0) ph[2 * kMlpH + 2] = lsum;
    // D2 = (D3 W2) * silu'(z2), D1 = (D2 W1) * silu'(z1), on the tensor
    // cores, one m-tile at a time
    uint32_t A[4][4];
    float acc[8][4];
    auto ident = [](float a, float b) { return pack_bf16(a, b); };
#pragma unroll
    for (int m = 0; m < 2; m++)
#pragma unroll
        for (int l = 1; l >= 0; l--) {
            mlp_repack(d[m], A, ident);
            mlp_layer(l == 1 ? S.W2T : S.W1T, nullptr, A, acc);
#pragma unroll
            for (int nt = 0; nt < 8; nt++)
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const long long row = quad_row(row0, 2 * m + h, g);
                    const int c = 8 * nt + 2 * t;
                    const float2 z = *reinterpret_cast<const float2 *>(&Z.z[l][row * kMlpH + c]);
                    d[m][nt][2 * h] = acc[nt][2 * h] * dsilu(z.x);
                    d[m][nt][2 * h + 1] = acc[nt][2 * h + 1] * dsilu(z.y);
                    *reinterpret_cast<float2 *>(&D.z[l][row * kMlpH + c]) =
                        make_float2(d[m][nt][2 * h], d[m][nt][2 * h + 1]);
                }
        }
}

// dW_l[j][k] = sum_rows D_{l+1}[row][j] in_l[row][k], db_l[j] = sum_rows D;
// in_0 = X (K = 2), in_l = bf16(silu(Z_l)) as the forward fed the tensor
// cores.  blockIdx.y = l; blocks stride over 64-row chunks staged in shared
// memory; each thread owns a 4 x 4 tile of (j, k), two float4 loads per row.
// Each block writes its partial sums (packed parameter order, layers 0-2)
// to its own row of `part`; k_mlp_reduce adds the rows in a fixed order.
constexpr int kWgRows = 64;
constexpr int kWgBlocks = 64;
__global__ void __launch_bounds__(256) k_mlp_wgrad(long long B, const float *__restrict__ X, MlpZ Z, MlpZ D,
                                                   float *__restrict__ part)
{
    float *grad = part + (size_t)blockIdx.x * kOffW3;
    __shared__ __align__(16) float Ds[kWgRows][kMlpH];
    __shared__ __align__(16) float As[kWgRows][kMlpH];
    const int l = blockIdx.y, kin = l == 0 ? 2 : kMlpH;
    const float *Dl = D.z[l];
    const int j0 = 4 * (threadIdx.x >> 4), k0 = 4 * (threadIdx.x & 15);
    float acc[4][4], bacc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < 4; b++) acc[a][b] = 0.f;
    for (long long r0 = (long long)blockIdx.x * kWgRows; r0 < B; r0 += (long long)gridDim.x * kWgRows) {
        __syncthreads();
        for (int idx = threadIdx.x; idx < kWgRows * kMlpH / 4; idx += blockDim.x) {
            const int r = idx / (kMlpH / 4), c = 4 * (idx % (kMlpH / 4));
            const long long row = r0 + r;
            float4 dv = make_float4(0.f, 0.f, 0.f, 0.f), av = dv;
            if (row < B) {
                dv = *reinterpret_cast<const float4 *>(&Dl[row * kMlpH + c]);
                if (l == 0) {
                    if (c == 0) av = make_float4(X[2 * row], X[2 * row + 1], 0.f, 0.f);
                } else {
                    const float4 z = *reinterpret_cast<const float4 *>(&Z.z[l - 1][row * kMlpH + c]);
                    const uint32_t a01 = silu2_bf16(z.x, z.y), a23 = silu2_bf16(z.z, z.w);
                    av = make_float4(bf16_lo(a01), bf16_hi(a01), bf16_lo(a23), bf16_hi(a23));
                }
            }
            *reinterpret_cast<float4 *>(&Ds[r][c]) = dv;
            *reinterpret_cast<float4 *>(&As[r][c]) = av;
        }
        __syncthreads();
#pragma unroll 4
        for (int r = 0; r < kWgRows; r++) {
            const float4 d = *reinterpret_cast<const float4 *>(&Ds[r][j0]);
            const float4 a = *reinterpret_cast<const float4 *>(&As[r][k0]);
            const float dd[4] = {d.x, d.y, d.z, d.w}, aa[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
            for (int p = 0; p < 4; p++) {
                bacc[p] += dd[p];
#pragma unroll
                for (int q = 0; q < 4; q++) acc[p][q] = fmaf(dd[p], aa[q], acc[p][q]);
            }
        }
    }
    const int offW = l == 0 ? kOffW0 : (l == 1 ? kOffW1 : kOffW2);
    const int offB = l == 0 ? kOffB0 : (l == 1 ? kOffB1 : kOffB2);
#pragma unroll
    for (int p = 0; p < 4; p++) {
#pragma unroll
        for (int q = 0; q < 4; q++)
            if (k0 + q < kin) grad[offW + (j0 + p) * kin + k0 + q] = acc[p][q];
        if (k0 == 0) grad[offB + j0 + p] = bacc[p];
    }
}

// the gradient and the loss from the partial sums, in a fixed order:
// layers 0-2 over the wgrad blocks, the head and the loss over the warps
__global__ void k_mlp_reduce(const float *__restrict__ part, int nblk, const float *__restrict__ head, int nwarp,
                             float *__restrict__ grad, float *loss)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kOffW3) {
        float s = 0.f;
        for (int b = 0; b < nblk; b++) s += part[(size_t)b * kOffW3 + i];
        grad[i] = s;
    } else if (i < kMlpNParams + 1) {
        const int q = i - kOffW3;  // 0..129: dW3, db3; 130: the loss
        float s = 0.f;
        for (int w = 0; w < nwarp; w++) s += head[(size_t)w * kHeadPartial + q];
        if (i < kMlpNParams) grad[i] = s;
        else *loss = s;
    }
}

__global__ void k_mlp_adam(float *__restrict__ P, float *__restrict__ M, float *__restrict__ V,
                           float *__restrict__ G, MlpImage *img, const int *it, MlpAdam a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kMlpNParams) return;
    const int k = *it;
    const double frac = a.iters > 1 ? fmin((double)k / (double)(a.iters - 1), 1.0) : 1.0;
    const double lr = a.lr_final + 0.5 * (a.lr0 - a.lr_final) * (1.0 + cos(3.14159265358979323846 * frac));
    const float g = G[i];
    G[i] = 0.f;
    const float m = a.beta1 * M[i] + (1.0f - a.beta1) * g;
    const float v = a.beta2 * V[i] + (1.0f - a.beta2) * g * g;
    M[i] = m;
    V[i] = v;
    const double c1 = 1.0 - pow((double)a.beta1, (double)(k + 1)), c2 = 1.0 - pow((double)a.beta2, (double)(k + 1));
    const float p = P[i] - (float)(lr * ((double)m / c1) / (sqrt((double)v / c2) + a.eps));
    P[i] = p;
    image_put(img, i, p);
}

__global__ void k_mlp_tick(int *it, float *loss, float *loss_last)
{
    *loss_last = *loss;
    *loss = 0.f;
    *it += 1;
}

// raw network on normalised inputs (testing): one warp per 32 rows
__global__ void __launch_bounds__(128) k_mlp_eval(const MlpImage *img, long long n, const float *__restrict__ X,
                                                  float *__restrict__ Y)
{
    extern __shared__ __align__(16) unsigned char smem[];
    mlp_stage(smem, img, kMlpStageBytes);
    __syncthreads();
    const MlpImage &S = *reinterpret_cast<const MlpImage *>(smem);
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (!__any_sync(0xffffffffu, i < n)) return;
    const bool ok = i < n;
    float y0, y1;
    mlp_eval_warp(S, ok ? X[2 * i] : 0.f, ok ? X[2 * i + 1] : 0.f, y0, y1);
    if (ok) {
        Y[2 * i] = y0;
        Y[2 * i + 1] = y1;
    }
}

// what the Monte Carlo uses for (chi, r): the network inside its range,
// the tables (of the simulation's precision) outside (r == nullptr: G;
// else the energy fraction)
template <typename R>
__global__ void __launch_bounds__(128) k_qed_eval_surr(const MlpImage *img, MlpNorm nrm, QedTables T, int p,
                                                       long long n, const double *__restrict__ chi,
                                                       const double *__restrict__ r, double *__restrict__ out)
{
    extern __shared__ __align__(16) unsigned char smem[];
    mlp_stage(smem, img, kMlpStageBytes);
    __syncthreads();
    const MlpImage &S = *reinterpret_cast<const MlpImage *>(smem);
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (!__any_sync(0xffffffffu, i < n)) return;
    const bool ok = i < n;
    const double c = ok ? chi[i] : 1.0, rv = ok && r ? r[i] : 0.5;
    double lnchi;
    const bool inr = ok && mlp_in_range(nrm, c, lnchi);
    float x0 = 0.f, x1 = 0.f, y0 = 0.f, y1 = 0.f;
    if (inr) mlp_inputs(nrm, p, lnchi, rv, x0, x1);
    if (__any_sync(0xffffffffu, inr)) mlp_eval_warp_sparse(S, inr, x0, x1, y0, y1);
    if (!ok) return;
    if constexpr (sizeof(R) == 4) {  // in FP32, as the FP32 pushes evaluate it
        const float cf = (float)c, rf = (float)rv;
        if (r) out[i] = inr ? mlp_fraction_f32(p, y0, rf) : qed_sample_f32(T, p, cf, rf);
        else out[i] = inr ? mlp_rate_f32(nrm, p, cf, y1) : qed_rate_f32(T, p, cf);
    } else {
        if (r) out[i] = inr ? mlp_fraction(p, y0, rv) : qed_sample<R>(T, p, c, rv);
        else out[i] = inr ? mlp_rate(nrm, p, c, y1) : qed_rate<R>(T, p, c);
    }
}

// errors of the network against the FP64 tables on a (ln chi, r) grid of
// cell midpoints: acc[0] = max |d ln G|, acc[1] = max |d s|, acc[2] = sum d s^2
__global__ void __launch_bounds__(128) k_mlp_validate(const MlpImage *img, MlpNorm nrm, QedTables T, int p, int nc,
                                                      int nr, double *acc)
{
    extern __shared__ __align__(16) unsigned char smem[];
    mlp_stage(smem, img, kMlpStageBytes);
    __syncthreads();
    const MlpImage &S = *reinterpret_cast<const MlpImage *>(smem);
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n = (long long)nc * nr;
    if (!__any_sync(0xffffffffu, i < n)) return;
    const bool ok = i < n;
    const int ic = ok ? (int)(i / nr) : 0, jr = ok ? (int)(i % nr) : 0;
    const double lnchi = nrm.lnchi_lo + (ic + 0.5) / nc * (nrm.lnchi_hi - nrm.lnchi_lo);
    const double r = (jr + 0.5) / nr;
    float x0, x1, y0, y1;
    mlp_inputs(nrm, p, lnchi, r, x0, x1);
    mlp_eval_warp(S, x0, x1, y0, y1);
    if (!ok) return;
    const double chi = exp(lnchi);
    const double s_tab = cbrt(qed_sample<double>(T, p, chi, p == QED_PAIR ? fmin(r, 1.0 - r) : r));
    const double es = fabs((double)y0 - s_tab);
    const double eg = fabs((double)fmaf(nrm.sd, y1, nrm.mu) - qed_lnG_table<double>(T, p, (lnchi - T.lnchi0) / T.dlnchi));
    // non-negative doubles order as their bit patterns
    atomicMax(reinterpret_cast<unsigned long long *>(&acc[0]), (unsigned long long)__double_as_longlong(eg));
    atomicMax(reinterpret_cast<unsigned long long *>(&acc[1]), (unsigned long long)__double_as_longlong(es));
    atomicAdd(&acc[2], es * es);
    const double ft = s_tab * s_tab * s_tab;
    atomicAdd(&acc[4 + 2 * ic], mlp_fraction(p, y0, r));
    atomicAdd(&acc[5 + 2 * ic], p == QED_PAIR && r > 0.5 ? 1.0 - ft : ft);
}

int div_up_i(long long a, int b) { return (int)((a + b - 1) / b); }

}  // namespace

void launch_mlp_image(const float *P, MlpImage *img, cudaStream_t st)
{
    note_launch();
    k_mlp_image<<<div_up_i(kMlpNParams, 256), 256, 0, st>>>(P, img);
}

void launch_mlp_forward(const MlpImage *img, long long B, const float *X, const MlpZ &Z, float *Y, cudaStream_t st)
{
    note_launch();
    k_mlp_fwd<<<div_up_i(B, 128), 128, kMlpStageBytes, st>>>(img, B, X, Z, Y);
}

size_t mlp_partial_floats(long long B) { return (size_t)kWgBlocks * kOffW3 + (size_t)(B / 32) * kHeadPartial; }

void launch_mlp_backward(const MlpImage *img, long long B, const float *X, const float *Tg, const float *Y,
                         const MlpZ &Z, const MlpZ &D, float *partials, float *grad, float w_rate, float *loss,
                         cudaStream_t st)
{
    float *part = partials, *head = partials + (size_t)kWgBlocks * kOffW3;
    note_launch(3);
    k_mlp_bwd<<<div_up_i(B, 128), 128, kMlpTrainStageBytes, st>>>(img, B, Tg, Y, Z, D, head, w_rate);
    const int nb = std::min(div_up_i(B, kWgRows), kWgBlocks);
    k_mlp_wgrad<<<dim3(nb, 3), 256, 0, st>>>(B, X, Z, D, part);
    k_mlp_reduce<<<div_up_i(kMlpNParams + 1, 256), 256, 0, st>>>(part, nb, head, (int)(B / 32), grad, loss);
}

void mlp_train_iteration(MlpNet &net, MlpScratch &S, const QedTables &T, int p, const uint32_t *key,
                         const MlpAdam &a, float w_rate, cudaStream_t st)
{
    note_launch();
    k_mlp_data<<<div_up_i(S.B, 256), 256, 0, st>>>(T, p, net.nrm, key[0], key[1], S.it, S.B, S.X, S.T);
    launch_mlp_forward(net.img, S.B, S.X, S.Z, S.Y, st);
    launch_mlp_backward(net.img, S.B, S.X, S.T, S.Y, S.Z, S.D, S.partials, net.G, w_rate, S.loss, st);
    note_launch(2);
    k_mlp_adam<<<div_up_i(kMlpNParams, 256), 256, 0, st>>>(net.P, net.M, net.V, net.G, net.img, S.it, a);
    k_mlp_tick<<<1, 1, 0, st>>>(S.it, S.loss, S.loss + 1);
}

void launch_mlp_eval(const MlpImage *img, long long n, const float *X, float *Y, cudaStream_t st)
{
    note_launch();
    k_mlp_eval<<<div_up_i(n, 128), 128, kMlpStageBytes, st>>>(img, n, X, Y);
}

void launch_qed_eval_surr(const MlpImage *img, const MlpNorm &nrm, const QedTables &T, bool f64, int p, long long n,
                          const double *chi, const double *r, double *out, cudaStream_t st)
{
    note_launch();
    if (f64) k_qed_eval_surr<double><<<div_up_i(n, 128), 128, kMlpStageBytes, st>>>(img, nrm, T, p, n, chi, r, out);
    else k_qed_eval_surr<float><<<div_up_i(n, 128), 128, kMlpStageBytes, st>>>(img, nrm, T, p, n, chi, r, out);
}

void launch_mlp_validate(const MlpImage *img, const MlpNorm &nrm, const QedTables &T, int p, int nc, int nr,
                         double *acc, cudaStream_t st)
{
    note_launch();
    k_mlp_validate<<<div_up_i((long long)nc * nr, 128), 128, kMlpStageBytes, st>>>(img, nrm, T, p, nc, nr, acc);
}

}  // namespace pic
