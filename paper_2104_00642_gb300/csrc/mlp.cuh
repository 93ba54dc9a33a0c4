// mlp.cuh -- the small network that stands in for the QED tables (Sec. IV
// rates of Eqs. (23)/(24) and their inverse CDFs) inside a trained chi range.
//
// One network per process, 2 -> 64 -> 64 -> 64 -> 2 with SiLU on the hidden
// layers.  Inputs: x0 = normalised ln chi, x1 = the tables' r coordinate of
// the CDF value r (mlp_rcoord).  Outputs: y0 = s = fraction^(1/3) at r,
// y1 = (ln G (+ 8/(3 chi) for pairs) - mu) / sd.
//
// Weights are BF16 (master copy FP32 during training), accumulation FP32.
// A warp evaluates 32 rows: the input layer (K = 2) runs on CUDA cores in
// FP32 so ln chi keeps its precision; the two 64 x 64 layers run on the
// tensor cores as mma.sync m16n8k16 BF16 with FP32 accumulators, whose
// output fragments are repacked in registers as the next layer's A
// fragments; the 64 -> 2 head runs in FP32 with a quad shuffle reduction.
#pragma once
#include <cuda_bf16.h>

#include <cstddef>
#include <cstdint>

namespace pic {

constexpr int kMlpH = 64;
constexpr int kMlpPitch = 36;  // u32 words per weight row (64 bf16 + 8 pad): conflict-free B-fragment loads
constexpr int kMlpNParams = kMlpH * 2 + kMlpH + 2 * (kMlpH * kMlpH + kMlpH) + 2 * kMlpH + 2;
// packed parameter vector: W0[64][2] b0[64] W1[64][64] b1[64] W2[64][64] b2[64] W3[2][64] b3[2]
constexpr int kOffW0 = 0, kOffB0 = 128, kOffW1 = 192, kOffB1 = kOffW1 + 4096, kOffW2 = kOffB1 + 64,
              kOffB2 = kOffW2 + 4096, kOffW3 = kOffB2 + 64, kOffB3 = kOffW3 + 128;
static_assert(kOffB3 + 2 == kMlpNParams, "parameter packing");

// Device image of one network.  The part before W1T is what a push kernel
// stages into shared memory; the transposes serve the backward pass.
struct MlpImage {
    uint32_t W1[kMlpH * kMlpPitch];  // bf16 pairs, row = output feature
    uint32_t W2[kMlpH * kMlpPitch];
    float W0[kMlpH * 2];  // bf16-rounded values, [out][in]
    float b0[kMlpH], b1[kMlpH], b2[kMlpH];
    float W3[2 * kMlpH];  // bf16-rounded values, [out][in]
    float b3[4];          // 2 used
    uint32_t W1T[kMlpH * kMlpPitch];  // row = input feature
    uint32_t W2T[kMlpH * kMlpPitch];
};
constexpr int kMlpStageBytes = (int)offsetof(MlpImage, W1T);
constexpr int kMlpTrainStageBytes = (int)sizeof(MlpImage);
static_assert(kMlpStageBytes % 16 == 0 && sizeof(MlpImage) % 16 == 0, "16-byte staging");

// per-layer row arrays [rows][64] (training: pre-activations or deltas)
struct MlpZ {
    float *z[3];
};

// normalisation of one network (host and device)
struct MlpNorm {
    double lnchi_lo, lnchi_hi;  // trained range of ln chi
    float x0a, x0b;             // x0 = x0a ln chi + x0b
    float mu, sd;               // ln G (reduced for pairs) = mu + sd y1
};

// copy `bytes` of an image from global into shared memory (whole block)
__device__ __forceinline__ void mlp_stage(void *dst, const void *src, int bytes)
{
    const int4 *s = reinterpret_cast<const int4 *>(src);
    int4 *d = reinterpret_cast<int4 *>(dst);
    for (int i = threadIdx.x; i < bytes / 16; i += blockDim.x) d[i] = s[i];
}

__device__ __forceinline__ float tanh_approx(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// SiLU z sigma(z) with sigma(z) = (1 + tanh(z/2)) / 2, and its derivative
__device__ __forceinline__ float silu(float z)
{
    const float h = 0.5f * z;
    return fmaf(h, tanh_approx(h), h);
}
__device__ __forceinline__ float dsilu(float z)
{
    const float h = 0.5f * z, t = tanh_approx(h);
    return fmaf(0.5f, t, 0.5f) + h * fmaf(-0.5f * t, t, 0.5f);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

// The hidden activations as the next layer's MMA takes them: SiLU of two
// pre-activations, as a BF16 pair.  t = tanh(z/2) is evaluated on the BF16
// pair of z/2 (tanh.approx.bf16x2: one special-function operation for both
// values, half the MUFU issue of two FP32 tanh -- the unit that bounds the
// evaluation), then silu = h + h t with h = z/2 in FP32, rounded to BF16
// once.  The BF16 t carries a relative error of a few 2^-9, the size of the
// BF16 rounding the activation gets anyway.
__device__ __forceinline__ uint32_t silu2_bf16(float z0, float z1)
{
    const float h0 = 0.5f * z0, h1 = 0.5f * z1;
    const uint32_t hp = pack_bf16(h0, h1);
    uint32_t tp;
    asm("tanh.approx.bf16x2 %0, %1;" : "=r"(tp) : "r"(hp));
    const float t0 = __uint_as_float(tp << 16), t1 = __uint_as_float(tp & 0xffff0000u);
    return pack_bf16(fmaf(h0, t0, h0), fmaf(h1, t1, h1));
}
__device__ __forceinline__ float bf16_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t v) { return __uint_as_float(v & 0xffff0000u); }

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// One 64 x 64 layer for one m-tile (16 rows) of the warp:
// acc[nt] = bias + A . W^T (W rows = output features, bf16 pairs at pitch
// kMlpPitch; b == nullptr: no bias).
// Fragment layout (m16n8k16, g = lane/4, t = lane%4): A k-tile kt holds
// rows g / g+8 at columns 16kt + 2t (+1) and 16kt + 8 + 2t (+1); the
// accumulator of n-tile nt holds rows g / g+8 at columns 8nt + 2t (+1).
// The warp's two m-tiles go through the network one after the other, so
// that only one tile's fragments (48 registers) are live at a time.
__device__ __forceinline__ void mlp_layer(const uint32_t *W, const float *b, const uint32_t (&A)[4][4],
                                          float (&acc)[8][4])
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int nt = 0; nt < 8; nt++) {
        const float c0 = b ? b[8 * nt + 2 * t] : 0.f, c1 = b ? b[8 * nt + 2 * t + 1] : 0.f;
        acc[nt][0] = c0;
        acc[nt][1] = c1;
        acc[nt][2] = c0;
        acc[nt][3] = c1;
    }
#pragma unroll
    for (int kt = 0; kt < 4; kt++) {
#pragma unroll
        for (int nt = 0; nt < 8; nt++) {
            const uint32_t *w = W + (8 * nt + g) * kMlpPitch + 8 * kt + t;
            mma_bf16(acc[nt], A[kt], w[0], w[4]);
        }
    }
}

// accumulator fragments of n-tiles 2kt, 2kt+1 -> A fragment of k-tile kt,
// each pair of values through f2 into a BF16 pair (silu2_bf16, or pack_bf16
// for the deltas of the backward pass)
template <typename Fn2>
__device__ __forceinline__ void mlp_repack(const float (&acc)[8][4], uint32_t (&A)[4][4], Fn2 f2)
{
#pragma unroll
    for (int kt = 0; kt < 4; kt++) {
        const float *lo = acc[2 * kt], *hi = acc[2 * kt + 1];
        A[kt][0] = f2(lo[0], lo[1]);
        A[kt][1] = f2(lo[2], lo[3]);
        A[kt][2] = f2(hi[0], hi[1]);
        A[kt][3] = f2(hi[2], hi[3]);
    }
}

// Forward pass of the warp's 32 rows.  Row index within the warp:
// rr = 16 m + 8 h + g; this thread supplies and receives the rows of its
// quad group g: x[2m+h][*] in, y[2m+h][*] out (identical on the quad's four
// lanes).  With STORE the pre-activations are stored at
// Z.z[l][(row0 + rr) * 64 + col] (training).
template <bool STORE = false>
__device__ __forceinline__ void mlp_forward_rows(const MlpImage &S, const float (&x)[4][2], float (&y)[4][2],
                                                 MlpZ Z = MlpZ{}, long long row0 = 0, int nm = 2)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    float ps[4][2];
#pragma unroll
    for (int r = 0; r < 4; r++) ps[r][0] = ps[r][1] = 0.f;
#pragma unroll 1
    for (int m = 0; m < nm; m++) {  // nm: m-tiles holding rows (warp-uniform)
        uint32_t A[4][4];
        float acc[8][4];
        const float xm[2][2] = {{m ? x[2][0] : x[0][0], m ? x[2][1] : x[0][1]},
                                {m ? x[3][0] : x[1][0], m ? x[3][1] : x[1][1]}};
        // input layer in FP32 on the CUDA cores
#pragma unroll
        for (int nt = 0; nt < 8; nt++) {
            const int c = 8 * nt + 2 * t;
            const float w00 = S.W0[2 * c], w01 = S.W0[2 * c + 1], w10 = S.W0[2 * c + 2], w11 = S.W0[2 * c + 3];
            const float c0 = S.b0[c], c1 = S.b0[c + 1];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                acc[nt][2 * h] = fmaf(w01, xm[h][1], fmaf(w00, xm[h][0], c0));
                acc[nt][2 * h + 1] = fmaf(w11, xm[h][1], fmaf(w10, xm[h][0], c1));
            }
        }
        auto store = [&](int l) {
            if constexpr (STORE) {
#pragma unroll
                for (int nt = 0; nt < 8; nt++)
#pragma unroll
                    for (int h = 0; h < 2; h++) {
                        const long long row = row0 + 16 * m + 8 * h + g;
                        *reinterpret_cast<float2 *>(&Z.z[l][row * kMlpH + 8 * nt + 2 * t]) =
                            make_float2(acc[nt][2 * h], acc[nt][2 * h + 1]);
                    }
            }
        };
        auto act = [](float a, float b) { return silu2_bf16(a, b); };
        store(0);
        mlp_repack(acc, A, act);
        mlp_layer(S.W1, S.b1, A, acc);
        store(1);
        mlp_repack(acc, A, act);
        mlp_layer(S.W2, S.b2, A, acc);
        store(2);
        // head in FP32
        float p[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
        for (int nt = 0; nt < 8; nt++)
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const int c = 8 * nt + 2 * t + (e & 1), h = e >> 1;
                const float a = silu(acc[nt][e]);
                p[h][0] = fmaf(a, S.W3[c], p[h][0]);
                p[h][1] = fmaf(a, S.W3[kMlpH + c], p[h][1]);
            }
#pragma unroll
        for (int h = 0; h < 2; h++) {
            if (m) {
                ps[2 + h][0] = p[h][0];
                ps[2 + h][1] = p[h][1];
            } else {
                ps[h][0] = p[h][0];
                ps[h][1] = p[h][1];
            }
        }
    }
#pragma unroll
    for (int r = 0; r < 4; r++)
#pragma unroll
        for (int o = 0; o < 2; o++) {
            float v = ps[r][o];
            v += __shfl_xor_sync(0xffffffffu, v, 1);
            v += __shfl_xor_sync(0xffffffffu, v, 2);
            y[r][o] = v + S.b3[o];
        }
}

// Warp-collective evaluation: every lane of the warp calls it with the
// inputs of its own row (any values on lanes whose result is unused).
__device__ __forceinline__ void mlp_eval_warp(const MlpImage &S, float x0, float x1, float &y0, float &y1)
{
    const int lane = threadIdx.x & 31, g = lane >> 2;
    float x[4][2], y[4][2];
#pragma unroll
    for (int r = 0; r < 4; r++) {
        const int src = 16 * (r >> 1) + 8 * (r & 1) + g;
        x[r][0] = __shfl_sync(0xffffffffu, x0, src);
        x[r][1] = __shfl_sync(0xffffffffu, x1, src);
    }
    mlp_forward_rows(S, x, y);
    const int mine = 2 * (lane >> 4) + ((lane >> 3) & 1), src = 4 * (lane & 7);
#pragma unroll
    for (int r = 0; r < 4; r++) {
        const float v0 = __shfl_sync(0xffffffffu, y[r][0], src), v1 = __shfl_sync(0xffffffffu, y[r][1], src);
        if (r == mine) {
            y0 = v0;
            y1 = v1;
        }
    }
}

// As mlp_eval_warp, for the lanes with need set only (others get nothing):
// the needing lanes' inputs are packed into the first rows, and when at most
// 16 lanes need the network the second m-tile is not computed (half the
// tensor-core and SiLU work of the warp).
__device__ __forceinline__ void mlp_eval_warp_sparse(const MlpImage &S, bool need, float x0, float x1, float &y0,
                                                     float &y1)
{
    const unsigned mask = __ballot_sync(0xffffffffu, need);
    const int k = __popc(mask);
    const int lane = threadIdx.x & 31, g = lane >> 2;
    float x[4][2], y[4][2];
#pragma unroll
    for (int r = 0; r < 4; r++) {
        const int row = 16 * (r >> 1) + 8 * (r & 1) + g;
        const unsigned src = __fns(mask, 0, row + 1);  // lane of the row-th needing lane
        const int sl = src < 32u ? (int)src : 0;
        x[r][0] = __shfl_sync(0xffffffffu, x0, sl);
        x[r][1] = __shfl_sync(0xffffffffu, x1, sl);
    }
    mlp_forward_rows(S, x, y, MlpZ{}, 0, (k + 15) >> 4);
    // this lane's row: its rank among the needing lanes
    const int q = __popc(mask & ((1u << lane) - 1u));
    const int mine = 2 * (q >> 4) + ((q >> 3) & 1), src = 4 * (q & 7);
#pragma unroll
    for (int r = 0; r < 4; r++) {
        const float v0 = __shfl_sync(0xffffffffu, y[r][0], src), v1 = __shfl_sync(0xffffffffu, y[r][1], src);
        if (r == mine) {
            y0 = v0;
            y1 = v1;
        }
    }
}

// Coordinates of the sample output.  Input x1 = 2 t - 1 with t the r-grid
// coordinate of the tables (emission t = 1 - sqrt(1 - r), dense toward the
// hard end; pairs t = sqrt(2 min(r, 1 - r)), the spectrum being symmetric).
// Output y0 = s = fraction^(1/3) itself: the fitted error is the absolute
// error of s, uniform over the spectrum (measured against log or relative
// coordinates, this one kept the hard end, which carries the energy, best).
__host__ __device__ __forceinline__ double mlp_rcoord(int process, double r)
{
    const double t = process == 0 ? 1.0 - sqrt(fmax(1.0 - r, 0.0)) : sqrt(2.0 * fmin(r, 1.0 - r));
    return 2.0 * t - 1.0;
}

}  // namespace pic
