// push_tile_dev.cuh -- device helpers shared by the tiled pushes (2D in
// push_tile.cu, 3D in push_tile3d.cu).
#pragma once
#include "push_dev.cuh"
#include "push_tile.cuh"

namespace pic {

// shapes of the start (i0, w0) and end (i1, w1) points on the 4-node union
// window [u0, u0+3], u0 = min(i0, i1) - 1 (|i1 - i0| <= 1)
__device__ __forceinline__ int union4(int i0, const float *w0, int i1, const float *w1, float *S0, float *dS)
{
    const int u0 = min(i0, i1) - 1;
    const int o0 = i0 - 1 - u0, o1 = i1 - 1 - u0;  // each 0 or 1
#pragma unroll
    for (int k = 0; k < 4; k++) {
        float s0 = o0 ? (k >= 1 ? w0[k - 1] : 0.f) : (k <= 2 ? w0[k] : 0.f);
        float s1 = o1 ? (k >= 1 ? w1[k - 1] : 0.f) : (k <= 2 ? w1[k] : 0.f);
        S0[k] = s0;
        dS[k] = s1 - s0;
    }
    return u0;
}

// current into the shared box as 32-bit fixed point (integer shared-memory
// atomics are native; float ones are not).  A chunk has at most kChunk
// particles and each adds at most C = |q w| max(dx_d/dt) in magnitude to a
// node, so with 2^20/C units per C a node holds at most 2^30: no overflow.
// Rounding each value to the unit costs at most 2^-21 C per particle and
// node, below 1e-6 of the node's sum of |contributions| scale.
struct AccShared {
    int *base;  // component 0 at (ux, uy) of the window
    int cs, rs;
    float scale;
    __device__ __forceinline__ void add(int c, int a, int b, float v)
    {
        // no zero test: a branch per node costs more than the occasional
        // zero add, and the warp issues the atomic for its other lanes anyway
        atomicAdd(base + c * cs + b * rs + a, __float2int_rn(v * scale));
    }
};

// as AccShared with the values already in fixed-point units (the caller
// folded the scale into the deposit's coefficients: one multiply fewer per
// node)
struct AccSharedUnits {
    int *base;
    int cs, rs;
    __device__ __forceinline__ void add(int c, int a, int b, float v)
    {
        atomicAdd(base + c * cs + b * rs + a, __float2int_rn(v));
    }
};

// the whole warp on one window: each value summed over the 32 lanes (one
// warp reduction; 32 values of at most 2^20 units stay inside int32) and
// added once by the lead lane
struct AccWarpAll {
    int *base;
    int cs, rs;
    bool lead;
    __device__ __forceinline__ void add(int c, int a, int b, float v)
    {
        const int s = __reduce_add_sync(0xffffffffu, __float2int_rn(v));
        if (lead) atomicAdd(base + c * cs + b * rs + a, s);
    }
};

// Boris (Eqs. (13)-(16)) with the FP32 reciprocal square root and divide
// of the special-function unit (a few ulp, far inside the FP32 tolerance)
__device__ __forceinline__ void boris_fast(float &ux, float &uy, float &uz, float ex, float ey, float ez, float bx,
                                           float by, float bz)
{
    float umx = ux + ex, umy = uy + ey, umz = uz + ez;
    float ginv = rsqrtf(1.0f + umx * umx + umy * umy + umz * umz);
    float tx = bx * ginv, ty = by * ginv, tz = bz * ginv;
    float t2 = tx * tx + ty * ty + tz * tz;
    float upx = umx + (umy * tz - umz * ty);
    float upy = umy + (umz * tx - umx * tz);
    float upz = umz + (umx * ty - umy * tx);
    float f = __fdividef(2.0f, 1.0f + t2);
    float sx = tx * f, sy = ty * f, sz = tz * f;
    ux = umx + (upy * sz - upz * sy) + ex;
    uy = umy + (upz * sx - upx * sz) + ey;
    uz = umz + (upx * sy - upy * sx) + ez;
}

// the FP64 island above gamma ~ 1e4, out of line: a lane below it never
// issues its FP64 instructions (this GPU runs FP64 at 1/73 of FP32)
static __device__ __noinline__ float inv_gamma_island(float ux, float uy, float uz)
{
    const double d2 = (double)ux * ux + (double)uy * uy + (double)uz * uz;
    return (float)(1.0 / sqrt(1.0 + d2));
}

__device__ __forceinline__ float inv_gamma_fast(float ux, float uy, float uz)
{
    float u2 = ux * ux + uy * uy + uz * uz;
    if (u2 < 1e8f) return rsqrtf(1.0f + u2);
    return inv_gamma_island(ux, uy, uz);
}

}  // namespace pic
