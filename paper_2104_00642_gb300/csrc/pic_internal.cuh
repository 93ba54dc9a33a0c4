// pic_internal.cuh -- device-side layout and helpers of the GB300 PIC path.
//
// Field layout in HBM: one allocation per simulation holding the 9 field
// components (Ex..Bz, Jx..Jz) back to back, each a padded box
// [-G, N+G) per active axis (G = 4 ghost layers), x fastest, the x pitch
// rounded up to 32 elements so that rows start on 128-byte boundaries and
// the interior origin sits 16 bytes into the row.  Along periodic axes the
// ghosts always hold copies of their periodic images (the solver computes
// them directly); along absorbing axes the ghosts are zero except the one
// layer of tangential B kept by the Mur condition.
//
// Particles: structure of arrays.  FP32 form: packed cell index (u32,
// i | j << bx | k << (bx+by), 0xFFFFFFFF = dead), FP32 offset in [0,1) per
// active axis, FP32 u per component.  FP64 form: absolute FP64 position per
// active axis, FP64 u, plus the packed cell as sort key.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pic {

constexpr int kGhost = 4;
constexpr uint32_t kDead = 0xFFFFFFFFu;

enum Comp { EX = 0, EY, EZ, BX, BY, BZ, JX, JY, JZ, NCOMP };
enum Bc { PERIODIC = 0, ABSORB = 1 };

// device error flags (bit mask, read by the host once per pic_step)
// (ERR_QEDDT: a Method II acceptance probability above one -- the step is too
// long for that sampler)
enum ErrFlag : int { ERR_CFL = 1, ERR_NONFINITE = 2, ERR_CAPACITY = 4, ERR_TIMEOUT = 8, ERR_QEDDT = 16 };

struct Grid {
    int dim;
    int order;         // shape order of Sec. II.D: 2 (W_2, three nodes) or 4 (W_4, five nodes)
    int n[3];          // cells per axis (1 on inactive axes)
    int G[3];          // ghost layers per side (kGhost on active axes, 0 otherwise)
    int ext[3];        // n + 2G
    long long sy, sz;  // element strides of y and z
    long long vol;     // elements per component (padded, rounded to 64)
    long long origin;  // offset of interior (0,0,0)
    int bc[3];
    double dx[3];
    double dt;
    int bits[3];       // packed-cell bit widths
    int tile_log2[3];  // log2 of tile edge per axis
    int ntile[3];      // tiles per axis
    long long ntiles;
    // 1/dx precomputed on the host: FP64 arithmetic on GB300 runs at a small
    // fraction of the FP32 rate, so kernels take their constants ready-made
    float rdx_f[3];
    double rdx_d[3];
};

template <typename R>
__host__ __device__ inline R rdx(const Grid &g, int d);
template <>
__host__ __device__ inline float rdx<float>(const Grid &g, int d) { return g.rdx_f[d]; }
template <>
__host__ __device__ inline double rdx<double>(const Grid &g, int d) { return g.rdx_d[d]; }

// Device view of the laser entering through x-min.  The transverse profile
// is precomputed once (FP64 on the host, stored in the field precision):
// for c = 0 (B_z, from E_y) and c = 1 (B_y, from E_z) and every transverse
// node (j, k): amplitude A_c = a0 * amp * exp(-r^2/w^2) and phase offset
// PHI_c = -r^2/(2R) + Gouy.  The temporal factors of the four time points a
// Mur update needs are computed on the host per launch: tau_q = t -/+ dx/2
// at the new and old B times, env_q = exp(-2 ln2 ((tau_q - t_peak)/fwhm)^2)
// and ph0_q = (tau_q - t_peak) mod 2 pi, so a boundary thread evaluates
// E_y = A env sin(ph0 + PHI) (and E_z with cos for circular polarisation).
struct Laser {
    int on, pol;
    int nty, ntz;          // transverse profile size (n_y, n_z; 1 on inactive axes)
    const void *A[2], *PHI[2];
    double env[4], ph0[4];  // q = 0: t_new at -dx/2, 1: t_old at -dx/2, 2: t_new at +dx/2, 3: t_old at +dx/2
};

// staggering of component c along axis d: 1 = half node
__host__ __device__ inline int stag(int c, int d)
{
    int b = c % 3;
    return (c >= BX && c <= BZ) ? (d != b) : (d == b);
}

__host__ __device__ inline long long goff(const Grid &g, int i, int j, int k)
{
    return g.origin + (long long)k * g.sz + (long long)j * g.sy + i;
}

// packed cell helpers
__host__ __device__ inline uint32_t pack_cell(const Grid &g, int i, int j, int k)
{
    return (uint32_t)i | ((uint32_t)j << g.bits[0]) | ((uint32_t)k << (g.bits[0] + g.bits[1]));
}
__host__ __device__ inline void unpack_cell(const Grid &g, uint32_t c, int &i, int &j, int &k)
{
    i = (int)(c & ((1u << g.bits[0]) - 1u));
    j = g.bits[1] ? (int)((c >> g.bits[0]) & ((1u << g.bits[1]) - 1u)) : 0;
    k = g.bits[2] ? (int)((c >> (g.bits[0] + g.bits[1])) & ((1u << g.bits[2]) - 1u)) : 0;
}
__host__ __device__ inline uint32_t tile_of(const Grid &g, int i, int j, int k)
{
    return (uint32_t)(((long long)(k >> g.tile_log2[2]) * g.ntile[1] + (j >> g.tile_log2[1])) * g.ntile[0] +
                      (i >> g.tile_log2[0]));
}

// W_2 weights (the cell integral of the hat shape S_2, Sec. II.D): nodes
// ic-1, ic, ic+1 for a particle at delta = X - ic in [-1/2, 1/2).
template <typename R>
__device__ __forceinline__ void w2(R delta, R *w)
{
    const R h = R(0.5);
    R a = h - delta, b = h + delta;
    w[0] = h * a * a;
    w[1] = R(0.75) - delta * delta;
    w[2] = h * b * b;
}

// Boris rotation (Eqs. (13)-(16)); E, B already multiplied by q_m dt / 2.
template <typename R>
__device__ __forceinline__ void boris(R &ux, R &uy, R &uz, R ex, R ey, R ez, R bx, R by, R bz)
{
    R umx = ux + ex, umy = uy + ey, umz = uz + ez;
    R ginv = R(1) / sqrt(R(1) + umx * umx + umy * umy + umz * umz);
    R tx = bx * ginv, ty = by * ginv, tz = bz * ginv;
    R t2 = tx * tx + ty * ty + tz * tz;
    R upx = umx + (umy * tz - umz * ty);
    R upy = umy + (umz * tx - umx * tz);
    R upz = umz + (umx * ty - umy * tx);
    R f = R(2) / (R(1) + t2);
    R sx = tx * f, sy = ty * f, sz = tz * f;
    ux = umx + (upy * sz - upz * sy) + ex;
    uy = umy + (upz * sx - upx * sz) + ey;
    uz = umz + (upx * sy - upy * sx) + ez;
}

// Vay's pusher (J.-L. Vay, Phys. Plasmas 15, 056701 (2008)), the
// alternative Sec. II.C names for fields whose electric and magnetic forces
// nearly cancel; E, B already multiplied by q_m dt / 2.  A first half kick
// with the full Lorentz force at the old velocity, then the second half kick
// solved for the new gamma in closed form: a particle at the E x B drift
// velocity (E + v x B = 0) keeps its momentum exactly.
template <typename R>
__device__ __forceinline__ void vay(R &ux, R &uy, R &uz, R ex, R ey, R ez, R bx, R by, R bz)
{
    const R g0inv = R(1) / sqrt(R(1) + ux * ux + uy * uy + uz * uz);
    const R upx = ux + R(2) * ex + (uy * bz - uz * by) * g0inv;
    const R upy = uy + R(2) * ey + (uz * bx - ux * bz) * g0inv;
    const R upz = uz + R(2) * ez + (ux * by - uy * bx) * g0inv;
    const R tau2 = bx * bx + by * by + bz * bz;
    const R ust = upx * bx + upy * by + upz * bz;
    const R sigma = R(1) + upx * upx + upy * upy + upz * upz - tau2;
    // gamma_new^2 = (sigma + sqrt(sigma^2 + 4a)) / 2 with a = tau^2 + u*^2.
    // For sigma < 0 (tau^2 > 1 + |u'|^2: strong B, slow particle) the sum
    // cancels; the same value written as 2a / (sqrt(sigma^2 + 4a) - sigma)
    // has no cancellation
    const R a4 = R(4) * (tau2 + ust * ust);
    const R root = sqrt(sigma * sigma + a4);
    const R g1 = sqrt(sigma >= R(0) ? R(0.5) * (sigma + root) : R(0.5) * a4 / (root - sigma));
    const R tx = bx / g1, ty = by / g1, tz = bz / g1;
    const R sinv = R(1) / (R(1) + tx * tx + ty * ty + tz * tz);
    const R ut = upx * tx + upy * ty + upz * tz;
    ux = sinv * (upx + ut * tx + (upy * tz - upz * ty));
    uy = sinv * (upy + ut * ty + (upz * tx - upx * tz));
    uz = sinv * (upz + ut * tz + (upx * ty - upy * tx));
}

// the momentum update of a push: Boris (pusher 0) or Vay (pusher 1)
template <typename R>
__device__ __forceinline__ void lorentz(int pusher, R &ux, R &uy, R &uz, R ex, R ey, R ez, R bx, R by, R bz)
{
    if (pusher) vay<R>(ux, uy, uz, ex, ey, ez, bx, by, bz);
    else boris<R>(ux, uy, uz, ex, ey, ez, bx, by, bz);
}

// 1/gamma: FP32 below u^2 = 1e8 (gamma ~ 1e4), FP64 above, where 1 + u^2
// loses the 1 in FP32.
__device__ __forceinline__ float inv_gamma(float ux, float uy, float uz)
{
    float u2 = ux * ux + uy * uy + uz * uz;
    if (u2 < 1e8f) return 1.0f / sqrtf(1.0f + u2);
    double d2 = (double)ux * ux + (double)uy * uy + (double)uz * uz;
    return (float)(1.0 / sqrt(1.0 + d2));
}
__device__ __forceinline__ double inv_gamma(double ux, double uy, double uz)
{
    return 1.0 / sqrt(1.0 + ux * ux + uy * uy + uz * uz);
}

inline int div_up(long long a, long long b) { return (int)((a + b - 1) / b); }

// host-side count of kernel launches issued by the library (profiling)
extern long long g_launches;
inline void note_launch(long long n = 1) { g_launches += n; }

}  // namespace pic
