// push.cu -- the particle half of the split PIC step (Sec. II.C-II.F):
// half drift to x^{n+1/2}, gather of E and B there (Eq. (19) with the W_2
// weights), relativistic Boris push (Eqs. (13)-(16)), drift to x^{n+1}
// (stored) and x^{n+3/2} (deposit end point), Esirkepov charge-conserving
// current on the straight path x^{n+1/2} -> x^{n+3/2} (Eqs. (20)-(22)),
// particle boundary conditions.
//
// Two precision forms share the arithmetic:
//  * FP32 cell+offset: integer cell and FP32 offset in [0,1) per axis.  A
//    drift adds delta = (dt/2) v / dx to the offset; crossing a face moves
//    the cell by one and the offset by one (exact: |delta| < 1/2).  The
//    periodic wrap is an integer operation, so the deposit end point of one
//    step and the deposit start point of the next are bit-identical.
//  * FP64 plain: absolute FP64 positions, FP64 fields and push.
#include <cstdio>

#include "push_dev.cuh"

namespace pic {

long long g_launches = 0;


// ---------------------------------------------------------------------
// FP32 cell+offset push
// ---------------------------------------------------------------------
template <int DIM, int ORDER = 2>
__device__ __forceinline__ void push_one_f32(const PartF32 &P, long long p, float *__restrict__ F, const Grid &g,
                                             const PushConst &pc, int *err, double *e_abs);

template <int DIM, int ORDER>
__global__ void __launch_bounds__(256) k_push_f32(PartF32 P, float *__restrict__ F, Grid g, PushConst pc,
                                                  int *err, double *e_abs)
{
    long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= *P.dn) return;
    push_one_f32<DIM, ORDER>(P, p, F, g, pc, err, e_abs);
}

// the particles of a list (the tiled push's deferred ones), grid-stride
template <int DIM>
__global__ void __launch_bounds__(256) k_push_list_f32(PartF32 P, const uint32_t *__restrict__ list,
                                                       const uint32_t *__restrict__ count, float *__restrict__ F,
                                                       Grid g, PushConst pc, int *err, double *e_abs)
{
    const uint32_t n = *count;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        push_one_f32<DIM>(P, list[i], F, g, pc, err, e_abs);
}

// one particle: half drift, gather (HBM), Boris, drifts, Esirkepov (global
// atomics), boundaries; shape order ORDER (W_2 or W_4 of Sec. II.D)
template <int DIM, int ORDER>
__device__ __forceinline__ void push_one_f32(const PartF32 &P, long long p, float *__restrict__ F, const Grid &g,
                                             const PushConst &pc, int *err, double *e_abs)
{
    uint32_t pc0 = P.cell[p];
    if (pc0 == kDead) return;
    int c[3];
    unpack_cell(g, pc0, c[0], c[1], c[2]);
    float o[3] = {P.off[0][p], DIM >= 2 ? P.off[1][p] : 0.f, DIM >= 3 ? P.off[2][p] : 0.f};
    float ux = P.u[0][p], uy = P.u[1][p], uz = P.u[2][p];
    float u[3];
    // x^{n+1/2}
    float ig = inv_gamma(ux, uy, uz);
    u[0] = ux; u[1] = uy; u[2] = uz;
#pragma unroll
    for (int d = 0; d < DIM; d++) drift_f32(c[d], o[d], pc.hdx_f[d] * u[d] * ig);
    int ch[3] = {c[0], c[1], c[2]};
    float oh[3] = {o[0], o[1], o[2]};
    // gather
    int icn[3] = {0, 0, 0}, ich[3] = {0, 0, 0};
    float wn[3][ORDER + 1], wh[3][ORDER + 1];
#pragma unroll
    for (int d = 0; d < DIM; d++) axis_w_f32<ORDER>(c[d], o[d], icn[d], wn[d], ich[d], wh[d]);
    float eb[6];
    gather<float, DIM, ORDER>(F, g, icn, wn, ich, wh, eb);
    // Boris
    const float k = pc.qmdt2_f;
    lorentz<float>(pc.pusher, ux, uy, uz, k * eb[0], k * eb[1], k * eb[2], k * eb[3], k * eb[4], k * eb[5]);
    float ig1 = inv_gamma(ux, uy, uz);
    u[0] = ux; u[1] = uy; u[2] = uz;
    // x^{n+1}, then x^{n+3/2}
#pragma unroll
    for (int d = 0; d < DIM; d++) drift_f32(c[d], o[d], pc.hdx_f[d] * u[d] * ig1);
    int c1[3] = {c[0], c[1], c[2]};
    float o1[3] = {o[0], o[1], o[2]};
#pragma unroll
    for (int d = 0; d < DIM; d++) drift_f32(c[d], o[d], pc.hdx_f[d] * u[d] * ig1);
    // Esirkepov on x^{n+1/2} -> x^{n+3/2}
    float S0[3][ORDER + 3], dS[3][ORDER + 3];
    int base[3] = {0, 0, 0};
    bool ok = true;
#pragma unroll
    for (int d = 0; d < DIM; d++) {
        int i0, i1;
        float w0[ORDER + 1], w1[ORDER + 1];
        axis_wn_f32<ORDER>(ch[d], oh[d], i0, w0);
        axis_wn_f32<ORDER>(c[d], o[d], i1, w1);
        ok &= window_n<float, ORDER>(i0, w0, i1, w1, S0[d], dS[d]);
        base[d] = i0 - ORDER / 2 - 1;
    }
    // a non-finite momentum (a NaN or infinite field) is reported and the particle
    // removed before anything uses its position: NaN positions would give no valid
    // cell or node index to the gather, the deposit or the diagnostics (and would
    // otherwise be reported as a Courant violation)
    if (!isfinite(ux + uy + uz)) {
        atomicOr(err, ERR_NONFINITE);
        P.cell[p] = kDead;
        return;
    }
    if (!ok) {
        atomicOr(err, ERR_CFL);
        return;
    }
    const float cJ[3] = {pc.cJ_f[0], pc.cJ_f[1], pc.cJ_f[2]};
    const float qw = pc.qw_f;
    deposit_global<float, DIM, ORDER>(F, g, base, S0, dS, cJ, qw * uy * ig1, qw * uz * ig1);
    // boundaries
    bool dead = false;
#pragma unroll
    for (int d = 0; d < DIM; d++) {
        if (g.bc[d] == PERIODIC) {
            if (c1[d] < 0) c1[d] += g.n[d];
            else if (c1[d] >= g.n[d]) c1[d] -= g.n[d];
        } else if (c1[d] < 0 || c1[d] >= g.n[d]) {
            dead = true;
        }
    }
    if (dead) {
        P.cell[p] = kDead;
        double uu = (double)ux * ux + (double)uy * uy + (double)uz * uz;
        atomicAdd(e_abs, pc.wmdV * uu / (sqrt(1.0 + uu) + 1.0));
    } else {
        P.cell[p] = pack_cell(g, c1[0], DIM >= 2 ? c1[1] : 0, DIM >= 3 ? c1[2] : 0);
    }
#pragma unroll
    for (int d = 0; d < DIM; d++) P.off[d][p] = o1[d];
    P.u[0][p] = ux;
    P.u[1][p] = uy;
    P.u[2][p] = uz;
}

// ---------------------------------------------------------------------
// FP64 plain push (absolute positions)
// ---------------------------------------------------------------------
template <int DIM, int ORDER>
__global__ void __launch_bounds__(256) k_push_f64(PartF64 P, double *__restrict__ F, Grid g, PushConst pc,
                                                  int *err, double *e_abs)
{
    long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= *P.dn) return;
    if (P.cell[p] == kDead) return;
    double x[3] = {P.x[0][p], DIM >= 2 ? P.x[1][p] : 0.0, DIM >= 3 ? P.x[2][p] : 0.0};
    double ux = P.u[0][p], uy = P.u[1][p], uz = P.u[2][p];
    double ig = inv_gamma(ux, uy, uz);
    double u[3] = {ux, uy, uz};
#pragma unroll
    for (int d = 0; d < DIM; d++) x[d] += pc.hdt * u[d] * ig;
    double xh[3] = {x[0], x[1], x[2]};
    int icn[3] = {0, 0, 0}, ich[3] = {0, 0, 0};
    double wn[3][ORDER + 1], wh[3][ORDER + 1];
#pragma unroll
    for (int d = 0; d < DIM; d++) axis_w_f64<ORDER>(x[d] / g.dx[d], icn[d], wn[d], ich[d], wh[d]);
    double eb[6];
    gather<double, DIM, ORDER>(F, g, icn, wn, ich, wh, eb);
    const double k = pc.qmdt2;
    lorentz<double>(pc.pusher, ux, uy, uz, k * eb[0], k * eb[1], k * eb[2], k * eb[3], k * eb[4], k * eb[5]);
    double ig1 = inv_gamma(ux, uy, uz);
    u[0] = ux; u[1] = uy; u[2] = uz;
#pragma unroll
    for (int d = 0; d < DIM; d++) x[d] += pc.hdt * u[d] * ig1;
    double x1[3] = {x[0], x[1], x[2]};
#pragma unroll
    for (int d = 0; d < DIM; d++) x[d] += pc.hdt * u[d] * ig1;
    double S0[3][ORDER + 3], dS[3][ORDER + 3];
    int base[3] = {0, 0, 0};
    bool ok = true;
#pragma unroll
    for (int d = 0; d < DIM; d++) {
        int i0, i1;
        double w0[ORDER + 1], w1[ORDER + 1];
        axis_wn_f64<ORDER>(xh[d] / g.dx[d], i0, w0);
        axis_wn_f64<ORDER>(x[d] / g.dx[d], i1, w1);
        ok &= window_n<double, ORDER>(i0, w0, i1, w1, S0[d], dS[d]);
        base[d] = i0 - ORDER / 2 - 1;
    }
    // a non-finite momentum (a NaN or infinite field) is reported and the particle
    // removed before anything uses its position: NaN positions would give no valid
    // cell or node index to the gather, the deposit or the diagnostics (and would
    // otherwise be reported as a Courant violation)
    if (!isfinite(ux + uy + uz)) {
        atomicOr(err, ERR_NONFINITE);
        P.cell[p] = kDead;
        return;
    }
    if (!ok) {
        atomicOr(err, ERR_CFL);
        return;
    }
    deposit_global<double, DIM, ORDER>(F, g, base, S0, dS, pc.cJ, pc.qw * uy * ig1, pc.qw * uz * ig1);
    bool dead = false;
    int cc[3] = {0, 0, 0};
#pragma unroll
    for (int d = 0; d < DIM; d++) {
        double L = (double)g.n[d] * g.dx[d];
        if (g.bc[d] == PERIODIC) {
            if (x1[d] < 0.0) x1[d] += L;
            if (x1[d] >= L) x1[d] -= L;
        } else if (x1[d] < 0.0 || x1[d] >= L) {
            dead = true;
        }
        int ci = (int)floor(x1[d] / g.dx[d]);
        cc[d] = ci < 0 ? 0 : (ci >= g.n[d] ? g.n[d] - 1 : ci);
    }
    if (dead) {
        P.cell[p] = kDead;
        double uu = ux * ux + uy * uy + uz * uz;
        atomicAdd(e_abs, pc.wmdV * uu / (sqrt(1.0 + uu) + 1.0));
    } else {
        P.cell[p] = pack_cell(g, cc[0], cc[1], cc[2]);
    }
#pragma unroll
    for (int d = 0; d < DIM; d++) P.x[d][p] = x1[d];
    P.u[0][p] = ux;
    P.u[1][p] = uy;
    P.u[2][p] = uz;
}

// ---------------------------------------------------------------------
// gather at the stored positions (inspection)
// ---------------------------------------------------------------------
template <int DIM, int ORDER>
__global__ void k_gather_f32(PartF32 P, const float *__restrict__ F, Grid g, double *out)
{
    long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= *P.dn) return;
    uint32_t cp = P.cell[p];
    if (cp == kDead) {
        for (int q = 0; q < 6; q++) out[6 * p + q] = 0.0;
        return;
    }
    int c[3];
    unpack_cell(g, cp, c[0], c[1], c[2]);
    int icn[3] = {0, 0, 0}, ich[3] = {0, 0, 0};
    float wn[3][ORDER + 1], wh[3][ORDER + 1];
#pragma unroll
    for (int d = 0; d < DIM; d++) axis_w_f32<ORDER>(c[d], P.off[d][p], icn[d], wn[d], ich[d], wh[d]);
    float eb[6];
    gather<float, DIM, ORDER>(F, g, icn, wn, ich, wh, eb);
    for (int q = 0; q < 6; q++) out[6 * p + q] = eb[q];
}

template <int DIM, int ORDER>
__global__ void k_gather_f64(PartF64 P, const double *__restrict__ F, Grid g, double *out)
{
    long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= *P.dn) return;
    if (P.cell[p] == kDead) {
        for (int q = 0; q < 6; q++) out[6 * p + q] = 0.0;
        return;
    }
    int icn[3] = {0, 0, 0}, ich[3] = {0, 0, 0};
    double wn[3][ORDER + 1], wh[3][ORDER + 1];
#pragma unroll
    for (int d = 0; d < DIM; d++) axis_w_f64<ORDER>(P.x[d][p] / g.dx[d], icn[d], wn[d], ich[d], wh[d]);
    double eb[6];
    gather<double, DIM, ORDER>(F, g, icn, wn, ich, wh, eb);
    for (int q = 0; q < 6; q++) out[6 * p + q] = eb[q];
}

// ---------------------------------------------------------------------
// load: FP64 absolute positions -> layout (positions already validated)
// ---------------------------------------------------------------------
// a particle outside [0, L) on an active axis, or with a non-finite
// momentum, is not stored: the lowest such index goes to *bad
__device__ __forceinline__ bool load_ok(const double *const *xs, const double *ux, const double *uy,
                                        const double *uz, long long a, const Grid &g, unsigned long long *bad)
{
    bool ok = isfinite(ux[a]) && isfinite(uy[a]) && isfinite(uz[a]);
    for (int d = 0; d < g.dim; d++) {
        const double xv = xs[d][a];
        ok &= xv >= 0.0 && xv < g.n[d] * g.dx[d];  // false for NaN
    }
    if (!ok) atomicMin(bad, (unsigned long long)a);
    return ok;
}

__global__ void k_load_f32(PartF32 P, long long first, long long n, const double *x, const double *y,
                           const double *z, const double *ux, const double *uy, const double *uz, Grid g,
                           unsigned long long *bad)
{
    long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    long long p = first + a;
    const double *xs[3] = {x, y, z};
    if (!load_ok(xs, ux, uy, uz, a, g, bad)) return;
    int c[3] = {0, 0, 0};
    for (int d = 0; d < g.dim; d++) {
        double X = xs[d][a] / g.dx[d];
        double f = floor(X);
        int ci = (int)f;
        float o = (float)(X - f);
        if (o >= 1.0f) { o = 0.0f; ci += 1; }
        if (ci >= g.n[d]) {  // x rounded onto the upper face
            if (g.bc[d] == PERIODIC) ci -= g.n[d];
            else { ci = g.n[d] - 1; o = 0.99999994f; }
        }
        if (ci < 0) { ci = 0; o = 0.0f; }
        c[d] = ci;
        P.off[d][p] = o;
    }
    P.cell[p] = pack_cell(g, c[0], c[1], c[2]);
    P.u[0][p] = (float)ux[a];
    P.u[1][p] = (float)uy[a];
    P.u[2][p] = (float)uz[a];
}

__global__ void k_load_f64(PartF64 P, long long first, long long n, const double *x, const double *y,
                           const double *z, const double *ux, const double *uy, const double *uz, Grid g,
                           unsigned long long *bad)
{
    long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    long long p = first + a;
    const double *xs[3] = {x, y, z};
    if (!load_ok(xs, ux, uy, uz, a, g, bad)) return;
    int c[3] = {0, 0, 0};
    for (int d = 0; d < g.dim; d++) {
        double xv = xs[d][a];
        int ci = (int)floor(xv / g.dx[d]);
        c[d] = ci < 0 ? 0 : (ci >= g.n[d] ? g.n[d] - 1 : ci);
        P.x[d][p] = xv;
    }
    P.cell[p] = pack_cell(g, c[0], c[1], c[2]);
    P.u[0][p] = ux[a];
    P.u[1][p] = uy[a];
    P.u[2][p] = uz[a];
}

// readback: absolute FP64 positions and u
__global__ void k_unload_f32(PartF32 P, Grid g, double *x, double *y, double *z, double *ux, double *uy,
                             double *uz, uint8_t *alive)
{
    long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= *P.dn) return;
    uint32_t cp = P.cell[p];
    int c[3] = {0, 0, 0};
    bool live = cp != kDead;
    if (live) unpack_cell(g, cp, c[0], c[1], c[2]);
    double *xs[3] = {x, y, z};
    for (int d = 0; d < 3; d++) {
        if (!xs[d]) continue;
        xs[d][p] = d < g.dim ? ((double)c[d] + (double)P.off[d][p]) * g.dx[d] : 0.0;
    }
    if (ux) ux[p] = P.u[0][p];
    if (uy) uy[p] = P.u[1][p];
    if (uz) uz[p] = P.u[2][p];
    if (alive) alive[p] = live ? 1 : 0;
}

__global__ void k_unload_f64(PartF64 P, Grid g, double *x, double *y, double *z, double *ux, double *uy,
                             double *uz, uint8_t *alive)
{
    long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= *P.dn) return;
    double *xs[3] = {x, y, z};
    for (int d = 0; d < 3; d++) {
        if (!xs[d]) continue;
        xs[d][p] = d < g.dim ? P.x[d][p] : 0.0;
    }
    if (ux) ux[p] = P.u[0][p];
    if (uy) uy[p] = P.u[1][p];
    if (uz) uz[p] = P.u[2][p];
    if (alive) alive[p] = P.cell[p] != kDead ? 1 : 0;
}

// ---------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------
void launch_push_f32(const PartF32 &P, float *F, const Grid &g, const PushConst &pc, int *err, double *e_abs,
                     cudaStream_t st)
{
    if (P.n == 0) return;
    note_launch();
    int bs = 256, nb = div_up(P.n, bs);
    if (g.order == 4) {
        if (g.dim == 1) k_push_f32<1, 4><<<nb, bs, 0, st>>>(P, F, g, pc, err, e_abs);
        else if (g.dim == 2) k_push_f32<2, 4><<<nb, bs, 0, st>>>(P, F, g, pc, err, e_abs);
        else k_push_f32<3, 4><<<nb, bs, 0, st>>>(P, F, g, pc, err, e_abs);
        return;
    }
    if (g.dim == 1) k_push_f32<1, 2><<<nb, bs, 0, st>>>(P, F, g, pc, err, e_abs);
    else if (g.dim == 2) k_push_f32<2, 2><<<nb, bs, 0, st>>>(P, F, g, pc, err, e_abs);
    else k_push_f32<3, 2><<<nb, bs, 0, st>>>(P, F, g, pc, err, e_abs);
}

void launch_push_list_f32(const PartF32 &P, const uint32_t *list, const uint32_t *count, long long max_n, float *F,
                          const Grid &g, const PushConst &pc, int *err, double *e_abs, cudaStream_t st)
{
    if (max_n <= 0) return;
    note_launch();
    const int nb = (int)std::min<long long>(div_up(max_n, 256), 152LL * 8);
    if (g.dim == 1) k_push_list_f32<1><<<nb, 256, 0, st>>>(P, list, count, F, g, pc, err, e_abs);
    else if (g.dim == 2) k_push_list_f32<2><<<nb, 256, 0, st>>>(P, list, count, F, g, pc, err, e_abs);
    else k_push_list_f32<3><<<nb, 256, 0, st>>>(P, list, count, F, g, pc, err, e_abs);
}

void launch_push_f64(const PartF64 &P, double *F, const Grid &g, const PushConst &pc, int *err, double *e_abs,
                     cudaStream_t st)
{
    if (P.n == 0) return;
    note_launch();
    int bs = 256, nb = div_up(P.n, bs);
    if (g.order == 4) {
        if (g.dim == 1) k_push_f64<1, 4><<<nb, bs, 0, st>>>(P, F, g, pc, err, e_abs);
        else if (g.dim == 2) k_push_f64<2, 4><<<nb, bs, 0, st>>>(P, F, g, pc, err, e_abs);
        else k_push_f64<3, 4><<<nb, bs, 0, st>>>(P, F, g, pc, err, e_abs);
        return;
    }
    if (g.dim == 1) k_push_f64<1, 2><<<nb, bs, 0, st>>>(P, F, g, pc, err, e_abs);
    else if (g.dim == 2) k_push_f64<2, 2><<<nb, bs, 0, st>>>(P, F, g, pc, err, e_abs);
    else k_push_f64<3, 2><<<nb, bs, 0, st>>>(P, F, g, pc, err, e_abs);
}

void launch_gather_f32(const PartF32 &P, const float *F, const Grid &g, double *out, cudaStream_t st)
{
    if (P.n == 0) return;
    note_launch();
    int bs = 256, nb = div_up(P.n, bs);
    if (g.order == 4) {
        if (g.dim == 1) k_gather_f32<1, 4><<<nb, bs, 0, st>>>(P, F, g, out);
        else if (g.dim == 2) k_gather_f32<2, 4><<<nb, bs, 0, st>>>(P, F, g, out);
        else k_gather_f32<3, 4><<<nb, bs, 0, st>>>(P, F, g, out);
        return;
    }
    if (g.dim == 1) k_gather_f32<1, 2><<<nb, bs, 0, st>>>(P, F, g, out);
    else if (g.dim == 2) k_gather_f32<2, 2><<<nb, bs, 0, st>>>(P, F, g, out);
    else k_gather_f32<3, 2><<<nb, bs, 0, st>>>(P, F, g, out);
}

void launch_gather_f64(const PartF64 &P, const double *F, const Grid &g, double *out, cudaStream_t st)
{
    if (P.n == 0) return;
    note_launch();
    int bs = 256, nb = div_up(P.n, bs);
    if (g.order == 4) {
        if (g.dim == 1) k_gather_f64<1, 4><<<nb, bs, 0, st>>>(P, F, g, out);
        else if (g.dim == 2) k_gather_f64<2, 4><<<nb, bs, 0, st>>>(P, F, g, out);
        else k_gather_f64<3, 4><<<nb, bs, 0, st>>>(P, F, g, out);
        return;
    }
    if (g.dim == 1) k_gather_f64<1, 2><<<nb, bs, 0, st>>>(P, F, g, out);
    else if (g.dim == 2) k_gather_f64<2, 2><<<nb, bs, 0, st>>>(P, F, g, out);
    else k_gather_f64<3, 2><<<nb, bs, 0, st>>>(P, F, g, out);
}

void launch_load_f32(const PartF32 &P, long long first, long long n, const double *const *xs,
                     const double *const *us, const Grid &g, unsigned long long *bad, cudaStream_t st)
{
    if (n == 0) return;
    note_launch();
    k_load_f32<<<div_up(n, 256), 256, 0, st>>>(P, first, n, xs[0], xs[1], xs[2], us[0], us[1], us[2], g, bad);
}

void launch_load_f64(const PartF64 &P, long long first, long long n, const double *const *xs,
                     const double *const *us, const Grid &g, unsigned long long *bad, cudaStream_t st)
{
    if (n == 0) return;
    note_launch();
    k_load_f64<<<div_up(n, 256), 256, 0, st>>>(P, first, n, xs[0], xs[1], xs[2], us[0], us[1], us[2], g, bad);
}

void launch_unload_f32(const PartF32 &P, const Grid &g, double *const *xs, double *const *us, uint8_t *alive,
                       cudaStream_t st)
{
    if (P.n == 0) return;
    note_launch();
    k_unload_f32<<<div_up(P.n, 256), 256, 0, st>>>(P, g, xs[0], xs[1], xs[2], us[0], us[1], us[2], alive);
}

void launch_unload_f64(const PartF64 &P, const Grid &g, double *const *xs, double *const *us, uint8_t *alive,
                       cudaStream_t st)
{
    if (P.n == 0) return;
    note_launch();
    k_unload_f64<<<div_up(P.n, 256), 256, 0, st>>>(P, g, xs[0], xs[1], xs[2], us[0], us[1], us[2], alive);
}

}  // namespace pic
