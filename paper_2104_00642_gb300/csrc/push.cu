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

#include "push.cuh"

namespace pic {

long long g_launches = 0;

// ---------------------------------------------------------------------
// per-axis nearest node and W_2 weights
// ---------------------------------------------------------------------

// FP32 form: X = c + o
__device__ __forceinline__ void axis_w_f32(int c, float o, int &icn, float *wn, int &ich, float *wh)
{
    bool up = o >= 0.5f;
    icn = c + (up ? 1 : 0);
    w2<float>(up ? o - 1.0f : o, wn);
    ich = c;
    w2<float>(o - 0.5f, wh);
}

__device__ __forceinline__ void axis_wn_f32(int c, float o, int &icn, float *wn)
{
    bool up = o >= 0.5f;
    icn = c + (up ? 1 : 0);
    w2<float>(up ? o - 1.0f : o, wn);
}

// FP64 form: X = x / dx
__device__ __forceinline__ void axis_w_f64(double X, int &icn, double *wn, int &ich, double *wh)
{
    icn = (int)floor(X + 0.5);
    w2<double>(X - (double)icn, wn);
    ich = (int)floor(X);
    w2<double>(X - ((double)ich + 0.5), wh);
}

__device__ __forceinline__ void axis_wn_f64(double X, int &icn, double *wn)
{
    icn = (int)floor(X + 0.5);
    w2<double>(X - (double)icn, wn);
}

// Eq. (19): each component with its own staggered nearest node per axis
template <typename R, int DIM>
__device__ __forceinline__ void gather(const R *__restrict__ F, const Grid &g, const int *icn, const R (*wn)[3],
                                       const int *ich, const R (*wh)[3], R *eb)
{
#pragma unroll
    for (int c = 0; c < 6; c++) {
        int ic[3];
        const R *w[3];
        ic[0] = stag(c, 0) ? ich[0] : icn[0];
        w[0] = stag(c, 0) ? wh[0] : wn[0];
        ic[1] = DIM >= 2 ? (stag(c, 1) ? ich[1] : icn[1]) : 0;
        w[1] = DIM >= 2 ? (stag(c, 1) ? wh[1] : wn[1]) : nullptr;
        ic[2] = DIM >= 3 ? (stag(c, 2) ? ich[2] : icn[2]) : 0;
        w[2] = DIM >= 3 ? (stag(c, 2) ? wh[2] : wn[2]) : nullptr;
        const R *Fc = F + (long long)c * g.vol;
        R acc = 0;
        if (DIM == 1) {
            long long o = goff(g, ic[0] - 1, 0, 0);
#pragma unroll
            for (int a = 0; a < 3; a++) acc += w[0][a] * __ldg(Fc + o + a);
        } else if (DIM == 2) {
#pragma unroll
            for (int b = 0; b < 3; b++) {
                long long o = goff(g, ic[0] - 1, ic[1] - 1 + b, 0);
                R r = 0;
#pragma unroll
                for (int a = 0; a < 3; a++) r += w[0][a] * __ldg(Fc + o + a);
                acc += w[1][b] * r;
            }
        } else {
#pragma unroll
            for (int cc = 0; cc < 3; cc++) {
                R r2 = 0;
#pragma unroll
                for (int b = 0; b < 3; b++) {
                    long long o = goff(g, ic[0] - 1, ic[1] - 1 + b, ic[2] - 1 + cc);
                    R r = 0;
#pragma unroll
                    for (int a = 0; a < 3; a++) r += w[0][a] * __ldg(Fc + o + a);
                    r2 += w[1][b] * r;
                }
                acc += w[2][cc] * r2;
            }
        }
        eb[c] = acc;
    }
}

// shapes of the start and end points on the 5-node window that starts two
// nodes left of the start point's nearest node; returns false when the
// nearest node moved by more than one (Courant condition violated)
template <typename R>
__device__ __forceinline__ bool window5(int ic0, const R *w0, int ic1, const R *w1, R *S0, R *dS)
{
    int sh = ic1 - ic0;
    R S1[5];
#pragma unroll
    for (int a = 0; a < 5; a++) { S0[a] = 0; S1[a] = 0; }
#pragma unroll
    for (int a = 0; a < 3; a++) S0[a + 1] = w0[a];
    if (sh < -1 || sh > 1) return false;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        int b = a + 1 + sh;
        S1[b] = w1[a];
    }
#pragma unroll
    for (int a = 0; a < 5; a++) dS[a] = S1[a] - S0[a];
    return true;
}

// Esirkepov deposit into the global current (red.global.add).  Along an
// active axis d: J_d(i+1/2) = J_d(i-1/2) - q w (dx_d/dt) W_d(i), summed
// from zero left of the window (the fifth partial sum is sum dS = 0).
// Along an inactive axis: q w v_d times the time average of the product of
// the node shapes, each linear in time between S0 and S1.
template <typename R, int DIM>
__device__ __forceinline__ void deposit_global(R *__restrict__ F, const Grid &g, const int *base,
                                               const R (*S0)[5], const R (*dS)[5], const R *cJ, R jvy, R jvz)
{
    R *Jx = F + JX * g.vol, *Jy = F + JY * g.vol, *Jz = F + JZ * g.vol;
    const R half = R(0.5), third = R(1.0 / 3.0);
    if (DIM == 1) {
        long long o = goff(g, base[0], 0, 0);
        R acc = 0;
#pragma unroll
        for (int a = 0; a < 4; a++) {
            acc += cJ[0] * dS[0][a];
            if (acc != R(0)) atomicAdd(Jx + o + a, acc);
        }
#pragma unroll
        for (int a = 0; a < 5; a++) {
            R f = S0[0][a] + half * dS[0][a];
            if (f != R(0)) {
                atomicAdd(Jy + o + a, jvy * f);
                atomicAdd(Jz + o + a, jvz * f);
            }
        }
    } else if (DIM == 2) {
#pragma unroll
        for (int b = 0; b < 5; b++) {
            long long o = goff(g, base[0], base[1] + b, 0);
            R ty = S0[1][b] + half * dS[1][b];
            R acc = 0;
#pragma unroll
            for (int a = 0; a < 4; a++) {
                acc += cJ[0] * (dS[0][a] * ty);
                if (acc != R(0)) atomicAdd(Jx + o + a, acc);
            }
        }
#pragma unroll
        for (int a = 0; a < 5; a++) {
            R tx = S0[0][a] + half * dS[0][a];
            R acc = 0;
#pragma unroll
            for (int b = 0; b < 4; b++) {
                acc += cJ[1] * (dS[1][b] * tx);
                if (acc != R(0)) atomicAdd(Jy + goff(g, base[0] + a, base[1] + b, 0), acc);
            }
        }
#pragma unroll
        for (int b = 0; b < 5; b++) {
            long long o = goff(g, base[0], base[1] + b, 0);
#pragma unroll
            for (int a = 0; a < 5; a++) {
                R wz = S0[0][a] * S0[1][b] + half * dS[0][a] * S0[1][b] + half * S0[0][a] * dS[1][b] +
                       third * dS[0][a] * dS[1][b];
                if (wz != R(0)) atomicAdd(Jz + o + a, jvz * wz);
            }
        }
    } else {
#pragma unroll
        for (int c = 0; c < 5; c++)
#pragma unroll
            for (int b = 0; b < 5; b++) {
                R t = S0[1][b] * S0[2][c] + half * dS[1][b] * S0[2][c] + half * S0[1][b] * dS[2][c] +
                      third * dS[1][b] * dS[2][c];
                long long o = goff(g, base[0], base[1] + b, base[2] + c);
                R acc = 0;
#pragma unroll
                for (int a = 0; a < 4; a++) {
                    acc += cJ[0] * (dS[0][a] * t);
                    if (acc != R(0)) atomicAdd(Jx + o + a, acc);
                }
            }
#pragma unroll
        for (int c = 0; c < 5; c++)
#pragma unroll
            for (int a = 0; a < 5; a++) {
                R t = S0[0][a] * S0[2][c] + half * dS[0][a] * S0[2][c] + half * S0[0][a] * dS[2][c] +
                      third * dS[0][a] * dS[2][c];
                R acc = 0;
#pragma unroll
                for (int b = 0; b < 4; b++) {
                    acc += cJ[1] * (dS[1][b] * t);
                    if (acc != R(0)) atomicAdd(Jy + goff(g, base[0] + a, base[1] + b, base[2] + c), acc);
                }
            }
#pragma unroll
        for (int b = 0; b < 5; b++)
#pragma unroll
            for (int a = 0; a < 5; a++) {
                R t = S0[0][a] * S0[1][b] + half * dS[0][a] * S0[1][b] + half * S0[0][a] * dS[1][b] +
                      third * dS[0][a] * dS[1][b];
                R acc = 0;
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    acc += cJ[2] * (dS[2][c] * t);
                    if (acc != R(0)) atomicAdd(Jz + goff(g, base[0] + a, base[1] + b, base[2] + c), acc);
                }
            }
    }
    (void)jvy;
}

// FP32 offset drift with face crossing
__device__ __forceinline__ void drift_f32(int &c, float &o, float d)
{
    float on = o + d;
    if (on >= 1.0f) {
        on -= 1.0f;
        c += 1;
    } else if (on < 0.0f) {
        on += 1.0f;
        c -= 1;
        if (on >= 1.0f) {  // a tiny negative offset rounded up to 1: the particle sits on the face
            on = 0.0f;
            c += 1;
        }
    }
    o = on;
}

// ---------------------------------------------------------------------
// FP32 cell+offset push
// ---------------------------------------------------------------------
template <int DIM>
__global__ void __launch_bounds__(256) k_push_f32(PartF32 P, float *__restrict__ F, Grid g, PushConst pc,
                                                  int *err, double *e_abs)
{
    long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= *P.dn) return;
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
    for (int d = 0; d < DIM; d++) drift_f32(c[d], o[d], (float)pc.hdx[d] * u[d] * ig);
    int ch[3] = {c[0], c[1], c[2]};
    float oh[3] = {o[0], o[1], o[2]};
    // gather
    int icn[3] = {0, 0, 0}, ich[3] = {0, 0, 0};
    float wn[3][3], wh[3][3];
#pragma unroll
    for (int d = 0; d < DIM; d++) axis_w_f32(c[d], o[d], icn[d], wn[d], ich[d], wh[d]);
    float eb[6];
    gather<float, DIM>(F, g, icn, wn, ich, wh, eb);
    // Boris
    const float k = (float)pc.qmdt2;
    boris<float>(ux, uy, uz, k * eb[0], k * eb[1], k * eb[2], k * eb[3], k * eb[4], k * eb[5]);
    float ig1 = inv_gamma(ux, uy, uz);
    u[0] = ux; u[1] = uy; u[2] = uz;
    // x^{n+1}, then x^{n+3/2}
#pragma unroll
    for (int d = 0; d < DIM; d++) drift_f32(c[d], o[d], (float)pc.hdx[d] * u[d] * ig1);
    int c1[3] = {c[0], c[1], c[2]};
    float o1[3] = {o[0], o[1], o[2]};
#pragma unroll
    for (int d = 0; d < DIM; d++) drift_f32(c[d], o[d], (float)pc.hdx[d] * u[d] * ig1);
    // Esirkepov on x^{n+1/2} -> x^{n+3/2}
    float S0[3][5], dS[3][5];
    int base[3] = {0, 0, 0};
    bool ok = true;
#pragma unroll
    for (int d = 0; d < DIM; d++) {
        int i0, i1;
        float w0[3], w1[3];
        axis_wn_f32(ch[d], oh[d], i0, w0);
        axis_wn_f32(c[d], o[d], i1, w1);
        ok &= window5<float>(i0, w0, i1, w1, S0[d], dS[d]);
        base[d] = i0 - 2;
    }
    if (!ok) {
        atomicOr(err, ERR_CFL);
        return;
    }
    float cJ[3] = {(float)pc.cJ[0], (float)pc.cJ[1], (float)pc.cJ[2]};
    float qw = (float)pc.qw;
    deposit_global<float, DIM>(F, g, base, S0, dS, cJ, qw * uy * ig1, qw * uz * ig1);
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
    if (!isfinite(ux + uy + uz)) atomicOr(err, ERR_NONFINITE);
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
template <int DIM>
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
    double wn[3][3], wh[3][3];
#pragma unroll
    for (int d = 0; d < DIM; d++) axis_w_f64(x[d] / g.dx[d], icn[d], wn[d], ich[d], wh[d]);
    double eb[6];
    gather<double, DIM>(F, g, icn, wn, ich, wh, eb);
    const double k = pc.qmdt2;
    boris<double>(ux, uy, uz, k * eb[0], k * eb[1], k * eb[2], k * eb[3], k * eb[4], k * eb[5]);
    double ig1 = inv_gamma(ux, uy, uz);
    u[0] = ux; u[1] = uy; u[2] = uz;
#pragma unroll
    for (int d = 0; d < DIM; d++) x[d] += pc.hdt * u[d] * ig1;
    double x1[3] = {x[0], x[1], x[2]};
#pragma unroll
    for (int d = 0; d < DIM; d++) x[d] += pc.hdt * u[d] * ig1;
    double S0[3][5], dS[3][5];
    int base[3] = {0, 0, 0};
    bool ok = true;
#pragma unroll
    for (int d = 0; d < DIM; d++) {
        int i0, i1;
        double w0[3], w1[3];
        axis_wn_f64(xh[d] / g.dx[d], i0, w0);
        axis_wn_f64(x[d] / g.dx[d], i1, w1);
        ok &= window5<double>(i0, w0, i1, w1, S0[d], dS[d]);
        base[d] = i0 - 2;
    }
    if (!ok) {
        atomicOr(err, ERR_CFL);
        return;
    }
    deposit_global<double, DIM>(F, g, base, S0, dS, pc.cJ, pc.qw * uy * ig1, pc.qw * uz * ig1);
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
    if (!isfinite(ux + uy + uz)) atomicOr(err, ERR_NONFINITE);
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
template <int DIM>
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
    float wn[3][3], wh[3][3];
#pragma unroll
    for (int d = 0; d < DIM; d++) axis_w_f32(c[d], P.off[d][p], icn[d], wn[d], ich[d], wh[d]);
    float eb[6];
    gather<float, DIM>(F, g, icn, wn, ich, wh, eb);
    for (int q = 0; q < 6; q++) out[6 * p + q] = eb[q];
}

template <int DIM>
__global__ void k_gather_f64(PartF64 P, const double *__restrict__ F, Grid g, double *out)
{
    long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= *P.dn) return;
    if (P.cell[p] == kDead) {
        for (int q = 0; q < 6; q++) out[6 * p + q] = 0.0;
        return;
    }
    int icn[3] = {0, 0, 0}, ich[3] = {0, 0, 0};
    double wn[3][3], wh[3][3];
#pragma unroll
    for (int d = 0; d < DIM; d++) axis_w_f64(P.x[d][p] / g.dx[d], icn[d], wn[d], ich[d], wh[d]);
    double eb[6];
    gather<double, DIM>(F, g, icn, wn, ich, wh, eb);
    for (int q = 0; q < 6; q++) out[6 * p + q] = eb[q];
}

// ---------------------------------------------------------------------
// load: FP64 absolute positions -> layout (positions already validated)
// ---------------------------------------------------------------------
__global__ void k_load_f32(PartF32 P, long long first, long long n, const double *x, const double *y,
                           const double *z, const double *ux, const double *uy, const double *uz, Grid g)
{
    long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    long long p = first + a;
    const double *xs[3] = {x, y, z};
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
                           const double *z, const double *ux, const double *uy, const double *uz, Grid g)
{
    long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    long long p = first + a;
    const double *xs[3] = {x, y, z};
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
    if (g.dim == 1) k_push_f32<1><<<nb, bs, 0, st>>>(P, F, g, pc, err, e_abs);
    else if (g.dim == 2) k_push_f32<2><<<nb, bs, 0, st>>>(P, F, g, pc, err, e_abs);
    else k_push_f32<3><<<nb, bs, 0, st>>>(P, F, g, pc, err, e_abs);
}

void launch_push_f64(const PartF64 &P, double *F, const Grid &g, const PushConst &pc, int *err, double *e_abs,
                     cudaStream_t st)
{
    if (P.n == 0) return;
    note_launch();
    int bs = 256, nb = div_up(P.n, bs);
    if (g.dim == 1) k_push_f64<1><<<nb, bs, 0, st>>>(P, F, g, pc, err, e_abs);
    else if (g.dim == 2) k_push_f64<2><<<nb, bs, 0, st>>>(P, F, g, pc, err, e_abs);
    else k_push_f64<3><<<nb, bs, 0, st>>>(P, F, g, pc, err, e_abs);
}

void launch_gather_f32(const PartF32 &P, const float *F, const Grid &g, double *out, cudaStream_t st)
{
    if (P.n == 0) return;
    note_launch();
    int bs = 256, nb = div_up(P.n, bs);
    if (g.dim == 1) k_gather_f32<1><<<nb, bs, 0, st>>>(P, F, g, out);
    else if (g.dim == 2) k_gather_f32<2><<<nb, bs, 0, st>>>(P, F, g, out);
    else k_gather_f32<3><<<nb, bs, 0, st>>>(P, F, g, out);
}

void launch_gather_f64(const PartF64 &P, const double *F, const Grid &g, double *out, cudaStream_t st)
{
    if (P.n == 0) return;
    note_launch();
    int bs = 256, nb = div_up(P.n, bs);
    if (g.dim == 1) k_gather_f64<1><<<nb, bs, 0, st>>>(P, F, g, out);
    else if (g.dim == 2) k_gather_f64<2><<<nb, bs, 0, st>>>(P, F, g, out);
    else k_gather_f64<3><<<nb, bs, 0, st>>>(P, F, g, out);
}

void launch_load_f32(const PartF32 &P, long long first, long long n, const double *const *xs,
                     const double *const *us, const Grid &g, cudaStream_t st)
{
    if (n == 0) return;
    note_launch();
    k_load_f32<<<div_up(n, 256), 256, 0, st>>>(P, first, n, xs[0], xs[1], xs[2], us[0], us[1], us[2], g);
}

void launch_load_f64(const PartF64 &P, long long first, long long n, const double *const *xs,
                     const double *const *us, const Grid &g, cudaStream_t st)
{
    if (n == 0) return;
    note_launch();
    k_load_f64<<<div_up(n, 256), 256, 0, st>>>(P, first, n, xs[0], xs[1], xs[2], us[0], us[1], us[2], g);
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
