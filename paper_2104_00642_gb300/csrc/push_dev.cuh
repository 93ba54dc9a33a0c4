// push_dev.cuh -- device helpers of the particle kernels: per-axis nearest
// node and W_2 weights (Sec. II.D), the gather of Eq. (19), Esirkepov's
// window and deposit (Eqs. (20)-(22)), and the FP32 offset drift.
#pragma once
#include "push.cuh"

namespace pic {

// ---------------------------------------------------------------------
// per-axis nearest node and W_2 weights
// ---------------------------------------------------------------------

// W_4 (the cell integral of the order-4 shape S_4 of Eq. (18), the quartic
// B-spline): nodes ic-2 .. ic+2 for a particle at delta in [-1/2, 1/2)
template <typename R>
__device__ __forceinline__ void w4(R delta, R *w)
{
    const R d2 = delta * delta, d4 = d2 * d2;
    const R a = R(1) - R(2) * delta, b = R(1) + R(2) * delta;
    w[0] = (a * a) * (a * a) * R(1.0 / 384.0);
    w[1] = (R(19) - R(44) * delta + R(24) * d2 + R(16) * d2 * delta - R(16) * d4) * R(1.0 / 96.0);
    w[2] = R(115.0 / 192.0) - R(0.625) * d2 + R(0.25) * d4;
    w[3] = (R(19) + R(44) * delta + R(24) * d2 - R(16) * d2 * delta - R(16) * d4) * R(1.0 / 96.0);
    w[4] = (b * b) * (b * b) * R(1.0 / 384.0);
}

// the weights of shape order ORDER (2: W_2 on 3 nodes, 4: W_4 on 5 nodes)
template <typename R, int ORDER>
__device__ __forceinline__ void shape_w(R delta, R *w)
{
    if constexpr (ORDER == 4) w4<R>(delta, w);
    else w2<R>(delta, w);
}

// FP32 form: X = c + o
template <int ORDER = 2>
__device__ __forceinline__ void axis_w_f32(int c, float o, int &icn, float *wn, int &ich, float *wh)
{
    bool up = o >= 0.5f;
    icn = c + (up ? 1 : 0);
    shape_w<float, ORDER>(up ? o - 1.0f : o, wn);
    ich = c;
    shape_w<float, ORDER>(o - 0.5f, wh);
}

template <int ORDER = 2>
__device__ __forceinline__ void axis_wn_f32(int c, float o, int &icn, float *wn)
{
    bool up = o >= 0.5f;
    icn = c + (up ? 1 : 0);
    shape_w<float, ORDER>(up ? o - 1.0f : o, wn);
}

// FP64 form: X = x / dx
template <int ORDER = 2>
__device__ __forceinline__ void axis_w_f64(double X, int &icn, double *wn, int &ich, double *wh)
{
    icn = (int)floor(X + 0.5);
    shape_w<double, ORDER>(X - (double)icn, wn);
    ich = (int)floor(X);
    shape_w<double, ORDER>(X - ((double)ich + 0.5), wh);
}

template <int ORDER = 2>
__device__ __forceinline__ void axis_wn_f64(double X, int &icn, double *wn)
{
    icn = (int)floor(X + 0.5);
    shape_w<double, ORDER>(X - (double)icn, wn);
}

// Eq. (19): each component with its own staggered nearest node per axis,
// ORDER + 1 nodes per axis from ic - ORDER/2
template <typename R, int DIM, int ORDER = 2>
__device__ __forceinline__ void gather(const R *__restrict__ F, const Grid &g, const int *icn,
                                       const R (*wn)[ORDER + 1], const int *ich, const R (*wh)[ORDER + 1], R *eb)
{
    constexpr int P = ORDER + 1, H = ORDER / 2;
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
            long long o = goff(g, ic[0] - H, 0, 0);
#pragma unroll
            for (int a = 0; a < P; a++) acc += w[0][a] * __ldg(Fc + o + a);
        } else if (DIM == 2) {
#pragma unroll
            for (int b = 0; b < P; b++) {
                long long o = goff(g, ic[0] - H, ic[1] - H + b, 0);
                R r = 0;
#pragma unroll
                for (int a = 0; a < P; a++) r += w[0][a] * __ldg(Fc + o + a);
                acc += w[1][b] * r;
            }
        } else {
#pragma unroll
            for (int cc = 0; cc < P; cc++) {
                R r2 = 0;
#pragma unroll
                for (int b = 0; b < P; b++) {
                    long long o = goff(g, ic[0] - H, ic[1] - H + b, ic[2] - H + cc);
                    R r = 0;
#pragma unroll
                    for (int a = 0; a < P; a++) r += w[0][a] * __ldg(Fc + o + a);
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

// shapes of the start and end points on the window of ORDER + 3 nodes that
// starts ORDER/2 + 1 nodes left of the start point's nearest node (ORDER 2:
// the 5-node window of window5, ORDER 4: 7 nodes); false when the nearest
// node moved by more than one
template <typename R, int ORDER>
__device__ __forceinline__ bool window_n(int ic0, const R *w0, int ic1, const R *w1, R *S0, R *dS)
{
    constexpr int P = ORDER + 1, WN = ORDER + 3;
    int sh = ic1 - ic0;
    R S1[WN];
#pragma unroll
    for (int a = 0; a < WN; a++) { S0[a] = 0; S1[a] = 0; }
#pragma unroll
    for (int a = 0; a < P; a++) S0[a + 1] = w0[a];
    if (sh < -1 || sh > 1) return false;
#pragma unroll
    for (int a = 0; a < P; a++) S1[a + 1 + sh] = w1[a];
#pragma unroll
    for (int a = 0; a < WN; a++) dS[a] = S1[a] - S0[a];
    return true;
}

// Esirkepov deposit into the global current (red.global.add).  Along an
// active axis d: J_d(i+1/2) = J_d(i-1/2) - q w (dx_d/dt) W_d(i), summed
// from zero left of the window (the fifth partial sum is sum dS = 0).
// Along an inactive axis: q w v_d times the time average of the product of
// the node shapes, each linear in time between S0 and S1.
template <typename R, int DIM, int ORDER = 2>
__device__ __forceinline__ void deposit_global(R *__restrict__ F, const Grid &g, const int *base,
                                               const R (*S0)[ORDER + 3], const R (*dS)[ORDER + 3], const R *cJ, R jvy,
                                               R jvz)
{
    constexpr int WN = ORDER + 3;
    R *Jx = F + JX * g.vol, *Jy = F + JY * g.vol, *Jz = F + JZ * g.vol;
    const R half = R(0.5), third = R(1.0 / 3.0);
    if (DIM == 1) {
        long long o = goff(g, base[0], 0, 0);
        R acc = 0;
#pragma unroll
        for (int a = 0; a < WN - 1; a++) {
            acc += cJ[0] * dS[0][a];
            if (acc != R(0)) atomicAdd(Jx + o + a, acc);
        }
#pragma unroll
        for (int a = 0; a < WN; a++) {
            R f = S0[0][a] + half * dS[0][a];
            if (f != R(0)) {
                atomicAdd(Jy + o + a, jvy * f);
                atomicAdd(Jz + o + a, jvz * f);
            }
        }
    } else if (DIM == 2) {
#pragma unroll
        for (int b = 0; b < WN; b++) {
            long long o = goff(g, base[0], base[1] + b, 0);
            R ty = S0[1][b] + half * dS[1][b];
            R acc = 0;
#pragma unroll
            for (int a = 0; a < WN - 1; a++) {
                acc += cJ[0] * (dS[0][a] * ty);
                if (acc != R(0)) atomicAdd(Jx + o + a, acc);
            }
        }
#pragma unroll
        for (int a = 0; a < WN; a++) {
            R tx = S0[0][a] + half * dS[0][a];
            R acc = 0;
#pragma unroll
            for (int b = 0; b < WN - 1; b++) {
                acc += cJ[1] * (dS[1][b] * tx);
                if (acc != R(0)) atomicAdd(Jy + goff(g, base[0] + a, base[1] + b, 0), acc);
            }
        }
#pragma unroll
        for (int b = 0; b < WN; b++) {
            long long o = goff(g, base[0], base[1] + b, 0);
#pragma unroll
            for (int a = 0; a < WN; a++) {
                R wz = S0[0][a] * S0[1][b] + half * dS[0][a] * S0[1][b] + half * S0[0][a] * dS[1][b] +
                       third * dS[0][a] * dS[1][b];
                if (wz != R(0)) atomicAdd(Jz + o + a, jvz * wz);
            }
        }
    } else {
#pragma unroll
        for (int c = 0; c < WN; c++)
#pragma unroll
            for (int b = 0; b < WN; b++) {
                R t = S0[1][b] * S0[2][c] + half * dS[1][b] * S0[2][c] + half * S0[1][b] * dS[2][c] +
                      third * dS[1][b] * dS[2][c];
                long long o = goff(g, base[0], base[1] + b, base[2] + c);
                R acc = 0;
#pragma unroll
                for (int a = 0; a < WN - 1; a++) {
                    acc += cJ[0] * (dS[0][a] * t);
                    if (acc != R(0)) atomicAdd(Jx + o + a, acc);
                }
            }
#pragma unroll
        for (int c = 0; c < WN; c++)
#pragma unroll
            for (int a = 0; a < WN; a++) {
                R t = S0[0][a] * S0[2][c] + half * dS[0][a] * S0[2][c] + half * S0[0][a] * dS[2][c] +
                      third * dS[0][a] * dS[2][c];
                R acc = 0;
#pragma unroll
                for (int b = 0; b < WN - 1; b++) {
                    acc += cJ[1] * (dS[1][b] * t);
                    if (acc != R(0)) atomicAdd(Jy + goff(g, base[0] + a, base[1] + b, base[2] + c), acc);
                }
            }
#pragma unroll
        for (int b = 0; b < WN; b++)
#pragma unroll
            for (int a = 0; a < WN; a++) {
                R t = S0[0][a] * S0[1][b] + half * dS[0][a] * S0[1][b] + half * S0[0][a] * dS[1][b] +
                      third * dS[0][a] * dS[1][b];
                R acc = 0;
#pragma unroll
                for (int c = 0; c < WN - 1; c++) {
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
}  // namespace pic
