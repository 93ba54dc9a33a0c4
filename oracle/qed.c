/*
 * qed.c -- FP64 oracle of the QED module (Sec. IV): nonlinear Compton
 * photon emission (Eq. (23)) and nonlinear Breit-Wheeler pair production
 * (Eq. (24)), with the optical-depth Monte Carlo (Method I) and the
 * rejection sampler (Method II).
 *
 * TEST INFRASTRUCTURE; shares no code or table with the CUDA path.
 *
 * Normalised forms (units of Eq. (8), E_s = m c^2 / (hbar omega_r)):
 *   dW_rad/du  = alpha E_s / (sqrt(3) pi gamma) * Frad(u, chi),
 *     Frad = ((1-u) + 1/(1-u)) K_{2/3}(y) - Int_y^inf K_{1/3},  y = 2u / (3 chi (1-u)),
 *     u = eps_gamma / eps_e  (Eq. (23): (u^2-2u+2)/(1-u) = (1-u) + 1/(1-u));
 *   dW_pair/dv = alpha E_s / (sqrt(3) pi k) * Fpair(v, chi),
 *     Fpair = ((v^2 + (1-v)^2) / (v (1-v))) K_{2/3}(y) + Int_y^inf K_{1/3},  y = 2 / (3 chi v (1-v)),
 *     v = eps_+ / eps_gamma  (Eq. (24) with eps_- = eps_gamma - eps_+).
 * Bessel functions from their integral representations
 *   K_nu(x) = Int_0^inf exp(-x cosh t) cosh(nu t) dt,
 *   Int_y^inf K_{1/3}(x) dx = Int_0^inf exp(-y cosh t) cosh(t/3) / cosh t dt,
 * by the trapezoid rule (exponentially convergent for these integrands).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#include "pic_oracle.h"

/* trapezoid rule on [0, T] with T where the exponent reaches -745 */
static double trap_k(double nu, double x, int kind)
{
    if (x <= 0.0) return INFINITY;
    /* the integrand is analytic in the strip |Im t| < pi/2, so the
     * trapezoid error falls like exp(-pi^2 / h): h = 0.05 is far below
     * round-off */
    double T = acosh(745.0 / x > 1.0 ? 745.0 / x : 1.0) + 1.0;
    double h = 0.05;
    int n = (int)ceil(T / h);
    h = T / n;
    double s = 0.0;
    for (int i = 0; i <= n; i++) {
        double t = i * h;
        double f = exp(-x * cosh(t)) * cosh(nu * t);
        if (kind == 1) f /= cosh(t);
        s += (i == 0 || i == n) ? 0.5 * f : f;
    }
    return s * h;
}

double or_bessel_k(double nu, double x) { return trap_k(nu, x, 0); }
double or_int_k13(double y) { return trap_k(1.0 / 3.0, y, 1); }

double or_qed_Frad(double u, double chi)
{
    if (u <= 0.0 || u >= 1.0 || chi <= 0.0) return 0.0;
    double y = 2.0 * u / (3.0 * chi * (1.0 - u));
    if (y > 700.0) return 0.0;
    return ((1.0 - u) + 1.0 / (1.0 - u)) * or_bessel_k(2.0 / 3.0, y) - or_int_k13(y);
}

double or_qed_Fpair(double v, double chi)
{
    if (v <= 0.0 || v >= 1.0 || chi <= 0.0) return 0.0;
    double y = 2.0 / (3.0 * chi * v * (1.0 - v));
    if (y > 700.0) return 0.0;
    return ((v * v + (1.0 - v) * (1.0 - v)) / (v * (1.0 - v))) * or_bessel_k(2.0 / 3.0, y) + or_int_k13(y);
}

/* 8-point Gauss-Legendre nodes/weights on [-1, 1] */
static const double GLX[8] = {-0.9602898564975363, -0.7966664774136267, -0.5255324099163290, -0.1834346424956498,
                              0.1834346424956498,  0.5255324099163290,  0.7966664774136267,  0.9602898564975363};
static const double GLW[8] = {0.1012285362903763, 0.2223810344533745, 0.3137066458778873, 0.3626837833783620,
                              0.3626837833783620, 0.3137066458778873, 0.2223810344533745, 0.1012285362903763};

/* Int_0^umax Frad(u) du for umax <= 1/2 with u = s^3 (removes the
 * u^{-2/3} end point), composite Gauss-Legendre over s in [0, umax^{1/3}] */
static double int_rad_lo(double umax, double chi, int npan)
{
    double smax = cbrt(umax), acc = 0.0, hp = smax / npan;
    for (int p = 0; p < npan; p++) {
        double a = p * hp;
        for (int q = 0; q < 8; q++) {
            double s = a + 0.5 * hp * (GLX[q] + 1.0);
            acc += 0.5 * hp * GLW[q] * 3.0 * s * s * or_qed_Frad(s * s * s, chi);
        }
    }
    return acc;
}

/* Int_{1-t1^3}^{1-t0^3} Frad(u) du with 1 - u = t^3, t in [t0, t1]: at large
 * chi the spectrum peaks like (1-u)^{-1/3} within ~1/(3 chi) of u = 1 */
static double int_rad_hi(double t0, double t1, double chi, int npan)
{
    double acc = 0.0, hp = (t1 - t0) / npan;
    for (int p = 0; p < npan; p++) {
        double a = t0 + p * hp;
        for (int q = 0; q < 8; q++) {
            double t = a + 0.5 * hp * (GLX[q] + 1.0);
            acc += 0.5 * hp * GLW[q] * 3.0 * t * t * or_qed_Frad(1.0 - t * t * t, chi);
        }
    }
    return acc;
}

/* Int_0^umax Frad(u) du */
static double int_rad(double umax, double chi, int npan)
{
    if (umax <= 0.5) return int_rad_lo(umax, chi, npan);
    return int_rad_lo(0.5, chi, npan) + int_rad_hi(cbrt(1.0 - umax), cbrt(0.5), chi, npan);
}

/* Int_0^vmax Fpair(v) dv for vmax <= 1/2 with v = s^3 (the spectrum
 * behaves like v^{-1/3} above its exponential cut-off at large chi),
 * composite Gauss-Legendre */
static double int_pair_half(double vmax, double chi, int npan)
{
    double smax = cbrt(vmax), acc = 0.0, hp = smax / npan;
    for (int p = 0; p < npan; p++) {
        double a = p * hp;
        for (int q = 0; q < 8; q++) {
            double s = a + 0.5 * hp * (GLX[q] + 1.0);
            acc += 0.5 * hp * GLW[q] * 3.0 * s * s * or_qed_Fpair(s * s * s, chi);
        }
    }
    return acc;
}

/* Int_0^vmax Fpair(v) dv using the symmetry Fpair(v) = Fpair(1 - v) */
static double int_pair(double vmax, double chi, int npan)
{
    if (vmax <= 0.5) return int_pair_half(vmax, chi, npan);
    double half = int_pair_half(0.5, chi, npan);
    return 2.0 * half - int_pair_half(1.0 - vmax, chi, npan);
}

double or_qed_Grad(double chi) { return int_rad(1.0, chi, 64); }
double or_qed_Gpair(double chi) { return int_pair(1.0, chi, 64); }
double or_qed_cdf_rad(double u, double chi) { return int_rad(u, chi, 64) / int_rad(1.0, chi, 64); }
double or_qed_cdf_pair(double v, double chi) { return int_pair(v, chi, 64) / int_pair(1.0, chi, 64); }

/* radiated power integral Int_0^1 u Frad du (classical limit 2 pi chi^2 / sqrt(3)) */
double or_qed_Prad(double chi)
{
    double acc = 0.0, smax = cbrt(0.5), hp = smax / 64;
    for (int p = 0; p < 64; p++) {
        double a = p * hp;
        for (int q = 0; q < 8; q++) {
            double s = a + 0.5 * hp * (GLX[q] + 1.0);
            double u = s * s * s, t = s, v = 1.0 - t * t * t;
            acc += 0.5 * hp * GLW[q] * 3.0 * s * s * u * or_qed_Frad(u, chi); /* u <= 1/2 */
            acc += 0.5 * hp * GLW[q] * 3.0 * t * t * v * or_qed_Frad(v, chi); /* u >= 1/2, 1 - u = t^3 */
        }
    }
    return acc;
}

/* one Gauss-Legendre cell of Int 3 w^2 F(g(w)) dw over [a, b], with
 * g(w) = w^3 (kind 0: emission below 1/2, kind 1: pairs) or 1 - w^3
 * (kind 2: emission above 1/2) */
static double cell_int(int kind, double a, double b, double chi)
{
    double acc = 0.0;
    for (int q = 0; q < 8; q++) {
        double w = a + 0.5 * (b - a) * (GLX[q] + 1.0), w3 = w * w * w;
        double F = kind == 1 ? or_qed_Fpair(w3, chi) : or_qed_Frad(kind == 2 ? 1.0 - w3 : w3, chi);
        acc += 0.5 * (b - a) * GLW[q] * 3.0 * w * w * F;
    }
    return acc;
}

/* the variable w in [0, wmax] with Int_0^w 3 w'^2 F(g(w')) dw' = target:
 * cumulative sums over 64 cells locate the cell, bisection inside it (the
 * cell integral is re-evaluated exactly at every step) */
static double invert_w(int kind, double chi, double wmax, double target)
{
    const int NC = 64;
    double h = wmax / NC, acc = 0.0;
    int c = 0;
    for (c = 0; c < NC; c++) {
        double part = cell_int(kind, c * h, (c + 1) * h, chi);
        if (acc + part >= target) break;
        acc += part;
    }
    if (c == NC) return wmax;
    double lo = c * h, hi = (c + 1) * h;
    for (int it = 0; it < 50; it++) {
        double mid = 0.5 * (lo + hi);
        if (acc + cell_int(kind, c * h, mid, chi) < target) lo = mid;
        else hi = mid;
    }
    return 0.5 * (lo + hi);
}

static double invert(int pair, double chi, double fmax, double target)
{
    double w = invert_w(pair ? 1 : 0, chi, cbrt(fmax), target);
    return w * w * w;
}

/* Method I: the energy fraction u with CDF(u) = r; below u = 1/2 in
 * s = u^(1/3), above it in t = (1-u)^(1/3) counted down from u = 1 */
double or_qed_sample_rad(double chi, double r)
{
    double lo = int_rad_lo(0.5, chi, 64), hi = int_rad_hi(0.0, cbrt(0.5), chi, 64);
    double target = r * (lo + hi);
    if (target <= lo) return invert(0, chi, 0.5, target);
    double t = invert_w(2, chi, cbrt(0.5), lo + hi - target); /* Int_{1-t^3}^1 F = (1 - r) G */
    return 1.0 - t * t * t;
}

/* pair fraction v with CDF(v) = r, using the symmetry CDF(1-v) = 1 - CDF(v) */
double or_qed_sample_pair(double chi, double r)
{
    double half = int_pair_half(0.5, chi, 64);
    if (r <= 0.5) return invert(1, chi, 0.5, 2.0 * r * half);
    return 1.0 - invert(1, chi, 0.5, 2.0 * (1.0 - r) * half);
}

/* Method II (Sec. IV): with r1, r2 uniform, u0 = r1^3 is accepted when
 * r2 < 3 r1^2 dW/du(u0) dt; dwdt = alpha E_s dt / (sqrt(3) pi gamma) is the
 * prefactor times dt.  Returns u0, -1 (no emission this step), or -2 when
 * the acceptance probability exceeds one (dt too large for the method). */
double or_qed_method2_rad(double chi, double dwdt, double r1, double r2)
{
    double u0 = r1 * r1 * r1;
    double p = 3.0 * r1 * r1 * dwdt * or_qed_Frad(u0, chi);
    if (p > 1.0) return -2.0;
    return r2 < p ? u0 : -1.0;
}
