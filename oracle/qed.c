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

/* Int_0^umax Frad(u) du with u = s^3 (removes the u^{-2/3} end point),
 * composite Gauss-Legendre, npan panels over s in [0, umax^{1/3}] */
static double int_rad(double umax, double chi, int npan)
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
    double acc = 0.0, hp = 1.0 / 64;
    for (int p = 0; p < 64; p++) {
        double a = p * hp;
        for (int q = 0; q < 8; q++) {
            double s = a + 0.5 * hp * (GLX[q] + 1.0);
            double u = s * s * s;
            acc += 0.5 * hp * GLW[q] * 3.0 * s * s * u * or_qed_Frad(u, chi);
        }
    }
    return acc;
}

/* Method I: the energy fraction u with CDF(u) = r (bisection on the exact CDF) */
double or_qed_sample_rad(double chi, double r)
{
    double tot = int_rad(1.0, chi, 64), lo = 0.0, hi = 1.0;
    for (int it = 0; it < 60; it++) {
        double mid = 0.5 * (lo + hi);
        if (int_rad(mid, chi, 64) / tot < r) lo = mid;
        else hi = mid;
    }
    return 0.5 * (lo + hi);
}

double or_qed_sample_pair(double chi, double r)
{
    double tot = int_pair(1.0, chi, 64), lo = 0.0, hi = 1.0;
    for (int it = 0; it < 60; it++) {
        double mid = 0.5 * (lo + hi);
        if (int_pair(mid, chi, 64) / tot < r) lo = mid;
        else hi = mid;
    }
    return 0.5 * (lo + hi);
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
