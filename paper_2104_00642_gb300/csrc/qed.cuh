// qed.cuh -- device side of the QED Monte Carlo (Sec. IV): counter-based
// random numbers, quantum parameters, tabulated rates and inverse CDFs of
// nonlinear Compton emission (Eq. (23)) and Breit-Wheeler pair creation
// (Eq. (24)).
//
// Normalised forms (units of Eq. (8); E_s = m c^2 / (hbar omega_r)):
//   dW_rad/du  = alpha E_s / (sqrt3 pi gamma) Frad(u, chi),   u = eps_gamma / eps_e,
//   dW_pair/dv = alpha E_s / (sqrt3 pi k)     Fpair(v, chi),  v = eps_+ / eps_gamma,
// tabulated as G(chi) = Int_0^1 F and as the inverse of the normalised CDF.
#pragma once
#include <cstdint>

#include "mlp.cuh"
#include "pic_internal.cuh"

namespace pic {

enum QedProcess { QED_RAD = 0, QED_PAIR = 1 };

// tables: ln chi_i = lnchi0 + i dlnchi, i < nchi.  lnG[0][i] = ln G_rad(chi_i),
// lnG[1][i] = ln G_pair(chi_i) + 8/(3 chi_i); inv[p][i*nr + j] = s with
// CDF_p(s^3) = r_j, t_j = j/(nr-1): r_j = 1 - (1-t_j)^2 on [0,1] for emission,
// r_j = t_j^2/2 on [0,1/2] for pairs (the pair spectrum is symmetric).
struct QedTables {
    int nchi, nr;
    double lnchi0, dlnchi;
    float lnchi0_f, inv_dlnchi_f;  // the same in FP32 for the FP32 rate (FP64 is scarce on the device)
    const float *lnG_f[2], *inv_f[2];
    const double *lnG_d[2], *inv_d[2];
    // Bessel functions of Eqs. (23)/(24) for Method II's differential rates:
    // ln K_{2/3}(y) + y and ln Int_y^inf K_{1/3} + y on nbes nodes of ln y
    const double *bes_k23, *bes_ik13;
    int nbes;
    double bes_lny0, bes_dlny, bes_ymin, bes_ymax;
};

struct QedParams {
    int on;           // this species takes part in the Monte Carlo
    int method;       // 1: Method I (optical depth), 2: Method II (per-step acceptance)
    double pref;      // alpha E_s dt / (sqrt3 pi): W dt = pref G(chi) / (gamma or k)
    double inv_Es;    // 1 / E_s
    float pref_f, inv_Es_f;        // the same in FP32 (the FP32 form's rate and chi)
    float net_lo_f, net_hi_f;      // the network's trained ln chi range in FP32
    double emin;      // lightest photon kept as a macro-photon (m c^2)
    uint32_t key[2];  // Philox key
    uint32_t step;    // step index (counter word 2)
    QedTables T;
    double *tau;      // optical depth left, per particle
    uint64_t *id;     // identity, per particle
    uint32_t *ev;     // event flag per particle (1 = emitted / converted)
    float *evk;       // event data, 4 floats per particle: photon momentum (and v for pairs)
    double *e_lost;   // energy of photons below emin (tally)
    double wdV;       // weight * cell volume of this species (energy tallies)
    const MlpImage *net;  // surrogate network of this species' process (nullptr: tables only)
    MlpNorm nrm;          // its trained chi range and normalisation
    // photons with the network: the tiled push appends the thinned sampler's
    // candidates here (photon index, ln chi, W_env's G, chi) for
    // k_photon_resolve; one slot per photon, cq_n counts them
    float4 *cq;
    uint32_t *cq_n;
};

// ---------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64
// multiplications (0xD2511F53, 0xCD9E8D57), key bumped by the Weyl
// constants (0x9E3779B9, 0xBB67AE85)
// ---------------------------------------------------------------------
__host__ __device__ inline void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                              uint32_t k1, uint32_t *out)
{
#pragma unroll
    for (int r = 0; r < 10; r++) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

// uniform deviate in (0,1) from the top 24 bits, exact in FP32 and FP64
__host__ __device__ inline double uniform24(uint32_t x) { return ((double)(x >> 8) + 0.5) * (1.0 / 16777216.0); }

// counter words 2-3 of the draws: (step, purpose)
// (QP_TRAIN + process: training samples of the surrogate network, with the
// sample index as counter words 0-1 and the training iteration as word 2)
// (QP_THIN: the acceptance draw of a candidate conversion in the surrogate
// form's thinned pair sampler, purpose 5: 3 and 4 are the two processes'
// training draws)
enum QedPurpose : uint32_t { QP_EMIT = 0, QP_PAIR = 1, QP_INIT = 2, QP_TRAIN = 3, QP_THIN = 5 };
constexpr uint32_t kInitStep = 0xFFFFFFFFu;

// initial optical depth of a particle with identity id
__host__ __device__ inline double initial_tau(uint64_t id, const uint32_t *key)
{
    uint32_t w[4];
    philox4x32_10((uint32_t)id, (uint32_t)(id >> 32), kInitStep, QP_INIT, key[0], key[1], w);
    return -log(uniform24(w[0]));
}

// quantum parameter chi = sqrt((g E + u x B)^2 - (u.E)^2) / E_s for a
// particle of momentum u (or a photon of momentum k, g = |k|)
template <typename R>
__device__ __forceinline__ double chi_of(R g, R ux, R uy, R uz, R ex, R ey, R ez, R bx, R by, R bz, double inv_Es)
{
    const double fx = (double)g * ex + ((double)uy * bz - (double)uz * by);
    const double fy = (double)g * ey + ((double)uz * bx - (double)ux * bz);
    const double fz = (double)g * ez + ((double)ux * by - (double)uy * bx);
    const double ue = (double)ux * ex + (double)uy * ey + (double)uz * ez;
    const double s = fx * fx + fy * fy + fz * fz - ue * ue;
    return s > 0.0 ? sqrt(s) * inv_Es : 0.0;
}

template <typename R>
__host__ __device__ __forceinline__ const R *qed_lnG_nodes(const QedTables &T, int p)
{
    return p == 0 ? (const R *)(sizeof(R) == 4 ? (const void *)T.lnG_f[0] : (const void *)T.lnG_d[0])
                  : (const R *)(sizeof(R) == 4 ? (const void *)T.lnG_f[1] : (const void *)T.lnG_d[1]);
}

// The tabulated ln G (pairs: ln G + 8/(3 chi)) at table coordinate
// x = (ln chi - lnchi0) / dlnchi > 0: Catmull-Rom inside the table, linear
// continuation above it
template <typename R>
__host__ __device__ __forceinline__ double qed_lnG_table(const QedTables &T, int p, double x)
{
    const R *L = qed_lnG_nodes<R>(T, p);
    if (x >= T.nchi - 1) {
        const int n = T.nchi;
        return (double)L[n - 1] + (x - (n - 1)) * ((double)L[n - 1] - (double)L[n - 2]);
    }
    int i = (int)x;
    const double t = x - i;
    const int i0 = max(i - 1, 0), i3 = min(i + 2, T.nchi - 1);
    const double p0 = L[i0], p1 = L[i], p2 = L[i + 1], p3 = L[i3];
    const double a = -0.5 * p0 + 1.5 * p1 - 1.5 * p2 + 0.5 * p3;
    const double b = p0 - 2.5 * p1 + 2.0 * p2 - 0.5 * p3;
    const double c = -0.5 * p0 + 0.5 * p2;
    return ((a * t + b) * t + c) * t + p1;
}

// G_p(chi): Catmull-Rom in ln chi on ln G (pairs: on ln G + 8/(3 chi), the
// exponential small-chi factor removed); below the table the emission rate
// follows its classical limit (ln G linear in ln chi) and the pair rate is
// zero; above it both continue linearly in ln chi
template <typename R>
__host__ __device__ __forceinline__ double qed_rate(const QedTables &T, int p, double chi)
{
    if (!(chi > 0.0)) return 0.0;
    const double x = (log(chi) - T.lnchi0) / T.dlnchi;
    const double sub = p == QED_PAIR ? 8.0 / (3.0 * chi) : 0.0;
    if (x <= 0.0) {
        if (p == QED_PAIR) return 0.0;
        const R *L = qed_lnG_nodes<R>(T, p);
        return exp((double)L[0] + x * ((double)L[1] - (double)L[0]));
    }
    return exp(qed_lnG_table<R>(T, p, x) - sub);
}

// fraction (u for emission, v for pairs) with CDF = r: bilinear in
// (ln chi, r) on s = fraction^(1/3), chi clamped to the table
template <typename R>
__host__ __device__ __forceinline__ double qed_sample(const QedTables &T, int p, double chi, double r)
{
    const R *I = (const R *)(sizeof(R) == 4 ? (const void *)T.inv_f[p] : (const void *)T.inv_d[p]);
    double x = (log(fmax(chi, 1e-300)) - T.lnchi0) / T.dlnchi;
    x = fmin(fmax(x, 0.0), (double)(T.nchi - 1) - 1e-9);
    const int i = (int)x;
    const double tx = x - i;
    bool flip = false;
    double rr = r;
    if (p == QED_PAIR && rr > 0.5) {
        rr = 1.0 - rr;
        flip = true;
    }
    // r grids: emission r_j = 1 - (1 - t_j)^2, pairs r_j = t_j^2 / 2, t_j uniform
    const double tj = p == QED_PAIR ? sqrt(2.0 * rr) : 1.0 - sqrt(fmax(1.0 - rr, 0.0));
    double y = tj * (T.nr - 1);
    y = fmin(fmax(y, 0.0), (double)(T.nr - 1) - 1e-9);
    const int j = (int)y;
    double ty = y - j;
    if (p == QED_RAD && rr < 0.5) {
        // below the median the inverse is close to linear in r itself (the
        // u^(-2/3) spectrum makes s = u^(1/3) proportional to r at small r),
        // so the in-cell weight is taken in r: linear in t would be off by
        // up to t_1/2 ~ 1e-3 in s near r = 0
        const double t0 = (double)j / (T.nr - 1), t1 = (double)(j + 1) / (T.nr - 1);
        const double r0 = 1.0 - (1.0 - t0) * (1.0 - t0), r1 = 1.0 - (1.0 - t1) * (1.0 - t1);
        ty = fmin(fmax((rr - r0) / (r1 - r0), 0.0), 1.0);
    }
    const R *a = I + (long long)i * T.nr + j, *b = a + T.nr;
    const double s0 = (1.0 - ty) * (double)a[0] + ty * (double)a[1];
    const double s1 = (1.0 - ty) * (double)b[0] + ty * (double)b[1];
    const double s = (1.0 - tx) * s0 + tx * s1;
    const double f = s * s * s;
    return flip ? 1.0 - f : f;
}

// ---------------------------------------------------------------------
// Bessel functions and spectra (Eqs. (23), (24)) for Method II
// ---------------------------------------------------------------------
// Catmull-Rom through the nodes L[0..n) at table coordinate x (clamped to
// the table)
__host__ __device__ __forceinline__ double qed_cr(const double *L, int n, double x)
{
    int i = (int)x;
    if (i < 0) i = 0;
    if (i > n - 2) i = n - 2;
    const double t = x - i;
    const double p0 = L[i > 0 ? i - 1 : 0], p1 = L[i], p2 = L[i + 1], p3 = L[i + 2 < n ? i + 2 : n - 1];
    return (((-0.5 * p0 + 1.5 * p1 - 1.5 * p2 + 0.5 * p3) * t + (p0 - 2.5 * p1 + 2.0 * p2 - 0.5 * p3)) * t +
            (-0.5 * p0 + 0.5 * p2)) * t + p1;
}

// K_{2/3}(y) and Int_y^inf K_{1/3}: the tables (ln K + y, smooth in ln y)
// inside [ymin, ymax); zero above; below, the small-argument forms
// K_{2/3} ~ y^{-2/3} and Int = pi/sqrt3 - c y^{2/3} matched at ymin
__host__ __device__ __forceinline__ void qed_bessel(const QedTables &T, double y, double &k23, double &ik13)
{
    if (y >= T.bes_ymax) {
        k23 = ik13 = 0.0;
        return;
    }
    if (y < T.bes_ymin) {
        const double k0 = exp(T.bes_k23[0] - T.bes_ymin), i0 = exp(T.bes_ik13[0] - T.bes_ymin);
        const double full = 1.8137993642342178, r = cbrt(y / T.bes_ymin);  // pi / sqrt3
        k23 = k0 / (r * r);
        ik13 = full - (full - i0) * r * r;
        return;
    }
    const double x = (log(y) - T.bes_lny0) / T.bes_dlny;
    k23 = exp(qed_cr(T.bes_k23, T.nbes, x) - y);
    ik13 = exp(qed_cr(T.bes_ik13, T.nbes, x) - y);
}

// Eq. (23) without its prefactor: ((1-u) + 1/(1-u)) K_{2/3}(y) - Int_y K_{1/3},
// y = 2u / (3 chi (1-u))
__host__ __device__ __forceinline__ double qed_spec_rad(const QedTables &T, double u, double chi)
{
    if (!(u > 0.0) || !(u < 1.0) || !(chi > 0.0)) return 0.0;
    double k, ik;
    qed_bessel(T, 2.0 * u / (3.0 * chi * (1.0 - u)), k, ik);
    return ((1.0 - u) + 1.0 / (1.0 - u)) * k - ik;
}

// Eq. (24) without its prefactor: ((v^2 + (1-v)^2) / (v (1-v))) K_{2/3}(y)
// + Int_y K_{1/3}, y = 2 / (3 chi v (1-v))
__host__ __device__ __forceinline__ double qed_spec_pair(const QedTables &T, double v, double chi)
{
    if (!(v > 0.0) || !(v < 1.0) || !(chi > 0.0)) return 0.0;
    double k, ik;
    qed_bessel(T, 2.0 / (3.0 * chi * v * (1.0 - v)), k, ik);
    return ((v * v + (1.0 - v) * (1.0 - v)) / (v * (1.0 - v))) * k + ik;
}

// --- FP32 form: chi and the rate in single precision (the optical depth
// they decrement stays FP64) ---
__device__ __forceinline__ float chi_f32(float g, float ux, float uy, float uz, float ex, float ey, float ez, float bx,
                                         float by, float bz, float inv_Es)
{
    const float fx = fmaf(g, ex, uy * bz - uz * by);
    const float fy = fmaf(g, ey, uz * bx - ux * bz);
    const float fz = fmaf(g, ez, ux * by - uy * bx);
    const float ue = ux * ex + uy * ey + uz * ez;
    const float s = fx * fx + fy * fy + fz * fz - ue * ue;
    return s > 0.f ? sqrtf(s) * inv_Es : 0.f;
}

// G_p(chi) from the FP32 tables, as qed_rate in single precision
__device__ __forceinline__ float qed_rate_f32(const QedTables &T, int p, float chi)
{
    if (!(chi > 0.f)) return 0.f;
    const float *L = T.lnG_f[p];
    const float x = (logf(chi) - T.lnchi0_f) * T.inv_dlnchi_f;
    const float sub = p == QED_PAIR ? 8.0f / (3.0f * chi) : 0.f;
    if (x <= 0.f) return p == QED_PAIR ? 0.f : expf(fmaf(x, L[1] - L[0], L[0]));
    const int n = T.nchi;
    if (x >= n - 1) return expf(fmaf(x - (n - 1), L[n - 1] - L[n - 2], L[n - 1]) - sub);
    const int i = (int)x;
    const float t = x - i;
    const float p0 = L[max(i - 1, 0)], p1 = L[i], p2 = L[i + 1], p3 = L[min(i + 2, n - 1)];
    const float a = -0.5f * p0 + 1.5f * p1 - 1.5f * p2 + 0.5f * p3;
    const float b = p0 - 2.5f * p1 + 2.0f * p2 - 0.5f * p3;
    const float c = -0.5f * p0 + 0.5f * p2;
    return expf(fmaf(fmaf(fmaf(a, t, b), t, c), t, p1) - sub);
}

// The FP32 form's sampler: qed_sample in single precision on the FP32
// tables (a draw's fraction to ~1e-6, far inside the tables' own 1e-3)
__device__ __forceinline__ float qed_sample_f32(const QedTables &T, int p, float chi, float r)
{
    const float *I = T.inv_f[p];
    float x = (logf(fmaxf(chi, 1e-30f)) - T.lnchi0_f) * T.inv_dlnchi_f;
    x = fminf(fmaxf(x, 0.f), (float)(T.nchi - 1) * 0.99999994f);
    const int i = min((int)x, T.nchi - 2);
    const float tx = x - i;
    bool flip = false;
    float rr = r;
    if (p == QED_PAIR && rr > 0.5f) {
        rr = 1.0f - rr;
        flip = true;
    }
    const float tj = p == QED_PAIR ? sqrtf(2.0f * rr) : 1.0f - sqrtf(fmaxf(1.0f - rr, 0.f));
    float y = fminf(fmaxf(tj * (float)(T.nr - 1), 0.f), (float)(T.nr - 1) * 0.99999994f);
    const int j = min((int)y, T.nr - 2);
    float ty = y - j;
    if (p == QED_RAD && rr < 0.5f) {
        // the in-cell weight in r itself below the median (see qed_sample)
        const float t0 = (float)j / (T.nr - 1), t1 = (float)(j + 1) / (T.nr - 1);
        const float r0 = 1.0f - (1.0f - t0) * (1.0f - t0), r1 = 1.0f - (1.0f - t1) * (1.0f - t1);
        ty = fminf(fmaxf((rr - r0) / (r1 - r0), 0.f), 1.f);
    }
    const float *a = I + (long long)i * T.nr + j, *b = a + T.nr;
    const float s0 = fmaf(ty, a[1] - a[0], a[0]);
    const float s1 = fmaf(ty, b[1] - b[0], b[0]);
    const float sv = fmaf(tx, s1 - s0, s0);
    const float f = sv * sv * sv;
    return flip ? 1.0f - f : f;
}

// -ln r of the 24-bit uniform r = (k + 1/2) 2^-24, k = x >> 8, in FP32 to an
// ulp: through log1p of the complement above the median, where r itself
// would lose the low bits of k
__device__ __forceinline__ float neg_log_uniform24_f32(uint32_t x)
{
    const uint32_t k = x >> 8;
    if (k < (1u << 23)) return -logf(((float)k + 0.5f) * 5.9604644775390625e-08f);
    const float m = (float)((1u << 24) - 1u - k) + 0.5f;  // (1 - r) 2^24, exact
    return -log1pf(-m * 5.9604644775390625e-08f);
}

// An analytic upper envelope of the pair rate G_pair(chi) of Eq. (24) for
// chi in [0.1, 100]: 2.05 chi^(2/3) exp(-8/(3 chi)).  G exp(8/(3 chi)) /
// chi^(2/3) rises from 0.57 at chi = 0.1 to 1.94 at chi = 100, so the
// envelope lies 5.5 % above the rate at the top of the range (the network's
// rate is within 1.3 % of the tables') and 3.6x above it at the bottom,
// where the rate itself is ~1e-12.
constexpr float kPairEnvelope = 2.05f;
// x > 0 for an optical depth (never NaN) from its bit pattern: an integer
// compare instead of an FP64 one (FP64 runs at 1/73 of FP32 on this GPU)
__device__ __forceinline__ bool depth_positive(double x) { return __double_as_longlong(x) > 0; }

__device__ __forceinline__ float pair_envelope_f32(float chi)
{
    return kPairEnvelope * cbrtf(chi * chi) * expf(-8.0f / (3.0f * chi));
}

// the FP32 form's initial optical depth of a child: the draw of
// initial_tau, its -ln r in FP32 (as the form's other restarts; a warp spawns
// whenever one of its parents had an event, and FP64 costs it ~16 cycles per
// instruction)
__device__ __forceinline__ double initial_tau_f32(uint64_t id, const uint32_t *key)
{
    uint32_t w[4];
    philox4x32_10((uint32_t)id, (uint32_t)(id >> 32), kInitStep, QP_INIT, key[0], key[1], w);
    return (double)neg_log_uniform24_f32(w[0]);
}

// --- surrogate network in place of the tables (trained chi range) ---
__device__ __forceinline__ bool mlp_in_range(const MlpNorm &n, double chi, double &lnchi)
{
    lnchi = chi > 0.0 ? log(chi) : -1e300;
    return lnchi >= n.lnchi_lo && lnchi <= n.lnchi_hi;
}
// network inputs for (ln chi, r)
__device__ __forceinline__ void mlp_inputs(const MlpNorm &n, int p, double lnchi, double r, float &x0, float &x1)
{
    x0 = fmaf(n.x0a, (float)lnchi, n.x0b);
    x1 = (float)mlp_rcoord(p, r);
}
// the same in FP32 (the push: r is a 24-bit uniform, exact in FP32)
__device__ __forceinline__ void mlp_inputs_f32(const MlpNorm &n, int p, float lnchi, float r, float &x0, float &x1)
{
    x0 = fmaf(n.x0a, lnchi, n.x0b);
    const float t = p == 0 ? 1.0f - sqrtf(fmaxf(1.0f - r, 0.f)) : sqrtf(2.0f * fminf(r, 1.0f - r));
    x1 = 2.0f * t - 1.0f;
}
// G from the rate output y1
__device__ __forceinline__ double mlp_rate(const MlpNorm &n, int p, double chi, float y1)
{
    return exp((double)fmaf(n.sd, y1, n.mu) - (p == QED_PAIR ? 8.0 / (3.0 * chi) : 0.0));
}
__device__ __forceinline__ float mlp_rate_f32(const MlpNorm &n, int p, float chi, float y1)
{
    return expf(fmaf(n.sd, y1, n.mu) - (p == QED_PAIR ? 8.0f / (3.0f * chi) : 0.f));
}
__device__ __forceinline__ bool mlp_in_range_f32(float lo, float hi, float chi, float &lnchi)
{
    lnchi = chi > 0.f ? logf(chi) : -1e30f;
    return lnchi >= lo && lnchi <= hi;
}
// a 24-bit uniform draw as the network's FP32 input (within an ulp of
// (float) uniform24(x): the +1/2 offset needs a 25th bit)
__device__ __forceinline__ float uniform24_f32(uint32_t x)
{
    return fmaf((float)(x >> 8), 5.9604644775390625e-08f, 2.98023223876953125e-08f);
}
// energy fraction from the sample output y0 at CDF r (FP32: the push)
__device__ __forceinline__ float mlp_fraction_f32(int p, float y0, float r)
{
    const float s = fminf(fmaxf(y0, 0.f), p == QED_PAIR ? 0.79370052598f : 1.0f), f = s * s * s;
    return p == QED_PAIR && r > 0.5f ? 1.0f - f : f;
}
// energy fraction from the sample output y0 at CDF r
__device__ __forceinline__ double mlp_fraction(int p, float y0, double r)
{
    // pairs: the network's v is that of min(r, 1 - r), at most 1/2
    const double s = fmin(fmax((double)y0, 0.0), p == QED_PAIR ? 0.7937005259840998 : 1.0), f = s * s * s;
    return p == QED_PAIR && r > 0.5 ? 1.0 - f : f;
}

}  // namespace pic
