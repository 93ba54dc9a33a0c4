// push_qed_dev.cuh -- the QED Monte Carlo of one lepton after its momentum
// update (Sec. IV), shared by the one-thread-per-particle push and the tiled
// push: chi from the gathered E, B and u^{n+1} (FP32; gamma in FP64 above
// u^2 = 1e8), the rate from the tables or, inside its chi range, the
// surrogate network; Method I in the optical-depth form (tau in FP64) or
// Method II (per-step acceptance).  On an event the photon momentum goes to
// evd (event = 1 when it is heavy enough to be kept, else its energy is
// tallied) and the lepton recoils to gamma (1 - u) along its direction.
#pragma once

#include "mlp_host.cuh"
#include "mlp_tc.cuh"
#include "push_dev.cuh"
#include "qed_host.cuh"

namespace pic {

// emission and recoil of the FP64 gamma island (gamma above 1e4, where
// 1 + u^2 loses the 1 in FP32): out of line, so that the lanes below the
// island never pay for its FP64 work
static __device__ __noinline__ void qed_recoil_f64(double frac, float &ux, float &uy, float &uz, float &eg, float &kx,
                                            float &ky, float &kz)
{
    const double uu = (double)ux * ux + (double)uy * uy + (double)uz * uz;
    const double gam = sqrt(1.0 + uu);
    const double e = frac * gam;
    const double umag = sqrt(uu);
    const double g1 = fmax(gam * (1.0 - frac), 1.0);
    const double s = umag > 0.0 ? sqrt(g1 * g1 - 1.0) / umag : 0.0;
    const double ek = umag > 0.0 ? e / umag : 0.0;
    kx = (float)(ek * ux);
    ky = (float)(ek * uy);
    kz = (float)(ek * uz);
    ux = (float)(ux * s);
    uy = (float)(uy * s);
    uz = (float)(uz * s);
    eg = (float)e;
}

// gamma of the island in FP64, out of line for the same reason
static __device__ __noinline__ float gamma_island_f32(float ux, float uy, float uz)
{
    return (float)sqrt(1.0 + (double)ux * ux + (double)uy * uy + (double)uz * uz);
}

// With SURR the call is warp-collective: every lane of the warp makes it
// (lanes with live false only take part in the network's evaluation);
// mlp_smem is the staged network image.  p indexes the QED arrays; a lane
// with live false touches nothing there.
template <bool SURR>
__device__ __forceinline__ void qed_lepton_f32(const QedParams &q, const unsigned char *mlp_smem, bool live,
                                               long long p, const float *eb, float &ux, float &uy, float &uz,
                                               int *err, uint32_t &event, float4 &evd)
{
    if (!q.on) return;
    // chi and the rate in FP32, gamma in FP64 above 1e4, tau in FP64.  FP64
    // runs at 1/73 of the FP32 rate on this GPU: the per-step path keeps to
    // the one FP64 add of the optical depth (and its compare); the event
    // kinematics, the FP64 gamma island and Method II take FP64 where needed
    const float uuf = ux * ux + uy * uy + uz * uz;
    const bool island = uuf > 1e8f;
    const float gamf = island ? gamma_island_f32(ux, uy, uz) : sqrtf(1.0f + uuf);
    const float chi = chi_f32(gamf, ux, uy, uz, eb[0], eb[1], eb[2], eb[3], eb[4], eb[5], q.inv_Es_f);
    uint32_t w[4];
    bool use_net = false;
    float y0 = 0.f, y1 = 0.f;
    if constexpr (SURR) {
        float lnchi;
        const bool inr = live && mlp_in_range_f32(q.net_lo_f, q.net_hi_f, chi, lnchi);
        if (__any_sync(0xffffffffu, inr)) {
            float x0 = 0.f, x1 = 0.f;
            if (inr) {
                const uint64_t id = q.id[p];
                philox4x32_10((uint32_t)id, (uint32_t)(id >> 32), q.step, QP_EMIT, q.key[0], q.key[1], w);
                mlp_inputs_f32(q.nrm, QED_RAD, lnchi, uniform24_f32(w[0]), x0, x1);
            }
            mlp_eval_warp_sparse(*reinterpret_cast<const MlpImage *>(mlp_smem), inr, x0, x1, y0, y1);
            use_net = inr;
        }
    }
    // a lane without a particle stops here, in every mode: p may index
    // another thread's particle (the tiled kernels' idle lanes), whose
    // optical depth it must not write
    if (!live) return;
    bool emit = false;
    double frac = 0.0, tau = 0.0;
    if (!SURR && q.method == 2) {
        // Method II: u0 = r1^3 emitted when r2 < 3 r1^2 dW/du(u0) dt
        const uint64_t id = q.id[p];
        philox4x32_10((uint32_t)id, (uint32_t)(id >> 32), q.step, QP_EMIT, q.key[0], q.key[1], w);
        const double r1 = uniform24(w[0]), r2 = uniform24(w[1]);
        const double u0 = r1 * r1 * r1;
        const double gam = island ? sqrt(1.0 + (double)ux * ux + (double)uy * uy + (double)uz * uz) : (double)gamf;
        const double pacc = 3.0 * r1 * r1 * q.pref * qed_spec_rad(q.T, u0, (double)chi) / gam;
        if (pacc > 1.0) atomicOr(err, ERR_QEDDT);
        emit = r2 < pacc;
        frac = u0;
    } else {
        const float G = use_net ? mlp_rate_f32(q.nrm, QED_RAD, chi, y1) : qed_rate_f32(q.T, QED_RAD, chi);
        tau = q.tau[p] - (double)(q.pref_f * G / gamf);
        if (tau <= 0.0) {
            // the event: fraction and new optical depth in FP32 (a warp takes
            // this branch whenever one of its lanes does, and each FP64
            // instruction there would cost the whole warp ~16 cycles)
            if (!use_net) {
                const uint64_t id = q.id[p];
                philox4x32_10((uint32_t)id, (uint32_t)(id >> 32), q.step, QP_EMIT, q.key[0], q.key[1], w);
            }
            frac = use_net ? mlp_fraction_f32(QED_RAD, y0, uniform24_f32(w[0]))
                           : qed_sample_f32(q.T, QED_RAD, chi, uniform24_f32(w[0]));
            tau = (double)neg_log_uniform24_f32(w[1]);
            emit = true;
        }
    }
    if (emit) {
        float kx, ky, kz, eg;
        if (!island) {
            // emission and recoil in FP32 (gamma below 1e4)
            const float umag = sqrtf(uuf), fr = (float)frac;
            eg = fr * gamf;
            const float g1 = fmaxf(gamf * (1.0f - fr), 1.0f);
            const float sc = umag > 0.f ? sqrtf(fmaf(g1, g1, -1.0f)) / umag : 0.f;
            const float ek = umag > 0.f ? eg / umag : 0.f;
            kx = ek * ux;
            ky = ek * uy;
            kz = ek * uz;
            ux *= sc;
            uy *= sc;
            uz *= sc;
        } else {
            qed_recoil_f64(frac, ux, uy, uz, eg, kx, ky, kz);
        }
        if ((double)eg >= q.emin) {
            event = 1;
            evd = make_float4(kx, ky, kz, 0.f);
        } else {
            atomicAdd(q.e_lost, (double)eg * q.wdV);
        }
    }
    if (SURR || q.method != 2) q.tau[p] = tau;
}

// The pair-creation Monte Carlo of one photon (Sec. IV): chi_gamma from k and
// the gathered E, B at x^{n+1/2}; W_pair from the tables or the surrogate
// network inside its chi range; Method I (optical depth, FP64) or Method II.
// On a conversion evd = (k, positron fraction v) and event = 1.  With SURR
// the call is warp-collective as qed_lepton_f32's.
template <bool SURR>
// tau_in: the photon's optical depth (q.tau[p], read by the caller: the
// tiled kernel stages it with the photon's state).
__device__ __forceinline__ void qed_photon_f32(const QedParams &q, const unsigned char *mlp_smem, bool live,
                                               long long p, float km, float kx, float ky, float kz, const float *eb,
                                               double tau_in, int *err, uint32_t &event, float4 &evd)
{
    const float chi = chi_f32(km, kx, ky, kz, eb[0], eb[1], eb[2], eb[3], eb[4], eb[5], q.inv_Es_f);
    uint32_t w[4];
    const bool use_net = false;  // (the network acts through the thinned sampler below)
    float y0 = 0.f, y1 = 0.f;
    if constexpr (SURR) {
        // Up to the top of the network's range the pair process is sampled
        // by thinning: the optical depth drains at the analytic envelope
        // W_env >= W (pair_envelope_f32); where it runs out (a candidate) the
        // candidate converts with probability W / W_env (a draw of its own)
        // and the depth restarts from -ln r after every candidate.  W and the
        // positron fraction come from the network inside its range, from the
        // tables below it.  The events are those of the rate W, and the
        // network -- 17 kflop per evaluation -- runs at candidates only, not
        // for every photon and step.
        float lnchi;
        const bool inr = live && km > 0.f && mlp_in_range_f32(q.net_lo_f, q.net_hi_f, chi, lnchi);
        const bool thin = live && km > 0.f && lnchi <= q.net_hi_f;
        double tau = tau_in;
        float genv = 0.f;
        bool cand = false, keep = false;
        if (thin) {
            genv = pair_envelope_f32(chi);
            const float dtau = q.pref_f * genv / km;
            // a decrement that is zero in FP32 (the envelope underflows below
            // chi ~ 0.03) leaves the depth as it is: nothing to update or store
            keep = dtau == 0.f && depth_positive(tau_in);
            if (!keep) {
                tau = tau_in - (double)dtau;
                cand = tau <= 0.0;
            }
        }
        if (cand) {
            const uint64_t id = q.id[p];
            philox4x32_10((uint32_t)id, (uint32_t)(id >> 32), q.step, QP_PAIR, q.key[0], q.key[1], w);
        }
        if (__any_sync(0xffffffffu, cand && inr)) {
            float x0 = 0.f, x1 = 0.f;
            if (cand && inr) mlp_inputs_f32(q.nrm, QED_PAIR, lnchi, uniform24_f32(w[0]), x0, x1);
            mlp_eval_warp_sparse(*reinterpret_cast<const MlpImage *>(mlp_smem), cand && inr, x0, x1, y0, y1);
        }
        if (!live) return;
        if (thin) {
            if (cand) {
                const float G = inr ? mlp_rate_f32(q.nrm, QED_PAIR, chi, y1) : qed_rate_f32(q.T, QED_PAIR, chi);
                const float pa = G / genv;
                if (pa > 1.0f) atomicOr(err, ERR_QEDDT);
                const uint64_t id = q.id[p];
                uint32_t v[4];
                philox4x32_10((uint32_t)id, (uint32_t)(id >> 32), q.step, QP_THIN, q.key[0], q.key[1], v);
                if (uniform24_f32(v[0]) < pa) {
                    const float r0 = uniform24_f32(w[0]);
                    event = 1;
                    evd = make_float4(kx, ky, kz,
                                      inr ? mlp_fraction_f32(QED_PAIR, y0, r0) : qed_sample_f32(q.T, QED_PAIR, chi, r0));
                }
                tau = (double)neg_log_uniform24_f32(w[1]);
            }
            if (!keep) q.tau[p] = tau;
            return;
        }
        // above the network's range: the tables, Method I, below
    }
    if (!live) return;  // as in qed_lepton_f32
    if (!SURR && q.method == 2) {
        // Method II for pairs: v0 = r1 accepted when r2 < dW_pair/dv(v0) dt
        if (km > 0.f) {
            const uint64_t id = q.id[p];
            philox4x32_10((uint32_t)id, (uint32_t)(id >> 32), q.step, QP_PAIR, q.key[0], q.key[1], w);
            const double r1 = uniform24(w[0]), r2 = uniform24(w[1]);
            const double pacc = q.pref * qed_spec_pair(q.T, r1, (double)chi) / (double)km;
            if (pacc > 1.0) atomicOr(err, ERR_QEDDT);
            if (r2 < pacc) {
                event = 1;
                evd = make_float4(kx, ky, kz, (float)r1);
            }
        }
    } else {
        const float G = use_net ? mlp_rate_f32(q.nrm, QED_PAIR, chi, y1) : qed_rate_f32(q.T, QED_PAIR, chi);
        const float dtau = km > 0.f ? q.pref_f * G / km : 0.f;
        if (dtau == 0.f && depth_positive(tau_in)) return;  // a zero rate in FP32 (chi below ~0.03): the depth stays, unstored
        double tau = tau_in - (double)dtau;
        if (tau <= 0.0) {
            if (!use_net) {
                const uint64_t id = q.id[p];
                philox4x32_10((uint32_t)id, (uint32_t)(id >> 32), q.step, QP_PAIR, q.key[0], q.key[1], w);
            }
            const float r0 = uniform24_f32(w[0]);
            const float vf = use_net ? mlp_fraction_f32(QED_PAIR, y0, r0) : qed_sample_f32(q.T, QED_PAIR, chi, r0);
            event = 1;
            evd = make_float4(kx, ky, kz, vf);
            tau = (double)neg_log_uniform24_f32(w[1]);
        }
        q.tau[p] = tau;
    }
}

}  // namespace pic
