// push_qed.cu -- particle push with the QED Monte Carlo (Sec. IV) fused in,
// FP32 cell+offset form, one thread per particle.
//
// Leptons: half drift, gather, Boris (as in push.cu), then the optical-depth
// form of Method I: tau -= W_rad(chi, gamma) dt in FP64 with chi from the
// gathered E^{n+1/2}, B^{n+1/2} and u^{n+1}; when tau <= 0 a photon of
// energy u gamma is emitted along u (u from the inverse CDF of Eq. (23) with
// a Philox draw), the lepton recoils to gamma (1 - u) along its direction and
// tau restarts from -ln r.  The recoiled momentum then drives both drifts
// and the Esirkepov deposit.
// Photons: move at c along k, gather E, B at x^{n+1/2}, tau -= W_pair dt with
// chi_gamma from k; when tau <= 0 the photon converts (the pair fraction v
// from the inverse CDF of Eq. (24)); no current.
#include <algorithm>

#include "push_qed_dev.cuh"

namespace pic {

// With SURR the surrogate network replaces the tables inside its chi range.
// Its evaluation is warp-collective, so lanes without a live particle stay
// in step (on a safe dummy particle in cell 0, storing nothing) until the
// network has run; a live lane draws its emission numbers every step, so a
// single evaluation yields both the rate and, if the event happens, the
// energy fraction.
//
// first (optional, device): the particles below it are pushed by the tiled
// kernel (the ones sorted into its work items); this launch takes the rest
// (those appended since the sort) and owns their event flags.
// one particle of k_push_qed_f32 (p0: the first particle it owns)
template <int DIM, bool SURR>
__device__ __forceinline__ void k_push_qed_f32_one(PartF32 &P, float *__restrict__ F, const Grid &g, const PushConst &pc, const QedParams &q, int *err, double *e_abs, const unsigned char *smem, long long p, long long p0)
{
    const bool mine = p >= p0;
    const bool live = mine && p < *P.dn && P.cell[p] != kDead;
    if (!SURR || !__any_sync(0xffffffffu, live)) {
        if (!live) {
            if (mine && p <= P.n) q.ev[p] = 0;  // dead slots and slots past the live count (and the scan's end slot)
            return;
        }
    }
    int c[3] = {0, 0, 0};
    float o[3] = {0.f, 0.f, 0.f};
    float ux = 0.f, uy = 0.f, uz = 0.f;
    if (live) {
        unpack_cell(g, P.cell[p], c[0], c[1], c[2]);
        o[0] = P.off[0][p];
        if (DIM >= 2) o[1] = P.off[1][p];
        if (DIM >= 3) o[2] = P.off[2][p];
        ux = P.u[0][p];
        uy = P.u[1][p];
        uz = P.u[2][p];
    }
    float u[3] = {ux, uy, uz};
    float ig = inv_gamma(ux, uy, uz);
#pragma unroll
    for (int d = 0; d < DIM; d++) drift_f32(c[d], o[d], pc.hdx_f[d] * u[d] * ig);
    const int ch[3] = {c[0], c[1], c[2]};
    const float oh[3] = {o[0], o[1], o[2]};
    int icn[3] = {0, 0, 0}, ich[3] = {0, 0, 0};
    float wn[3][3], wh[3][3];
#pragma unroll
    for (int d = 0; d < DIM; d++) axis_w_f32(c[d], o[d], icn[d], wn[d], ich[d], wh[d]);
    float eb[6];
    gather<float, DIM>(F, g, icn, wn, ich, wh, eb);
    const float k = pc.qmdt2_f;
    lorentz<float>(pc.pusher, ux, uy, uz, k * eb[0], k * eb[1], k * eb[2], k * eb[3], k * eb[4], k * eb[5]);
    // --- QED: optical depth, emission, recoil ---
    uint32_t event = 0;
    float4 evd = make_float4(0.f, 0.f, 0.f, 0.f);
    qed_lepton_f32<SURR>(q, smem, live, p, eb, ux, uy, uz, err, event, evd);
    if (SURR && !live) {
        if (mine && p <= P.n) q.ev[p] = 0;
        return;
    }
    const float ig1 = inv_gamma(ux, uy, uz);
    u[0] = ux;
    u[1] = uy;
    u[2] = uz;
#pragma unroll
    for (int d = 0; d < DIM; d++) drift_f32(c[d], o[d], pc.hdx_f[d] * u[d] * ig1);
    int c1[3] = {c[0], c[1], c[2]};
    const float o1[3] = {o[0], o[1], o[2]};
#pragma unroll
    for (int d = 0; d < DIM; d++) drift_f32(c[d], o[d], pc.hdx_f[d] * u[d] * ig1);
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
    // a non-finite momentum (a NaN or infinite field) is reported and the particle
    // removed before anything uses its position: NaN positions would give no valid
    // cell or node index to the gather, the deposit or the diagnostics (and would
    // otherwise be reported as a Courant violation)
    if (!isfinite(ux + uy + uz)) {
        atomicOr(err, ERR_NONFINITE);
        P.cell[p] = kDead;
        q.ev[p] = 0;
        return;
    }
    if (!ok) {
        atomicOr(err, ERR_CFL);
        q.ev[p] = 0;
        return;
    }
    const float cJ[3] = {pc.cJ_f[0], pc.cJ_f[1], pc.cJ_f[2]};
    deposit_global<float, DIM>(F, g, base, S0, dS, cJ, pc.qw_f * uy * ig1, pc.qw_f * uz * ig1);
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
        const double uu = (double)ux * ux + (double)uy * uy + (double)uz * uz;
        atomicAdd(e_abs, pc.wmdV * uu / (sqrt(1.0 + uu) + 1.0));
        event = 0;  // an emitter absorbed in the same step records no photon
    } else {
        P.cell[p] = pack_cell(g, c1[0], DIM >= 2 ? c1[1] : 0, DIM >= 3 ? c1[2] : 0);
    }
#pragma unroll
    for (int d = 0; d < DIM; d++) P.off[d][p] = o1[d];
    P.u[0][p] = ux;
    P.u[1][p] = uy;
    P.u[2][p] = uz;
    q.ev[p] = event;
    if (event) reinterpret_cast<float4 *>(q.evk)[p] = evd;
}

template <int DIM, bool SURR>
__global__ void __launch_bounds__(256, SURR ? 2 : 1) k_push_qed_f32(PartF32 P, float *__restrict__ F, Grid g, PushConst pc,
                                                      QedParams q, int *err, double *e_abs,
                                                      const uint32_t *__restrict__ first)
{
    extern __shared__ __align__(16) unsigned char smem[];
    if constexpr (SURR) {
        mlp_stage(smem, q.net, kMlpStageBytes);
        __syncthreads();
    }
    if (!first) {
        k_push_qed_f32_one<DIM, SURR>(P, F, g, pc, q, err, e_abs, smem, (long long)blockIdx.x * blockDim.x + threadIdx.x, 0);
        return;
    }
    // the tail after the tiled kernel's particles: a block-uniform grid
    // stride over [first, P.n] (a grid over the whole range would launch a
    // block per 256 slots only to find most of them the tiled kernel's)
    const long long p0 = (long long)*first;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = (p0 / blockDim.x + blockIdx.x) * blockDim.x; base <= P.n; base += stride)
        k_push_qed_f32_one<DIM, SURR>(P, F, g, pc, q, err, e_abs, smem, base + threadIdx.x, p0);
}

// SURR: the pair network inside its chi range, as in k_push_qed_f32
// (first: as in k_push_qed_f32 -- the photons below it are the tiled kernel's)
// one particle of k_push_photon_f32 (p0: the first particle it owns)
template <int DIM, bool SURR>
__device__ __forceinline__ void k_push_photon_f32_one(PartF32 &P, const float *__restrict__ F, const Grid &g, const PushConst &pc, const QedParams &q, int *err, const unsigned char *smem, long long p, long long p0)
{
    const bool mine = p >= p0;
    const bool live = mine && p < *P.dn && P.cell[p] != kDead;
    if (!SURR || !__any_sync(0xffffffffu, live)) {
        if (!live) {
            if (mine && p <= P.n) q.ev[p] = 0;  // dead slots and slots past the live count (and the scan's end slot)
            return;
        }
    }
    int c[3] = {0, 0, 0};
    float o[3] = {0.f, 0.f, 0.f};
    float kx = 0.f, ky = 0.f, kz = 0.f;
    if (live) {
        unpack_cell(g, P.cell[p], c[0], c[1], c[2]);
        o[0] = P.off[0][p];
        if (DIM >= 2) o[1] = P.off[1][p];
        if (DIM >= 3) o[2] = P.off[2][p];
        kx = P.u[0][p];
        ky = P.u[1][p];
        kz = P.u[2][p];
    }
    const float km = sqrtf(kx * kx + ky * ky + kz * kz);
    const float ik = km > 0.f ? 1.0f / km : 0.f;
    const float v[3] = {kx * ik, ky * ik, kz * ik};
#pragma unroll
    for (int d = 0; d < DIM; d++) drift_f32(c[d], o[d], pc.hdx_f[d] * v[d]);
    uint32_t event = 0;
    float4 evd = make_float4(0.f, 0.f, 0.f, 0.f);
    if (q.on) {
        int icn[3] = {0, 0, 0}, ich[3] = {0, 0, 0};
        float wn[3][3], wh[3][3];
#pragma unroll
        for (int d = 0; d < DIM; d++) axis_w_f32(c[d], o[d], icn[d], wn[d], ich[d], wh[d]);
        float eb[6];
        gather<float, DIM>(F, g, icn, wn, ich, wh, eb);
        qed_photon_f32<SURR>(q, smem, live, p, km, kx, ky, kz, eb, live ? q.tau[p] : 0.0, err, event, evd);
        if (SURR && !live) {
            if (mine && p <= P.n) q.ev[p] = 0;
            return;
        }
    } else if (SURR && !live) {
        if (mine && p <= P.n) q.ev[p] = 0;
        return;
    }
#pragma unroll
    for (int d = 0; d < DIM; d++) drift_f32(c[d], o[d], pc.hdx_f[d] * v[d]);
    bool dead = false;
#pragma unroll
    for (int d = 0; d < DIM; d++) {
        if (g.bc[d] == PERIODIC) {
            if (c[d] < 0) c[d] += g.n[d];
            else if (c[d] >= g.n[d]) c[d] -= g.n[d];
        } else if (c[d] < 0 || c[d] >= g.n[d]) {
            dead = true;
        }
    }
    if (dead) {
        P.cell[p] = kDead;
        event = 0;  // a photon leaving through an absorbing face does not convert
    } else {
        P.cell[p] = pack_cell(g, c[0], DIM >= 2 ? c[1] : 0, DIM >= 3 ? c[2] : 0);
    }
#pragma unroll
    for (int d = 0; d < DIM; d++) P.off[d][p] = o[d];
    q.ev[p] = event;
    if (event) reinterpret_cast<float4 *>(q.evk)[p] = evd;
}

template <int DIM, bool SURR>
__global__ void __launch_bounds__(256, SURR ? 2 : 1) k_push_photon_f32(PartF32 P, const float *__restrict__ F, Grid g, PushConst pc,
                                                         QedParams q, int *err, const uint32_t *__restrict__ first)
{
    extern __shared__ __align__(16) unsigned char smem[];
    if constexpr (SURR) {
        mlp_stage(smem, q.net, kMlpStageBytes);
        __syncthreads();
    }
    if (!first) {
        k_push_photon_f32_one<DIM, SURR>(P, F, g, pc, q, err, smem, (long long)blockIdx.x * blockDim.x + threadIdx.x, 0);
        return;
    }
    // the tail after the tiled kernel's particles: a block-uniform grid
    // stride over [first, P.n] (a grid over the whole range would launch a
    // block per 256 slots only to find most of them the tiled kernel's)
    const long long p0 = (long long)*first;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = (p0 / blockDim.x + blockIdx.x) * blockDim.x; base <= P.n; base += stride)
        k_push_photon_f32_one<DIM, SURR>(P, F, g, pc, q, err, smem, base + threadIdx.x, p0);
}

// The photon push with the pair network on the tcgen05 tensor cores:
// persistent CTAs of 128 threads walk tiles of 128 photon slots (slots up
// to P.n, so that the scan's end slot and the dead slots get a zero flag);
// the network is evaluated by the whole CTA (mlp_eval_cta: one row per
// thread, accumulators in tensor memory) for every tile with a photon in
// its chi range.  Everything else is k_push_photon_f32<DIM, true>.  (On the
// QED collision it runs at the speed of the warp-level kernel, 2 % behind:
// the network's cost is its per-row SiLU and FP32 work, which both share;
// the push uses it when asked for, PIC_PUSH_MLP_TC.)
template <int DIM>
__global__ void __launch_bounds__(kMlpTcRows, 4) k_push_photon_tc(PartF32 P, const float *__restrict__ F, Grid g,
                                                                PushConst pc, QedParams q, int *err)
{
    extern __shared__ unsigned char smem_raw[];
    MlpTcSmem &S = *reinterpret_cast<MlpTcSmem *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    mlp_tc_setup(S, q.net);
    uint32_t phase = 0;
    const long long nlive = *P.dn;
    for (long long tile = blockIdx.x; tile * kMlpTcRows <= P.n; tile += gridDim.x) {
        const long long p = tile * kMlpTcRows + threadIdx.x;
        const bool live = p < nlive && P.cell[p] != kDead;
        int c[3] = {0, 0, 0};
        float o[3] = {0.f, 0.f, 0.f};
        float kx = 0.f, ky = 0.f, kz = 0.f;
        if (live) {
            unpack_cell(g, P.cell[p], c[0], c[1], c[2]);
            o[0] = P.off[0][p];
            if (DIM >= 2) o[1] = P.off[1][p];
            if (DIM >= 3) o[2] = P.off[2][p];
            kx = P.u[0][p];
            ky = P.u[1][p];
            kz = P.u[2][p];
        }
        const float km = sqrtf(kx * kx + ky * ky + kz * kz);
        const float ik = km > 0.f ? 1.0f / km : 0.f;
        const float v[3] = {kx * ik, ky * ik, kz * ik};
#pragma unroll
        for (int d = 0; d < DIM; d++) drift_f32(c[d], o[d], pc.hdx_f[d] * v[d]);
        float chi = 0.f, x0 = 0.f, x1 = 0.f, y0 = 0.f, y1 = 0.f;
        uint32_t w[4] = {0u, 0u, 0u, 0u};
        bool inr = false;
        if (q.on && live) {
            int icn[3] = {0, 0, 0}, ich[3] = {0, 0, 0};
            float wn[3][3], wh[3][3];
#pragma unroll
            for (int d = 0; d < DIM; d++) axis_w_f32(c[d], o[d], icn[d], wn[d], ich[d], wh[d]);
            float eb[6];
            gather<float, DIM>(F, g, icn, wn, ich, wh, eb);
            chi = chi_f32(km, kx, ky, kz, eb[0], eb[1], eb[2], eb[3], eb[4], eb[5], q.inv_Es_f);
            float lnchi;
            inr = km > 0.f && mlp_in_range_f32(q.net_lo_f, q.net_hi_f, chi, lnchi);
            if (inr) {
                const uint64_t id = q.id[p];
                philox4x32_10((uint32_t)id, (uint32_t)(id >> 32), q.step, QP_PAIR, q.key[0], q.key[1], w);
                mlp_inputs_f32(q.nrm, QED_PAIR, lnchi, uniform24_f32(w[0]), x0, x1);
            }
        }
        if (q.on && __syncthreads_or(inr)) {
            if (!mlp_eval_cta(S, phase, x0, x1, y0, y1)) {
                // the tensor cores did not answer: flag it, give the MMAs in
                // flight a last bounded wait, free the tensor memory, stop
                if (threadIdx.x == 0) atomicOr(err, ERR_TIMEOUT);
                mbar_wait(&S.bar, phase, 1 << 20);
                break;
            }
        }
        if (!live) {
            if (p <= P.n) q.ev[p] = 0;
            continue;
        }
        uint32_t event = 0;
        float4 evd = make_float4(0.f, 0.f, 0.f, 0.f);
        if (q.on) {
            const float G = inr ? mlp_rate_f32(q.nrm, QED_PAIR, chi, y1) : qed_rate_f32(q.T, QED_PAIR, chi);
            double tau = q.tau[p] - (km > 0.f ? (double)(q.pref_f * G / km) : 0.0);
            if (tau <= 0.0) {
                if (!inr) {
                    const uint64_t id = q.id[p];
                    philox4x32_10((uint32_t)id, (uint32_t)(id >> 32), q.step, QP_PAIR, q.key[0], q.key[1], w);
                }
                const double r0 = uniform24(w[0]);
                const double vf = inr ? mlp_fraction(QED_PAIR, y0, r0) : qed_sample<float>(q.T, QED_PAIR, chi, r0);
                event = 1;
                evd = make_float4(kx, ky, kz, (float)vf);
                tau = -log(uniform24(w[1]));
            }
            q.tau[p] = tau;
        }
#pragma unroll
        for (int d = 0; d < DIM; d++) drift_f32(c[d], o[d], pc.hdx_f[d] * v[d]);
        bool dead = false;
#pragma unroll
        for (int d = 0; d < DIM; d++) {
            if (g.bc[d] == PERIODIC) {
                if (c[d] < 0) c[d] += g.n[d];
                else if (c[d] >= g.n[d]) c[d] -= g.n[d];
            } else if (c[d] < 0 || c[d] >= g.n[d]) {
                dead = true;
            }
        }
        if (dead) {
            P.cell[p] = kDead;
            event = 0;  // a photon leaving through an absorbing face does not convert
        } else {
            P.cell[p] = pack_cell(g, c[0], DIM >= 2 ? c[1] : 0, DIM >= 3 ? c[2] : 0);
        }
#pragma unroll
        for (int d = 0; d < DIM; d++) P.off[d][p] = o[d];
        q.ev[p] = event;
        if (event) reinterpret_cast<float4 *>(q.evk)[p] = evd;
    }
    mlp_tc_teardown(S);
}

// ---------------------------------------------------------------------
// FP64 plain form: absolute positions, everything in double precision,
// the tables' FP64 copy (no surrogate).  Event data: 4 doubles per particle.
// ---------------------------------------------------------------------
template <int DIM>
__global__ void __launch_bounds__(256) k_push_qed_f64(PartF64 P, double *__restrict__ F, Grid g, PushConst pc,
                                                      QedParams q, int *err, double *e_abs)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= *P.dn || P.cell[p] == kDead) {
        if (p <= P.n) q.ev[p] = 0;
        return;
    }
    double x[3] = {P.x[0][p], DIM >= 2 ? P.x[1][p] : 0.0, DIM >= 3 ? P.x[2][p] : 0.0};
    double ux = P.u[0][p], uy = P.u[1][p], uz = P.u[2][p];
    const double ig = inv_gamma(ux, uy, uz);
    double u[3] = {ux, uy, uz};
#pragma unroll
    for (int d = 0; d < DIM; d++) x[d] += pc.hdt * u[d] * ig;
    const double xh[3] = {x[0], x[1], x[2]};
    int icn[3] = {0, 0, 0}, ich[3] = {0, 0, 0};
    double wn[3][3], wh[3][3];
#pragma unroll
    for (int d = 0; d < DIM; d++) axis_w_f64(x[d] / g.dx[d], icn[d], wn[d], ich[d], wh[d]);
    double eb[6];
    gather<double, DIM>(F, g, icn, wn, ich, wh, eb);
    const double k = pc.qmdt2;
    lorentz<double>(pc.pusher, ux, uy, uz, k * eb[0], k * eb[1], k * eb[2], k * eb[3], k * eb[4], k * eb[5]);
    uint32_t event = 0;
    double4 evd = make_double4(0.0, 0.0, 0.0, 0.0);
    if (q.on) {
        const double uu = ux * ux + uy * uy + uz * uz;
        const double gam = sqrt(1.0 + uu);
        const double chi = chi_of<double>(gam, ux, uy, uz, eb[0], eb[1], eb[2], eb[3], eb[4], eb[5], q.inv_Es);
        bool emit = false;
        double frac = 0.0, tau = 0.0;
        uint32_t w[4];
        const uint64_t id = q.id[p];
        if (q.method == 2) {
            // Method II: u0 = r1^3 emitted when r2 < 3 r1^2 dW/du(u0) dt
            philox4x32_10((uint32_t)id, (uint32_t)(id >> 32), q.step, QP_EMIT, q.key[0], q.key[1], w);
            const double r1 = uniform24(w[0]), r2 = uniform24(w[1]);
            const double u0 = r1 * r1 * r1;
            const double pacc = 3.0 * r1 * r1 * q.pref * qed_spec_rad(q.T, u0, chi) / gam;
            if (pacc > 1.0) atomicOr(err, ERR_QEDDT);
            emit = r2 < pacc;
            frac = u0;
        } else {
            tau = q.tau[p] - q.pref * qed_rate<double>(q.T, QED_RAD, chi) / gam;
            if (tau <= 0.0) {
                philox4x32_10((uint32_t)id, (uint32_t)(id >> 32), q.step, QP_EMIT, q.key[0], q.key[1], w);
                frac = qed_sample<double>(q.T, QED_RAD, chi, uniform24(w[0]));
                tau = -log(uniform24(w[1]));
                emit = true;
            }
        }
        if (emit) {
            const double eg = frac * gam, umag = sqrt(uu);
            const double g1 = fmax(gam * (1.0 - frac), 1.0);
            const double s = umag > 0.0 ? sqrt(g1 * g1 - 1.0) / umag : 0.0;
            const double e = umag > 0.0 ? eg / umag : 0.0;
            const double kx = e * ux, ky = e * uy, kz = e * uz;
            ux *= s;
            uy *= s;
            uz *= s;
            if (eg >= q.emin) {
                event = 1;
                evd = make_double4(kx, ky, kz, 0.0);
            } else {
                atomicAdd(q.e_lost, eg * q.wdV);
            }
        }
        if (q.method != 2) q.tau[p] = tau;
    }
    const double ig1 = inv_gamma(ux, uy, uz);
    u[0] = ux;
    u[1] = uy;
    u[2] = uz;
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
    // a non-finite momentum (a NaN or infinite field) is reported and the particle
    // removed before anything uses its position: NaN positions would give no valid
    // cell or node index to the gather, the deposit or the diagnostics (and would
    // otherwise be reported as a Courant violation)
    if (!isfinite(ux + uy + uz)) {
        atomicOr(err, ERR_NONFINITE);
        P.cell[p] = kDead;
        q.ev[p] = 0;
        return;
    }
    if (!ok) {
        atomicOr(err, ERR_CFL);
        q.ev[p] = 0;
        return;
    }
    deposit_global<double, DIM>(F, g, base, S0, dS, pc.cJ, pc.qw * uy * ig1, pc.qw * uz * ig1);
    bool dead = false;
    int cc[3] = {0, 0, 0};
#pragma unroll
    for (int d = 0; d < DIM; d++) {
        const double L = (double)g.n[d] * g.dx[d];
        if (g.bc[d] == PERIODIC) {
            if (x1[d] < 0.0) x1[d] += L;
            if (x1[d] >= L) x1[d] -= L;
        } else if (x1[d] < 0.0 || x1[d] >= L) {
            dead = true;
        }
        const int ci = (int)floor(x1[d] / g.dx[d]);
        cc[d] = ci < 0 ? 0 : (ci >= g.n[d] ? g.n[d] - 1 : ci);
    }
    if (dead) {
        P.cell[p] = kDead;
        const double uu = ux * ux + uy * uy + uz * uz;
        atomicAdd(e_abs, pc.wmdV * uu / (sqrt(1.0 + uu) + 1.0));
        event = 0;
    } else {
        P.cell[p] = pack_cell(g, cc[0], cc[1], cc[2]);
    }
#pragma unroll
    for (int d = 0; d < DIM; d++) P.x[d][p] = x1[d];
    P.u[0][p] = ux;
    P.u[1][p] = uy;
    P.u[2][p] = uz;
    q.ev[p] = event;
    if (event) reinterpret_cast<double4 *>(q.evk)[p] = evd;
}

template <int DIM>
__global__ void __launch_bounds__(256) k_push_photon_f64(PartF64 P, const double *__restrict__ F, Grid g,
                                                         PushConst pc, QedParams q, int *err)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= *P.dn || P.cell[p] == kDead) {
        if (p <= P.n) q.ev[p] = 0;
        return;
    }
    double x[3] = {P.x[0][p], DIM >= 2 ? P.x[1][p] : 0.0, DIM >= 3 ? P.x[2][p] : 0.0};
    const double kx = P.u[0][p], ky = P.u[1][p], kz = P.u[2][p];
    const double km = sqrt(kx * kx + ky * ky + kz * kz);
    const double ik = km > 0.0 ? 1.0 / km : 0.0;
    const double v[3] = {kx * ik, ky * ik, kz * ik};
#pragma unroll
    for (int d = 0; d < DIM; d++) x[d] += pc.hdt * v[d];
    uint32_t event = 0;
    double4 evd = make_double4(0.0, 0.0, 0.0, 0.0);
    if (q.on) {
        int icn[3] = {0, 0, 0}, ich[3] = {0, 0, 0};
        double wn[3][3], wh[3][3];
#pragma unroll
        for (int d = 0; d < DIM; d++) axis_w_f64(x[d] / g.dx[d], icn[d], wn[d], ich[d], wh[d]);
        double eb[6];
        gather<double, DIM>(F, g, icn, wn, ich, wh, eb);
        const double chi = chi_of<double>(km, kx, ky, kz, eb[0], eb[1], eb[2], eb[3], eb[4], eb[5], q.inv_Es);
        if (q.method == 2) {
            // Method II for pairs: v0 = r1 accepted when r2 < dW_pair/dv(v0) dt
            if (km > 0.0) {
                uint32_t w[4];
                const uint64_t id = q.id[p];
                philox4x32_10((uint32_t)id, (uint32_t)(id >> 32), q.step, QP_PAIR, q.key[0], q.key[1], w);
                const double r1 = uniform24(w[0]), r2 = uniform24(w[1]);
                const double pacc = q.pref * qed_spec_pair(q.T, r1, chi) / km;
                if (pacc > 1.0) atomicOr(err, ERR_QEDDT);
                if (r2 < pacc) {
                    event = 1;
                    evd = make_double4(kx, ky, kz, r1);
                }
            }
        } else {
            double tau = q.tau[p] - (km > 0.0 ? q.pref * qed_rate<double>(q.T, QED_PAIR, chi) / km : 0.0);
            if (tau <= 0.0) {
                uint32_t w[4];
                const uint64_t id = q.id[p];
                philox4x32_10((uint32_t)id, (uint32_t)(id >> 32), q.step, QP_PAIR, q.key[0], q.key[1], w);
                event = 1;
                evd = make_double4(kx, ky, kz, qed_sample<double>(q.T, QED_PAIR, chi, uniform24(w[0])));
                tau = -log(uniform24(w[1]));
            }
            q.tau[p] = tau;
        }
    }
#pragma unroll
    for (int d = 0; d < DIM; d++) x[d] += pc.hdt * v[d];
    bool dead = false;
    int cc[3] = {0, 0, 0};
#pragma unroll
    for (int d = 0; d < DIM; d++) {
        const double L = (double)g.n[d] * g.dx[d];
        if (g.bc[d] == PERIODIC) {
            if (x[d] < 0.0) x[d] += L;
            if (x[d] >= L) x[d] -= L;
        } else if (x[d] < 0.0 || x[d] >= L) {
            dead = true;
        }
        const int ci = (int)floor(x[d] / g.dx[d]);
        cc[d] = ci < 0 ? 0 : (ci >= g.n[d] ? g.n[d] - 1 : ci);
    }
    if (dead) {
        P.cell[p] = kDead;
        event = 0;
    } else {
        P.cell[p] = pack_cell(g, cc[0], cc[1], cc[2]);
    }
#pragma unroll
    for (int d = 0; d < DIM; d++) P.x[d][p] = x[d];
    q.ev[p] = event;
    if (event) reinterpret_cast<double4 *>(q.evk)[p] = evd;
}

void launch_push_qed_f64(const PartF64 &P, double *F, const Grid &g, const PushConst &pc, const QedParams &q,
                         int *err, double *e_abs, cudaStream_t st)
{
    if (P.n == 0) return;
    note_launch();
    const int nb = div_up(P.n + 1, 256);
    if (g.dim == 1) k_push_qed_f64<1><<<nb, 256, 0, st>>>(P, F, g, pc, q, err, e_abs);
    else if (g.dim == 2) k_push_qed_f64<2><<<nb, 256, 0, st>>>(P, F, g, pc, q, err, e_abs);
    else k_push_qed_f64<3><<<nb, 256, 0, st>>>(P, F, g, pc, q, err, e_abs);
}

void launch_push_photon_f64(const PartF64 &P, const double *F, const Grid &g, const PushConst &pc,
                            const QedParams &q, int *err, cudaStream_t st)
{
    if (P.n == 0) return;
    note_launch();
    const int nb = div_up(P.n + 1, 256);
    if (g.dim == 1) k_push_photon_f64<1><<<nb, 256, 0, st>>>(P, F, g, pc, q, err);
    else if (g.dim == 2) k_push_photon_f64<2><<<nb, 256, 0, st>>>(P, F, g, pc, q, err);
    else k_push_photon_f64<3><<<nb, 256, 0, st>>>(P, F, g, pc, q, err);
}

void launch_push_qed_f32(const PartF32 &P, float *F, const Grid &g, const PushConst &pc, const QedParams &q,
                         int *err, double *e_abs, cudaStream_t st, const uint32_t *first)
{
    if (P.n == 0) return;
    note_launch();
    const int nb = first ? (int)std::min<long long>(div_up(P.n + 1, 256), 152ll * 8) : div_up(P.n + 1, 256);
    if (q.on && q.net) {
        const int sm = kMlpStageBytes;
        if (g.dim == 1) k_push_qed_f32<1, true><<<nb, 256, sm, st>>>(P, F, g, pc, q, err, e_abs, first);
        else if (g.dim == 2) k_push_qed_f32<2, true><<<nb, 256, sm, st>>>(P, F, g, pc, q, err, e_abs, first);
        else k_push_qed_f32<3, true><<<nb, 256, sm, st>>>(P, F, g, pc, q, err, e_abs, first);
    } else {
        if (g.dim == 1) k_push_qed_f32<1, false><<<nb, 256, 0, st>>>(P, F, g, pc, q, err, e_abs, first);
        else if (g.dim == 2) k_push_qed_f32<2, false><<<nb, 256, 0, st>>>(P, F, g, pc, q, err, e_abs, first);
        else k_push_qed_f32<3, false><<<nb, 256, 0, st>>>(P, F, g, pc, q, err, e_abs, first);
    }
}

void launch_push_photon_f32(const PartF32 &P, const float *F, const Grid &g, const PushConst &pc,
                            const QedParams &q, int *err, cudaStream_t st, bool tc, const uint32_t *first)
{
    if (P.n == 0) return;
    note_launch();
    const int nb = first ? (int)std::min<long long>(div_up(P.n + 1, 256), 152ll * 8) : div_up(P.n + 1, 256);
    if (q.on && q.net && tc && !first) {
        const int sm = (int)mlp_tc_smem_bytes();
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_push_photon_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            cudaFuncSetAttribute(k_push_photon_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            cudaFuncSetAttribute(k_push_photon_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            attr = true;
        }
        static int nsm = 0;
        if (!nsm) {
            int dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        }
        const long long tiles = P.n / kMlpTcRows + 1;  // slots 0..P.n
        const int grid = (int)std::min<long long>(tiles, 4ll * nsm);
        if (g.dim == 1) k_push_photon_tc<1><<<grid, kMlpTcRows, sm, st>>>(P, F, g, pc, q, err);
        else if (g.dim == 2) k_push_photon_tc<2><<<grid, kMlpTcRows, sm, st>>>(P, F, g, pc, q, err);
        else k_push_photon_tc<3><<<grid, kMlpTcRows, sm, st>>>(P, F, g, pc, q, err);
    } else if (q.on && q.net) {
        const int sm = kMlpStageBytes;
        if (g.dim == 1) k_push_photon_f32<1, true><<<nb, 256, sm, st>>>(P, F, g, pc, q, err, first);
        else if (g.dim == 2) k_push_photon_f32<2, true><<<nb, 256, sm, st>>>(P, F, g, pc, q, err, first);
        else k_push_photon_f32<3, true><<<nb, 256, sm, st>>>(P, F, g, pc, q, err, first);
    } else {
        if (g.dim == 1) k_push_photon_f32<1, false><<<nb, 256, 0, st>>>(P, F, g, pc, q, err, first);
        else if (g.dim == 2) k_push_photon_f32<2, false><<<nb, 256, 0, st>>>(P, F, g, pc, q, err, first);
        else k_push_photon_f32<3, false><<<nb, 256, 0, st>>>(P, F, g, pc, q, err, first);
    }
}

}  // namespace pic
