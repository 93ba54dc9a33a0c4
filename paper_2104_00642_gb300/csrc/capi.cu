// capi.cu -- host runtime behind the C ABI of include/pic.h: simulation
// state, device memory, step orchestration on one stream, error flags.
//
// Per step n -> n+1 (the split step of Sec. II.F):
//   [sort every K steps] E half (with J^n, then J := 0) -> B half + Mur ->
//   push/deposit every species -> current fold -> B half + Mur -> E half
//   (with J^{n+1}).
// Nothing inside a step waits for the host; the device error flags are read
// once at the end of pic_step.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "diag.cuh"
#include "fdtd.cuh"
#include "sim.cuh"
#include "sort.cuh"

using namespace pic;

namespace {

std::string g_create_error;

}  // namespace

namespace pic {
// message reported by pic_last_error(NULL) for calls that have no pic_sim
void set_global_error(const std::string &msg) { g_create_error = msg; }
}  // namespace pic

namespace pic {

int fail(pic_sim *s, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (s) s->err = buf;
    else g_create_error = buf;
    return code;
}

// every device buffer starts on a 256-byte boundary (vector loads, TMA)
static int raw_alloc(pic_sim *s, void **p, size_t bytes)
{
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (s->alloc_fn) {
        *p = s->alloc_fn(s->alloc_ctx, bytes, (void *)s->st);
        if (!*p) return fail(s, PIC_ERR_NOMEM, "caller allocator: %zu bytes refused", bytes);
        if (reinterpret_cast<uintptr_t>(*p) & 255) {
            s->free_fn(s->alloc_ctx, *p, (void *)s->st);
            *p = nullptr;
            return fail(s, PIC_ERR_NOMEM, "caller allocator: a block not aligned to 256 bytes");
        }
        return PIC_OK;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail(s, PIC_ERR_NOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
    return PIC_OK;
}

static void raw_free(pic_sim *s, void *p)
{
    if (!p) return;
    if (s->alloc_fn) s->free_fn(s->alloc_ctx, p, (void *)s->st);
    else cudaFree(p);
}

int dalloc(pic_sim *s, void **p, size_t bytes)
{
    int rc = raw_alloc(s, p, bytes);
    if (!rc) s->allocs.push_back(*p);
    return rc;
}

int talloc(pic_sim *s, void **p, size_t bytes) { return raw_alloc(s, p, bytes); }
void tfree(pic_sim *s, void *p) { raw_free(s, p); }

}  // namespace pic

namespace {

PartF32 view32(pic_sim *s, int i, int buf)
{
    SpeciesState &p = s->sp[i];
    PartF32 v{};
    v.cell = p.cell[buf];
    for (int d = 0; d < 3; d++) {
        v.off[d] = p.off[buf][d];
        v.u[d] = p.uf[buf][d];
    }
    v.n = p.n_hi;
    v.dn = p.d_count;
    v.tau = p.tau[buf];
    v.id = p.id[buf];
    return v;
}

PartF64 view64(pic_sim *s, int i, int buf)
{
    SpeciesState &p = s->sp[i];
    PartF64 v{};
    v.cell = p.cell[buf];
    for (int d = 0; d < 3; d++) {
        v.x[d] = p.x[buf][d];
        v.u[d] = p.ud[buf][d];
    }
    v.n = p.n_hi;
    v.dn = p.d_count;
    v.tau = p.tau[buf];
    v.id = p.id[buf];
    return v;
}

int ilog2_ceil(long long v)
{
    int b = 0;
    while ((1ll << b) < v) b++;
    return b;
}

PushConst push_const(const pic_sim *s, const SpeciesState &p)
{
    PushConst pc{};
    const Grid &g = s->g;
    pc.qmdt2 = p.q / p.m * 0.5 * g.dt;
    pc.qw = p.q * p.w;
    pc.hdt = 0.5 * g.dt;
    double dV = 1.0;
    for (int d = 0; d < 3; d++) {
        pc.hdx[d] = 0.5 * g.dt / g.dx[d];
        pc.cJ[d] = -p.q * p.w * g.dx[d] / g.dt;
        if (d < g.dim) dV *= g.dx[d];
    }
    pc.wmdV = p.w * p.m * dV;
    pc.pusher = s->pusher;
    pc.qmdt2_f = (float)pc.qmdt2;
    pc.qw_f = (float)pc.qw;
    for (int d = 0; d < 3; d++) {
        pc.hdx_f[d] = (float)pc.hdx[d];
        pc.cJ_f[d] = (float)pc.cJ[d];
    }
    return pc;
}

// counting sort of one species by tile into the other buffer
int sort_species(pic_sim *s, int i)
{
    SpeciesState &p = s->sp[i];
    if (p.n_hi == 0) return PIC_OK;
    const uint32_t *perm = nullptr, *skeys = nullptr;
    sort_by_tile(p.cell[p.cur], p.n_hi, p.d_count, s->g, s->sort_scratch, p.tile_start, p.d_count, &perm, &skeys,
                 s->st);
    int o = 1 - p.cur;
    if (s->precision == PIC_PREC_FP64_PLAIN)
        launch_permute_f64(view64(s, i, p.cur), view64(s, i, o), perm, p.d_count, p.n_hi, s->g.dim, s->st);
    else
        launch_permute_f32(view32(s, i, p.cur), view32(s, i, o), perm, p.d_count, p.n_hi, s->g.dim, s->st);
    p.cur = o;
    if (p.items) {
        build_tile_items(p.tile_start, s->g.ntiles, s->g.dim, p.item_cnt, p.item_scan, p.items, p.nitems, s->st);
        p.items_valid = true;
    }
    CK(cudaGetLastError());
    return PIC_OK;
}

bool use_tile_push(const pic_sim *s, const SpeciesState &p)
{
    // the tiled kernels stage order-2 stencils; order 4 runs on the simple kernels
    if (s->push_variant == PIC_PUSH_SIMPLE || !p.items_valid || s->precision != PIC_PREC_FP32_CELLOFF ||
        s->g.order != 2 || p.kind != PIC_KIND_MASSIVE)
        return false;
    if (s->g.dim == 3) return tile3d_push_supported(s->g);
    return s->g.dim == 2 && s->g.tile_log2[0] == s->g.tile_log2[1] &&
           (s->g.tile_log2[0] == 3 || s->g.tile_log2[0] == 4);
}

// photons: the tiled photon push (2D) on the work items of the last sort
bool use_tile_photon_push(const pic_sim *s, const SpeciesState &p)
{
    if (s->push_variant == PIC_PUSH_SIMPLE || s->push_variant == PIC_PUSH_MLP_TC || !p.items_valid ||
        s->precision != PIC_PREC_FP32_CELLOFF || p.kind != PIC_KIND_PHOTON)
        return false;
    return s->g.dim == 2 && s->g.tile_log2[0] == s->g.tile_log2[1] &&
           (s->g.tile_log2[0] == 3 || s->g.tile_log2[0] == 4);
}

int read_count(pic_sim *s, int i, long long *n)
{
    CK(cudaMemcpyAsync(n, s->sp[i].d_count, sizeof(long long), cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    s->sp[i].n_hi = *n;
    return PIC_OK;
}

// exchange box (x fastest): [0,N) periodic, [0,N] absorbing
void out_box(const Grid &g, long long *m)
{
    for (int d = 0; d < 3; d++)
        m[d] = d >= g.dim ? 1 : (g.bc[d] == ABSORB ? g.n[d] + 1 : g.n[d]);
}

template <typename R>
int copy_comp_out(pic_sim *s, const R *dev, double *host_out)
{
    const Grid &g = s->g;
    std::vector<R> h((size_t)g.vol);
    CK(cudaMemcpyAsync(h.data(), dev, (size_t)g.vol * sizeof(R), cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    long long m[3];
    out_box(g, m);
    for (long long k = 0; k < m[2]; k++)
        for (long long j = 0; j < m[1]; j++)
            for (long long i = 0; i < m[0]; i++)
                host_out[(k * m[1] + j) * m[0] + i] = (double)h[(size_t)goff(g, (int)i, (int)j, (int)k)];
    return PIC_OK;
}

template <typename R>
int copy_comp_in(pic_sim *s, R *dev, const double *host_in)
{
    const Grid &g = s->g;
    std::vector<R> h((size_t)g.vol);
    CK(cudaMemcpyAsync(h.data(), dev, (size_t)g.vol * sizeof(R), cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    long long m[3];
    out_box(g, m);
    // every padded cell whose (periodic image of the) index lies in the box
    for (int k = -g.G[2]; k < g.n[2] + g.G[2]; k++)
        for (int j = -g.G[1]; j < g.n[1] + g.G[1]; j++)
            for (int i = -g.G[0]; i < g.n[0] + g.G[0]; i++) {
                int p[3] = {i, j, k};
                bool in = true;
                for (int d = 0; d < 3 && in; d++) {
                    if (d >= g.dim) continue;
                    if (g.bc[d] == PERIODIC) p[d] = ((p[d] % g.n[d]) + g.n[d]) % g.n[d];
                    else if (p[d] < 0 || p[d] >= m[d]) in = false;
                }
                if (!in) continue;
                h[(size_t)goff(g, i, j, k)] = (R)host_in[((long long)p[2] * m[1] + p[1]) * m[0] + p[0]];
            }
    CK(cudaMemcpyAsync(dev, h.data(), (size_t)g.vol * sizeof(R), cudaMemcpyHostToDevice, s->st));
    CK(cudaStreamSynchronize(s->st));
    return PIC_OK;
}

int compute_rho(pic_sim *s)
{
    const Grid &g = s->g;
    CK(cudaMemsetAsync(s->rho, 0, (size_t)g.vol * sizeof(double), s->st));
    for (int i = 0; i < s->nsp; i++) {
        SpeciesState &p = s->sp[i];
        if (p.n_hi == 0) continue;
        if (s->precision == PIC_PREC_FP64_PLAIN) diag_rho_f64(view64(s, i, p.cur), g, p.q * p.w, s->rho, s->st);
        else diag_rho_f32(view32(s, i, p.cur), g, p.q * p.w, s->rho, s->st);
    }
    launch_fold_rho(s->rho, g, s->st);
    CK(cudaGetLastError());
    return PIC_OK;
}

void ph_begin(pic_sim *s)
{
    s->cur_l0 = g_launches;
    if (!s->prof) return;
    cudaEventCreate(&s->cur_a);
    cudaEventRecord(s->cur_a, s->st);
}

void ph_end(pic_sim *s, int phase)
{
    if (!s->prof) return;
    cudaEvent_t b;
    cudaEventCreate(&b);
    cudaEventRecord(b, s->st);
    s->marks.push_back({phase, s->cur_a, b});
    s->prof_launch[phase] += g_launches - s->cur_l0;
}

// the laser view for a B update that ends at t_new (the Mur condition needs
// B_inc(x, t) = E_L(t - x) at x = -/+ dx/2 and at the new and old B times)
Laser laser_at(const pic_sim *s, double t_new)
{
    Laser L = s->laser;
    if (!L.on) return L;
    const double h = 0.5 * s->g.dt, hx = 0.5 * s->g.dx[0];
    const double tau[4] = {t_new + hx, t_new - h + hx, t_new - hx, t_new - h - hx};
    const double two_pi = 6.283185307179586476925286766559;
    for (int q = 0; q < 4; q++) {
        const double a = (tau[q] - s->lp.t_peak) / s->lp.fwhm;
        L.env[q] = std::exp(-2.0 * 0.69314718055994530942 * a * a);
        L.ph0[q] = std::fmod(tau[q] - s->lp.t_peak, two_pi);
    }
    return L;
}

QedParams qed_params(pic_sim *s, int i)
{
    SpeciesState &p = s->sp[i];
    QedParams q{};
    const double alpha = 1.0 / 137.035999084;
    // (photons: only the QED photon species converts; the spawn takes its events)
    q.on = s->qed_on && (p.kind == PIC_KIND_PHOTON
                             ? (i == s->qed.photon_sp && s->qed.electron_sp >= 0 && s->qed.positron_sp >= 0)
                             : (p.qed && s->qed.photon_sp >= 0));
    q.method = s->qed.method == PIC_QED_METHOD2 ? 2 : 1;
    q.pref = alpha * s->Es * s->g.dt / (std::sqrt(3.0) * 3.14159265358979323846);
    q.inv_Es = s->Es > 0.0 ? 1.0 / s->Es : 0.0;
    q.pref_f = (float)q.pref;
    q.inv_Es_f = (float)q.inv_Es;
    q.emin = s->qed.photon_emin;
    q.key[0] = (uint32_t)s->seed;
    q.key[1] = (uint32_t)(s->seed >> 32);
    q.step = (uint32_t)s->step;
    q.T = s->T;
    q.tau = p.tau[p.cur];
    q.id = p.id[p.cur];
    q.ev = p.ev;
    q.evk = p.evk;
    q.e_lost = s->d_elost;
    double dV = 1.0;
    for (int d = 0; d < s->g.dim; d++) dV *= s->g.dx[d];
    q.wdV = p.w * dV;
    const MlpNet &net = s->net[p.kind == PIC_KIND_PHOTON ? QED_PAIR : QED_RAD];
    const bool surr = s->qed.mode == PIC_QED_SURROGATE && net.ready && s->precision == PIC_PREC_FP32_CELLOFF;
    q.net = surr ? net.img : nullptr;
    q.nrm = net.nrm;
    q.net_lo_f = (float)net.nrm.lnchi_lo;
    q.net_hi_f = (float)net.nrm.lnchi_hi;
    q.cq = surr && p.kind == PIC_KIND_PHOTON ? s->cand_q : nullptr;
    q.cq_n = s->cand_n;
    return q;
}

void push_species(pic_sim *s, int i, float *F)
{
    SpeciesState &p = s->sp[i];
    if (p.kind == PIC_KIND_PHOTON) {
        const QedParams q = qed_params(s, i);
        const PartF32 P = view32(s, i, p.cur);
        if (use_tile_photon_push(s, p)) {
            // the photons sorted into work items on the tiled kernel, then
            // those emitted since, as items of consecutive photons
            const long long max_items = (long long)tile_items_capacity(p.n_hi, s->g.ntiles, s->g.dim);
            if (q.on && q.net) cudaMemsetAsync(q.cq_n, 0, sizeof(uint32_t), s->st);  // the candidates' queue
            launch_push_photon_tile2d(P, p.items, p.nitems, max_items, F, s->g, push_const(s, p), q, s->d_err, s->st);
            // the photons appended since the sort: items of consecutive
            // photons (appended in their parents' tile order), on the same kernel
            launch_tail_items(P, p.tile_start + s->g.ntiles, s->g, p.tail_items, p.tail_nitems, s->st);
            launch_push_photon_tile2d(P, p.tail_items, p.tail_nitems, (long long)tail_items_capacity(p.n_hi), F, s->g,
                                      push_const(s, p), q, s->d_err, s->st);
            launch_photon_resolve(q, P, s->d_err, s->st);
        } else {
            launch_push_photon_f32(P, F, s->g, push_const(s, p), q, s->d_err, s->st,
                                   s->push_variant == PIC_PUSH_MLP_TC);
        }
        return;
    }
    if (s->qed_on && p.qed) {
        const QedParams q = qed_params(s, i);
        const PartF32 P = view32(s, i, p.cur);
        if (use_tile_push(s, p)) {
            // the particles sorted into work items on the tiled kernel, those
            // appended since (pairs) on the one-thread-per-particle kernel
            const long long max_items = (long long)tile_items_capacity(p.n_hi, s->g.ntiles, s->g.dim);
            if (s->g.dim == 3)
                launch_push_tile3d(P, p.items, p.nitems, max_items, F, s->g, push_const(s, p), s->d_err, s->d_eabs,
                                   p.defer + 1, p.defer, s->st, &q);
            else
                launch_push_tile2d(P, p.items, p.nitems, max_items, F, s->g, push_const(s, p), s->d_err,
                                   s->d_eabs, s->st, true, &q);
            launch_push_qed_f32(P, F, s->g, push_const(s, p), q, s->d_err, s->d_eabs, s->st,
                                p.tile_start + s->g.ntiles);
        } else {
            launch_push_qed_f32(P, F, s->g, push_const(s, p), q, s->d_err, s->d_eabs, s->st);
        }
        return;
    }
    if (use_tile_push(s, p)) {
        const long long max_items = (long long)tile_items_capacity(p.n_hi, s->g.ntiles, s->g.dim);
        if (s->g.dim == 3)
            launch_push_tile3d(view32(s, i, p.cur), p.items, p.nitems, max_items, F, s->g, push_const(s, p), s->d_err,
                               s->d_eabs, p.defer + 1, p.defer, s->st);
        else
            launch_push_tile2d(view32(s, i, p.cur), p.items, p.nitems, max_items, F, s->g, push_const(s, p), s->d_err,
                               s->d_eabs, s->st, s->push_variant == PIC_PUSH_TILE_AGG);
    } else
        launch_push_f32(view32(s, i, p.cur), F, s->g, push_const(s, p), s->d_err, s->d_eabs, s->st);
}

void push_species(pic_sim *s, int i, double *F)
{
    SpeciesState &p = s->sp[i];
    if (p.kind == PIC_KIND_PHOTON) {
        launch_push_photon_f64(view64(s, i, p.cur), F, s->g, push_const(s, p), qed_params(s, i), s->d_err, s->st);
        return;
    }
    if (s->qed_on && p.qed) {
        launch_push_qed_f64(view64(s, i, p.cur), F, s->g, push_const(s, p), qed_params(s, i), s->d_err, s->d_eabs,
                            s->st);
        return;
    }
    launch_push_f64(view64(s, i, p.cur), F, s->g, push_const(s, p), s->d_err, s->d_eabs, s->st);
}

// Append this step's QED children, in a fixed order: first the pairs of the
// photons that converted (electrons, then positrons, in photon order), then
// the photons emitted by each emitting species in species order (in parent
// order).  The event flags are ranked in array order.
template <typename R>
void qed_spawn_views(pic_sim *s)
{
    auto view = [&](int i) {
        if constexpr (sizeof(R) == 8) return view64(s, i, s->sp[i].cur);
        else return view32(s, i, s->sp[i].cur);
    };
    uint32_t *off = (uint32_t *)s->sort_scratch;
    const int ph = s->qed.photon_sp, el = s->qed.electron_sp, po = s->qed.positron_sp;
    const int dim = s->g.dim;
    // the scanned sums of the flags' blocks (the spawn kernels rank within a block)
    auto scan = [&](const SpeciesState &p) {
        const long long nb = scan_blocks(p.n_hi + 1);
        scan_block_sums(p.ev, p.n_hi + 1, off, off + nb + 64, s->st, p.d_count);
        return off + nb;  // total
    };
    if (ph >= 0 && el >= 0 && po >= 0 && s->sp[ph].n_hi > 0) {
        SpeciesState &P = s->sp[ph], &E = s->sp[el], &O = s->sp[po];
        const uint32_t *tot = scan(P);
        launch_spawn_pairs(view(ph), off, tot, P.n_hi + 1, qed_params(s, ph), view(el), E.tau[E.cur], E.id[E.cur], E.ev,
                           E.d_count, E.cap, view(po), O.tau[O.cur], O.id[O.cur], O.ev, O.d_count, O.cap, dim,
                           s->d_err, s->st);
        E.n_hi = std::min(E.cap, E.n_hi + P.n_hi);
        O.n_hi = std::min(O.cap, O.n_hi + P.n_hi);
        // the pairs land past the sorted particles (tile_start[ntiles]): the
        // work items stay valid for the ones before, the QED lepton push
        // takes the rest on its one-thread-per-particle kernel
        if (!E.qed) E.items_valid = false;
        if (!O.qed) O.items_valid = false;
    }
    if (ph < 0) return;
    for (int i = 0; i < s->nsp; i++) {
        SpeciesState &p = s->sp[i];
        if (p.kind == PIC_KIND_PHOTON || !p.qed || p.n_hi == 0) continue;
        SpeciesState &P = s->sp[ph];
        const uint32_t *tot = scan(p);
        launch_spawn_photons(view(i), off, tot, p.n_hi + 1, qed_params(s, i), view(ph), P.tau[P.cur], P.id[P.cur], P.ev,
                             P.d_count, P.cap, dim, s->d_err, s->st);
        P.n_hi = std::min(P.cap, P.n_hi + p.n_hi);
        // (the photons land past the sorted ones: the photon push takes them
        // as items of consecutive photons, the sort's work items stay valid)
    }
}

void qed_spawn(pic_sim *s)
{
    if (!s->qed_on) return;
    if (s->precision == PIC_PREC_FP64_PLAIN) qed_spawn_views<double>(s);
    else qed_spawn_views<float>(s);
}

// nsteps split steps (Sec. II.F).  The first half step of a call runs
// alone; between steps the second E half step of step n and the first of
// step n+1 are one fused launch (the same curl B and J^{n+1} applied twice);
// the last step of a call ends with its own E half step, so fields and
// particles are at the integer step when the call returns.
template <typename R>
int step_loop(pic_sim *s, int64_t nsteps)
{
    const Grid &g = s->g;
    const double h = 0.5 * g.dt;
    R *F = (R *)s->F;
    for (int64_t it = 0; it < nsteps; it++) {
        if (s->sort_interval > 0 && s->step % s->sort_interval == 0) {
            ph_begin(s);
            for (int i = 0; i < s->nsp; i++) {
                int rc = sort_species(s, i);
                if (rc) return rc;
            }
            ph_end(s, PIC_PHASE_SORT);
        }
        const double t0 = (double)s->step * g.dt;
        if (it == 0) {
            ph_begin(s);
            launch_update_E<R>(F, g, h, false, true, s->st);  // E^{n+1/2}, then J := 0
            launch_update_B<R>(F, g, h, t0 + h, laser_at(s, t0 + h), s->st);
            ph_end(s, PIC_PHASE_FIELDS);
        }
        ph_begin(s);
        for (int i = 0; i < s->nsp; i++) {
            if (s->sp[i].n_hi) s->prof_push++;
            cudaEvent_t sa = nullptr;
            if (s->prof && s->sp[i].n_hi) {
                cudaEventCreate(&sa);
                cudaEventRecord(sa, s->st);
            }
            push_species(s, i, F);
            if (sa) {
                cudaEvent_t sb;
                cudaEventCreate(&sb);
                cudaEventRecord(sb, s->st);
                s->marks.push_back({PIC_NPHASE + i, sa, sb});
            }
        }
        qed_spawn(s);
        ph_end(s, PIC_PHASE_PUSH);
        ph_begin(s);
        launch_fold<R>(F, g, s->st);
        ph_end(s, PIC_PHASE_FOLD);
        ph_begin(s);
        launch_update_B<R>(F, g, h, t0 + g.dt, laser_at(s, t0 + g.dt), s->st);  // B^{n+1}
        if (it == nsteps - 1) {
            launch_update_E<R>(F, g, h, false, false, s->st);  // E^{n+1}
        } else {
            launch_update_E<R>(F, g, h, true, true, s->st);  // E^{n+3/2}, then J := 0
            launch_update_B<R>(F, g, h, t0 + g.dt + h, laser_at(s, t0 + g.dt + h), s->st);  // B^{n+3/2}
        }
        ph_end(s, PIC_PHASE_FIELDS);
        CK(cudaGetLastError());
        s->step++;
    }
    return PIC_OK;
}

int check_flags(pic_sim *s)
{
    int h = 0;
    CK(cudaMemcpyAsync(&h, s->d_err, sizeof(int), cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    if (h) {
        CK(cudaMemsetAsync(s->d_err, 0, sizeof(int), s->st));
        if (h & ERR_NONFINITE) return fail(s, PIC_ERR_NONFINITE, "non-finite particle momentum");
        if (h & ERR_CFL) return fail(s, PIC_ERR_CFL, "a particle moved more than one cell in a step");
        if (h & ERR_QEDDT)
            return fail(s, PIC_ERR_CFL,
                        "QED: an acceptance probability above one (Method II: dt too long for it; surrogate: the "
                        "pair network's rate above the thinning envelope)");
        if (h & ERR_CAPACITY) return fail(s, PIC_ERR_CAPACITY, "species capacity exceeded");
        if (h & ERR_TIMEOUT)
            return fail(s, PIC_ERR_TIMEOUT, "a bounded wait in a kernel ran out (bulk copy or tensor-core commit)");
    }
    return PIC_OK;
}

}  // namespace

// ---------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------
extern "C" {

int pic_create(const pic_grid *grid, double dt, const pic_species *species, int nsp, const pic_options *opt,
               pic_sim **out)
{
    if (out) *out = nullptr;
    pic_sim *s = nullptr;
    if (!grid || !out || (nsp > 0 && !species) || nsp < 0 || nsp > PIC_MAX_SPECIES)
        return fail(s, PIC_ERR_ARG, "pic_create: null argument or bad species count");
    // the caller's options, copied by the size it was compiled with
    pic_options o{};
    if (opt) {
        if (opt->struct_size != (int)sizeof(pic_options))
            return fail(s, PIC_ERR_ARG, "pic_create: pic_options.struct_size is %d, this library expects %d",
                        opt->struct_size, (int)sizeof(pic_options));
        std::memcpy(&o, opt, sizeof o);
        if ((o.alloc == nullptr) != (o.free == nullptr))
            return fail(s, PIC_ERR_ARG, "pic_create: give both alloc and free, or neither");
        opt = &o;
    }
    if (grid->dim < 1 || grid->dim > 3) return fail(s, PIC_ERR_ARG, "pic_create: dim must be 1, 2 or 3");
    if (grid->order != 2 && grid->order != 4) return fail(s, PIC_ERR_ARG, "pic_create: shape order must be 2 or 4");
    int prec = opt ? opt->precision : PIC_PREC_FP32_CELLOFF;
    if (prec != PIC_PREC_FP32_CELLOFF && prec != PIC_PREC_FP64_PLAIN)
        return fail(s, PIC_ERR_ARG, "pic_create: unknown precision");
    if (opt && (opt->push_variant < PIC_PUSH_AUTO || opt->push_variant > PIC_PUSH_TILE_AGG))
        return fail(s, PIC_ERR_ARG, "pic_create: unknown push variant");
    if (opt && opt->pusher != PIC_PUSHER_BORIS && opt->pusher != PIC_PUSHER_VAY)
        return fail(s, PIC_ERR_ARG, "pic_create: unknown pusher");
    Grid g{};
    g.dim = grid->dim;
    g.order = grid->order;
    g.dt = dt;
    double cfl = 0.0;
    int bitsum = 0;
    for (int d = 0; d < 3; d++) {
        bool act = d < g.dim;
        if (act) {
            if (grid->n[d] < 1 || grid->n[d] > (1 << 24) || !(grid->dx[d] > 0.0))
                return fail(s, PIC_ERR_ARG, "pic_create: bad n/dx on axis %d", d);
            if (grid->bc[d] != PIC_BC_PERIODIC && grid->bc[d] != PIC_BC_ABSORB)
                return fail(s, PIC_ERR_ARG, "pic_create: bad boundary on axis %d", d);
            if (grid->bc[d] == PIC_BC_PERIODIC && grid->n[d] < 2 * kGhost)
                return fail(s, PIC_ERR_ARG, "pic_create: periodic axis %d needs n >= %d", d, 2 * kGhost);
            cfl += 1.0 / (grid->dx[d] * grid->dx[d]);
        }
        g.n[d] = act ? (int)grid->n[d] : 1;
        g.dx[d] = act ? grid->dx[d] : 1.0;
        g.rdx_d[d] = 1.0 / g.dx[d];
        g.rdx_f[d] = (float)g.rdx_d[d];
        g.bc[d] = act ? grid->bc[d] : PERIODIC;
        g.G[d] = act ? kGhost : 0;
        g.ext[d] = g.n[d] + 2 * g.G[d];
        g.bits[d] = act ? ilog2_ceil(g.n[d]) : 0;
        bitsum += g.bits[d];
        int t = opt && opt->tile[d] > 0 ? opt->tile[d] : (g.dim == 1 ? 64 : (g.dim == 2 ? 16 : 8));
        if (!act) t = 1;
        if (t & (t - 1)) return fail(s, PIC_ERR_ARG, "pic_create: tile sizes must be powers of two");
        g.tile_log2[d] = ilog2_ceil(t);
        g.ntile[d] = (g.n[d] + t - 1) / t;
    }
    if (bitsum > 31) return fail(s, PIC_ERR_ARG, "pic_create: grid too large for the packed cell index");
    if (!(dt > 0.0) || dt * std::sqrt(cfl) >= 1.0)
        return fail(s, PIC_ERR_CFL, "pic_create: dt=%g violates the Courant limit %g", dt, 1.0 / std::sqrt(cfl));
    g.ntiles = (long long)g.ntile[0] * g.ntile[1] * g.ntile[2];
    long long pitch = ((g.ext[0] + 31) / 32) * 32;
    g.sy = pitch;
    g.sz = pitch * g.ext[1];
    g.vol = ((g.sz * g.ext[2] + 63) / 64) * 64;
    g.origin = (long long)g.G[2] * g.sz + (long long)g.G[1] * g.sy + g.G[0];
    if (g.vol >= (1ll << 31))  // kernels address one component with 32-bit offsets
        return fail(s, PIC_ERR_ARG, "pic_create: padded grid of %lld cells exceeds 2^31", g.vol);

    s = new pic_sim();
    s->g = g;
    s->precision = prec;
    s->sort_interval = opt ? opt->sort_interval : 0;
    s->push_variant = opt ? opt->push_variant : PIC_PUSH_AUTO;
    s->pusher = opt ? opt->pusher : PIC_PUSHER_BORIS;
    s->seed = opt ? opt->seed : 0;
    s->rho_bg = opt ? opt->rho_bg : 0.0;
    s->st = opt ? (cudaStream_t)opt->stream : nullptr;
    s->alloc_fn = opt ? opt->alloc : nullptr;
    s->free_fn = opt ? opt->free : nullptr;
    s->alloc_ctx = opt ? opt->alloc_ctx : nullptr;
    s->nsp = nsp;
    int dev_count = 0;
    cudaError_t e = cudaGetDeviceCount(&dev_count);
    if (e != cudaSuccess || dev_count == 0) {
        int rc = fail(nullptr, PIC_ERR_CUDA, "pic_create: no CUDA device (%s)", cudaGetErrorString(e));
        delete s;
        return rc;
    }
    int rc = PIC_OK;
    size_t R = rsize(s);
    long long maxcap = 0;
    rc = rc ? rc : dalloc(s, &s->F, (size_t)NCOMP * g.vol * R);
    rc = rc ? rc : dalloc(s, (void **)&s->rho, (size_t)g.vol * sizeof(double));
    for (int i = 0; i < nsp && !rc; i++) {
        SpeciesState &p = s->sp[i];
        const pic_species &q = species[i];
        const bool photon = q.kind == PIC_KIND_PHOTON;
        if ((q.kind != PIC_KIND_MASSIVE && !photon) || (!photon && !(q.m > 0.0)) ||
            (photon && (q.q != 0.0 || q.m != 0.0 || q.qed)) || q.capacity < 0 || q.capacity > 0x7FFFFFFFll) {
            rc = fail(s, PIC_ERR_ARG, "pic_create: bad species %d", i);
            break;
        }
        p.q = q.q;
        p.m = q.m;
        p.w = q.w;
        p.cap = q.capacity;
        p.kind = q.kind;
        p.qed = q.qed;
        if (photon || q.qed) {
            for (int b = 0; b < 2 && !rc; b++) {
                rc = dalloc(s, (void **)&p.tau[b], (size_t)p.cap * 8);
                rc = rc ? rc : dalloc(s, (void **)&p.id[b], (size_t)p.cap * 8);
            }
            rc = rc ? rc : dalloc(s, (void **)&p.ev, (size_t)(p.cap + 1) * 4);
            // event data: 4 floats per particle, 4 doubles in the FP64 form
            rc = rc ? rc : dalloc(s, (void **)&p.evk, (size_t)(p.cap + 1) * 4 * rsize(s));
        }
        maxcap = std::max(maxcap, p.cap);
        rc = rc ? rc : dalloc(s, (void **)&p.d_count, sizeof(long long));
        rc = rc ? rc : dalloc(s, (void **)&p.tile_start, (size_t)(g.ntiles + 1) * sizeof(uint32_t));
        if (prec == PIC_PREC_FP32_CELLOFF && (g.dim == 2 || (g.dim == 3 && tile3d_push_supported(g)))) {
            p.items_cap = (long long)tile_items_capacity(p.cap, g.ntiles, g.dim);
            rc = rc ? rc : dalloc(s, (void **)&p.items, (size_t)p.items_cap * sizeof(TileItem));
            rc = rc ? rc : dalloc(s, (void **)&p.nitems, sizeof(uint32_t));
            rc = rc ? rc : dalloc(s, (void **)&p.item_cnt, (size_t)(g.ntiles + 1) * sizeof(uint32_t));
            rc = rc ? rc : dalloc(s, (void **)&p.item_scan, scan_scratch_words(g.ntiles + 1) * sizeof(uint32_t));
            if (g.dim == 3) rc = rc ? rc : dalloc(s, (void **)&p.defer, (size_t)(p.cap + 1) * sizeof(uint32_t));
            if (photon && g.dim == 2) {
                rc = rc ? rc : dalloc(s, (void **)&p.tail_items, tail_items_capacity(p.cap) * sizeof(TileItem));
                rc = rc ? rc : dalloc(s, (void **)&p.tail_nitems, sizeof(uint32_t));
            }
        }
        for (int b = 0; b < 2 && !rc; b++) {
            rc = dalloc(s, (void **)&p.cell[b], (size_t)p.cap * 4);
            for (int d = 0; d < 3 && !rc; d++) {
                if (prec == PIC_PREC_FP64_PLAIN) {
                    if (d < g.dim) rc = dalloc(s, (void **)&p.x[b][d], (size_t)p.cap * 8);
                    if (!rc) rc = dalloc(s, (void **)&p.ud[b][d], (size_t)p.cap * 8);
                } else {
                    if (d < g.dim) rc = dalloc(s, (void **)&p.off[b][d], (size_t)p.cap * 4);
                    if (!rc) rc = dalloc(s, (void **)&p.uf[b][d], (size_t)p.cap * 4);
                }
            }
        }
    }
    rc = rc ? rc : dalloc(s, &s->sort_scratch, sort_scratch_bytes(maxcap));
    rc = rc ? rc : dalloc(s, (void **)&s->diag_scratch, diag_scratch_doubles() * sizeof(double));
    rc = rc ? rc : dalloc(s, (void **)&s->diag_out, 16 * sizeof(double));
    rc = rc ? rc : dalloc(s, (void **)&s->d_err, sizeof(int));
    rc = rc ? rc : dalloc(s, (void **)&s->d_eabs, sizeof(double));
    rc = rc ? rc : dalloc(s, (void **)&s->d_elost, sizeof(double));
    if (!rc) {
        cudaError_t z = cudaMemsetAsync(s->F, 0, (size_t)NCOMP * g.vol * R, s->st);
        if (z == cudaSuccess) z = cudaMemsetAsync(s->d_err, 0, sizeof(int), s->st);
        if (z == cudaSuccess) z = cudaMemsetAsync(s->d_eabs, 0, sizeof(double), s->st);
        if (z == cudaSuccess) z = cudaMemsetAsync(s->d_elost, 0, sizeof(double), s->st);
        for (int i = 0; i < nsp && z == cudaSuccess; i++)
            if (s->sp[i].ev) z = cudaMemsetAsync(s->sp[i].ev, 0, (size_t)(s->sp[i].cap + 1) * 4, s->st);
        for (int i = 0; i < nsp && z == cudaSuccess; i++)
            z = cudaMemsetAsync(s->sp[i].d_count, 0, sizeof(long long), s->st);
        if (z == cudaSuccess) z = cudaStreamSynchronize(s->st);
        if (z != cudaSuccess) rc = fail(s, PIC_ERR_CUDA, "pic_create: %s", cudaGetErrorString(z));
    }
    if (rc) {
        g_create_error = s->err;
        pic_destroy(s);
        return rc;
    }
    *out = s;
    return PIC_OK;
}

void pic_destroy(pic_sim *s)
{
    if (!s) return;
    if (s->st) cudaStreamSynchronize(s->st);
    else cudaDeviceSynchronize();
    for (void *p : s->allocs) raw_free(s, p);
    delete s;
}

const char *pic_last_error(const pic_sim *s) { return s ? s->err.c_str() : g_create_error.c_str(); }

int pic_sync(pic_sim *s)
{
    if (!s) return PIC_ERR_ARG;
    CK(cudaStreamSynchronize(s->st));
    return PIC_OK;
}

// the device address of a page-locked, mapped host array, else nullptr
static const double *mapped_device_ptr(const double *h)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
        cudaGetLastError();  // not a pointer the runtime knows: clear the error
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost && a.devicePointer ? static_cast<const double *>(a.devicePointer) : nullptr;
}

int pic_load_particles(pic_sim *s, int sp, int64_t n, const double *x, const double *y, const double *z,
                       const double *ux, const double *uy, const double *uz)
{
    if (!s) return PIC_ERR_ARG;
    if (sp < 0 || sp >= s->nsp || n < 0) return fail(s, PIC_ERR_ARG, "pic_load_particles: bad species or count");
    if (n == 0) return PIC_OK;
    const Grid &g = s->g;
    const double *xs[3] = {x, y, z};
    const double *us[3] = {ux, uy, uz};
    for (int d = 0; d < 3; d++)
        if (!us[d] || (d < g.dim && !xs[d])) return fail(s, PIC_ERR_ARG, "pic_load_particles: null array");
    SpeciesState &p = s->sp[sp];
    long long cnt = 0;
    int rc = read_count(s, sp, &cnt);
    if (rc) return rc;
    if (cnt + n > p.cap) return fail(s, PIC_ERR_CAPACITY, "pic_load_particles: capacity %lld exceeded", p.cap);
    // Page-locked host arrays mapped into the device's address space are read
    // in place by the load kernel; any other host array goes through a device
    // staging buffer first.
    const double *cx[3] = {nullptr, nullptr, nullptr}, *cu[3] = {nullptr, nullptr, nullptr};
    bool direct = true;
    for (int d = 0; d < 3; d++) {
        direct &= (cu[d] = mapped_device_ptr(us[d])) != nullptr;
        if (d < g.dim) direct &= (cx[d] = mapped_device_ptr(xs[d])) != nullptr;
    }
    const size_t stage = direct ? 0 : (size_t)n * 6 * sizeof(double);
    double *dtmp = nullptr;
    if (int rc_ = talloc(s, (void **)&dtmp, stage + sizeof(unsigned long long))) return rc_;
    unsigned long long *dbad = reinterpret_cast<unsigned long long *>((char *)dtmp + stage), hbad = ~0ull;
    cudaError_t e = cudaMemsetAsync(dbad, 0xFF, sizeof(unsigned long long), s->st);
    if (!direct) {
        for (int d = 0; d < 3 && e == cudaSuccess; d++) {
            double *dxd = dtmp + (size_t)d * n, *dud = dtmp + (size_t)(3 + d) * n;
            if (d < g.dim) e = cudaMemcpyAsync(dxd, xs[d], n * sizeof(double), cudaMemcpyHostToDevice, s->st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(dud, us[d], n * sizeof(double), cudaMemcpyHostToDevice, s->st);
            cx[d] = d < g.dim ? dxd : nullptr;
            cu[d] = dud;
        }
    }
    if (e == cudaSuccess) {
        if (s->precision == PIC_PREC_FP64_PLAIN) launch_load_f64(view64(s, sp, p.cur), cnt, n, cx, cu, g, dbad, s->st);
        else launch_load_f32(view32(s, sp, p.cur), cnt, n, cx, cu, g, dbad, s->st);
        e = cudaGetLastError();
    }
    // the positions and momenta are checked on the device (a host loop over
    // them cost more than the upload); the count moves only if all passed
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, dbad, sizeof hbad, cudaMemcpyDeviceToHost, s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    if (e == cudaSuccess && hbad != ~0ull) {
        tfree(s, dtmp);
        return fail(s, PIC_ERR_ARG, "pic_load_particles: particle %llu outside the domain or with a non-finite u",
                    hbad);
    }
    long long newn = cnt + n;
    if (e == cudaSuccess) e = cudaMemcpyAsync(p.d_count, &newn, sizeof(long long), cudaMemcpyHostToDevice, s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    tfree(s, dtmp);
    if (e != cudaSuccess) return fail(s, PIC_ERR_CUDA, "pic_load_particles: %s", cudaGetErrorString(e));
    p.n_hi = newn;
    p.items_valid = false;  // appended particles are in no tile's work item until the next sort
    if (p.has_qed_arrays()) {
        // identity (species << 48) | load index, optical depth -ln r of its Philox draw
        const uint32_t key[2] = {(uint32_t)s->seed, (uint32_t)(s->seed >> 32)};
        launch_init_qed(cnt, n, (uint64_t)sp << 48, p.id[p.cur], p.tau[p.cur], key, s->st);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(s->st));
    }
    return PIC_OK;
}

int pic_set_qed(pic_sim *s, const pic_qed *Q)
{
    if (!s || !Q) return PIC_ERR_ARG;
    if (Q->mode != PIC_QED_OFF && Q->mode != PIC_QED_TABLE && Q->mode != PIC_QED_SURROGATE)
        return fail(s, PIC_ERR_ARG, "pic_set_qed: bad mode");
    if (Q->mode != PIC_QED_OFF && s->g.order != 2)
        return fail(s, PIC_ERR_ARG, "pic_set_qed: the QED push kernels use the order-2 shape");
    if (Q->method != 0 && Q->method != PIC_QED_METHOD1 && Q->method != PIC_QED_METHOD2)
        return fail(s, PIC_ERR_ARG, "pic_set_qed: method must be PIC_QED_METHOD1 or PIC_QED_METHOD2");
    if (Q->method == PIC_QED_METHOD2 && Q->mode == PIC_QED_SURROGATE)
        return fail(s, PIC_ERR_ARG, "pic_set_qed: the surrogate replaces Method I's rate and inverse CDF");
    auto kind_ok = [&](int i, int kind) { return i == -1 || (i >= 0 && i < s->nsp && s->sp[i].kind == kind); };
    if (!kind_ok(Q->photon_sp, PIC_KIND_PHOTON) || !kind_ok(Q->electron_sp, PIC_KIND_MASSIVE) ||
        !kind_ok(Q->positron_sp, PIC_KIND_MASSIVE) || !(Q->lambda_r_m > 0.0) || Q->photon_emin < 0.0)
        return fail(s, PIC_ERR_ARG, "pic_set_qed: bad species index, kind or wavelength");
    if (Q->electron_sp >= 0 && (s->sp[Q->electron_sp].q >= 0.0 || !s->sp[Q->electron_sp].has_qed_arrays()))
        return fail(s, PIC_ERR_ARG, "pic_set_qed: the pair-electron species must be a negative QED species");
    if (Q->positron_sp >= 0 && (s->sp[Q->positron_sp].q <= 0.0 || !s->sp[Q->positron_sp].has_qed_arrays()))
        return fail(s, PIC_ERR_ARG, "pic_set_qed: the pair-positron species must be a positive QED species");
    if (!s->qed_tables) {
        int rc = dalloc(s, &s->qed_tables, qed_table_bytes());
        if (rc) return rc;
        if (qed_upload_tables(s->qed_tables, &s->T, s->st)) return fail(s, PIC_ERR_CUDA, "pic_set_qed: table upload");
    }
    if (Q->mode == PIC_QED_SURROGATE && Q->photon_sp >= 0 && s->precision == PIC_PREC_FP32_CELLOFF) {
        // the queue of the thinned pair sampler's candidates: one slot per
        // photon (each queues at most once per step), 32-bit photon indices
        const long long cap = s->sp[Q->photon_sp].cap;
        if (cap >= (1ll << 31)) return fail(s, PIC_ERR_ARG, "pic_set_qed: surrogate photons need a capacity below 2^31");
        if (s->cand_q && s->cand_cap < cap) {  // (the QED photon species changed to a larger one)
            s->allocs.erase(std::find(s->allocs.begin(), s->allocs.end(), (void *)s->cand_q));
            raw_free(s, s->cand_q);
            s->cand_q = nullptr;
        }
        if (!s->cand_q) {
            if (int rc = dalloc(s, (void **)&s->cand_q, (size_t)(cap + 32) * sizeof(float4))) return rc;
            s->cand_cap = cap;
        }
        if (!s->cand_n)
            if (int rc = dalloc(s, (void **)&s->cand_n, sizeof(uint32_t))) return rc;
    }
    // E_s = m c^2 / (hbar omega_r) = m c^2 lambda_r / (h c)
    const double mc2_eV = 510998.95, hc_eVm = 1.239841984e-6;
    s->Es = mc2_eV * Q->lambda_r_m / hc_eVm;
    s->qed = *Q;
    s->qed_on = Q->mode != PIC_QED_OFF;
    return PIC_OK;
}

int pic_qed_eval(pic_sim *s, int process, int64_t n, const double *chi, const double *r, double *out)
{
    if (!s) return PIC_ERR_ARG;
    if ((process != PIC_QED_EMISSION && process != PIC_QED_PAIR) || n < 0 || !chi || !out)
        return fail(s, PIC_ERR_ARG, "pic_qed_eval: bad arguments");
    if (!s->qed_tables) return fail(s, PIC_ERR_STATE, "pic_qed_eval: call pic_set_qed first");
    if (n == 0) return PIC_OK;
    double *d = nullptr;
    if (int rc_ = talloc(s, (void **)&d, (size_t)n * 3 * sizeof(double))) return rc_;
    cudaError_t e = cudaMemcpyAsync(d, chi, n * 8, cudaMemcpyHostToDevice, s->st);
    if (e == cudaSuccess && r) e = cudaMemcpyAsync(d + n, r, n * 8, cudaMemcpyHostToDevice, s->st);
    if (e == cudaSuccess) {
        const MlpNet &net = s->net[process];
        if (s->qed.mode == PIC_QED_SURROGATE && net.ready && s->precision == PIC_PREC_FP32_CELLOFF)
            launch_qed_eval_surr(net.img, net.nrm, s->T, false, process, n, d, r ? d + n : nullptr, d + 2 * n, s->st);
        else
            launch_qed_eval(s->T, s->precision == PIC_PREC_FP64_PLAIN, process, n, d, r ? d + n : nullptr, d + 2 * n,
                            s->st);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d + 2 * n, n * 8, cudaMemcpyDeviceToHost, s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    tfree(s, d);
    if (e != cudaSuccess) return fail(s, PIC_ERR_CUDA, "pic_qed_eval: %s", cudaGetErrorString(e));
    return PIC_OK;
}

int pic_get_qed_state(pic_sim *s, int sp, int64_t cap, uint64_t *id, double *tau)
{
    if (!s) return PIC_ERR_ARG;
    if (sp < 0 || sp >= s->nsp || !s->sp[sp].has_qed_arrays())
        return fail(s, PIC_ERR_ARG, "pic_get_qed_state: not a QED species");
    long long cnt = 0;
    int rc = read_count(s, sp, &cnt);
    if (rc) return rc;
    if (cnt > cap) return fail(s, PIC_ERR_CAPACITY, "pic_get_qed_state: capacity");
    SpeciesState &p = s->sp[sp];
    if (cnt && id) CK(cudaMemcpyAsync(id, p.id[p.cur], cnt * 8, cudaMemcpyDeviceToHost, s->st));
    if (cnt && tau) CK(cudaMemcpyAsync(tau, p.tau[p.cur], cnt * 8, cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    return PIC_OK;
}

int pic_set_laser(pic_sim *s, const pic_laser *L)
{
    if (!s || !L) return PIC_ERR_ARG;
    if (s->g.bc[0] != ABSORB) return fail(s, PIC_ERR_ARG, "pic_set_laser: the x-min face must be absorbing");
    if (!(L->fwhm > 0.0) || (s->g.dim > 1 && !(L->waist > 0.0)) || (L->pol != 0 && L->pol != 1))
        return fail(s, PIC_ERR_ARG, "pic_set_laser: bad laser parameters");
    // transverse profile of the paraxial Gaussian beam at the x-min face
    // (focus at x_focus; 2D: sqrt(w0/w) amplitude and half the Gouy phase)
    const Grid &g = s->g;
    const int nty = g.dim >= 2 ? g.n[1] : 1, ntz = g.dim >= 3 ? g.n[2] : 1;
    const size_t nt = (size_t)nty * ntz;
    double amp = 1.0, wxi = 1.0, rinv = 0.0, gouy = 0.0;
    if (g.dim >= 2) {
        const double xr = 0.5 * L->waist * L->waist, xi = -L->x_focus;
        wxi = L->waist * std::sqrt(1.0 + (xi / xr) * (xi / xr));
        rinv = xi / (xi * xi + xr * xr);
        gouy = std::atan(xi / xr);
        amp = g.dim == 3 ? L->waist / wxi : std::sqrt(L->waist / wxi);
        if (g.dim == 2) gouy *= 0.5;
    }
    std::vector<double> prof(4 * nt);  // A_Bz, PHI_Bz, A_By, PHI_By
    for (int c = 0; c < 2; c++) {
        const double sy = c == 0 ? 0.5 : 0.0, sz = c == 0 ? 0.0 : 0.5;  // B_z at (j+1/2, k), B_y at (j, k+1/2)
        for (int k = 0; k < ntz; k++)
            for (int j = 0; j < nty; j++) {
                double r2 = 0.0;
                if (g.dim >= 2) r2 += std::pow((j + sy) * g.dx[1] - L->yc, 2);
                if (g.dim >= 3) r2 += std::pow((k + sz) * g.dx[2] - L->zc, 2);
                const double trans = g.dim >= 2 ? std::exp(-r2 / (wxi * wxi)) : 1.0;
                prof[(2 * c) * nt + (size_t)k * nty + j] = L->a0 * amp * trans;
                prof[(2 * c + 1) * nt + (size_t)k * nty + j] = -0.5 * r2 * rinv + gouy;
            }
    }
    if (!s->laser_prof) {
        int rc = dalloc(s, &s->laser_prof, 4 * nt * rsize(s));
        if (rc) return rc;
    }
    if (s->precision == PIC_PREC_FP64_PLAIN) {
        CK(cudaMemcpyAsync(s->laser_prof, prof.data(), 4 * nt * 8, cudaMemcpyHostToDevice, s->st));
    } else {
        std::vector<float> pf(prof.begin(), prof.end());
        CK(cudaMemcpyAsync(s->laser_prof, pf.data(), 4 * nt * 4, cudaMemcpyHostToDevice, s->st));
    }
    CK(cudaStreamSynchronize(s->st));
    const size_t rb = rsize(s);
    s->laser.on = 1;
    s->laser.pol = L->pol;
    s->laser.nty = nty;
    s->laser.ntz = ntz;
    for (int c = 0; c < 2; c++) {
        s->laser.A[c] = (const char *)s->laser_prof + (2 * c) * nt * rb;
        s->laser.PHI[c] = (const char *)s->laser_prof + (2 * c + 1) * nt * rb;
    }
    s->lp = *L;
    return PIC_OK;
}

int pic_set_field(pic_sim *s, int comp, const double *host_in)
{
    if (!s) return PIC_ERR_ARG;
    if (comp < PIC_EX || comp > PIC_JZ || !host_in) return fail(s, PIC_ERR_ARG, "pic_set_field: bad component");
    if (s->precision == PIC_PREC_FP64_PLAIN)
        return copy_comp_in<double>(s, (double *)s->F + comp * s->g.vol, host_in);
    return copy_comp_in<float>(s, (float *)s->F + comp * s->g.vol, host_in);
}

int pic_step(pic_sim *s, int64_t nsteps)
{
    if (!s) return PIC_ERR_ARG;
    if (nsteps < 0) return fail(s, PIC_ERR_ARG, "pic_step: negative step count");
    int rc = s->precision == PIC_PREC_FP64_PLAIN ? step_loop<double>(s, nsteps) : step_loop<float>(s, nsteps);
    if (rc) return rc;
    return check_flags(s);
}

int pic_profile(pic_sim *s, int enable)
{
    if (!s) return PIC_ERR_ARG;
    CK(cudaStreamSynchronize(s->st));
    for (auto &m : s->marks) {
        cudaEventDestroy(m.a);
        cudaEventDestroy(m.b);
    }
    s->marks.clear();
    for (int p = 0; p < PIC_NPHASE; p++) s->prof_launch[p] = 0;
    s->prof_push = 0;
    if (enable) {  // the per-species times gathered so far stay readable after disabling
        for (int i = 0; i < PIC_MAX_SPECIES; i++) {
            s->prof_sp_ms[i] = 0.0;
            s->prof_sp_n[i] = 0;
        }
    }
    s->prof = enable != 0;
    return PIC_OK;
}

int pic_profile_read(pic_sim *s, double *ms, int64_t *launches, int64_t *push_launches)
{
    if (!s) return PIC_ERR_ARG;
    CK(cudaStreamSynchronize(s->st));
    double acc[PIC_NPHASE] = {0, 0, 0, 0};
    for (auto &m : s->marks) {
        float t = 0.f;
        cudaEventElapsedTime(&t, m.a, m.b);
        if (m.phase >= PIC_NPHASE) {  // one species' push
            s->prof_sp_ms[m.phase - PIC_NPHASE] += t;
            s->prof_sp_n[m.phase - PIC_NPHASE]++;
        } else {
            acc[m.phase] += t;
        }
        cudaEventDestroy(m.a);
        cudaEventDestroy(m.b);
    }
    s->marks.clear();
    for (int p = 0; p < PIC_NPHASE; p++) {
        if (ms) ms[p] = acc[p];
        if (launches) launches[p] = s->prof_launch[p];
        s->prof_launch[p] = 0;
    }
    if (push_launches) *push_launches = s->prof_push;
    s->prof_push = 0;
    return PIC_OK;
}

int pic_profile_read_species(pic_sim *s, double *ms, int64_t *pushes)
{
    if (!s) return PIC_ERR_ARG;
    for (int i = 0; i < s->nsp; i++) {
        if (ms) ms[i] = s->prof_sp_ms[i];
        if (pushes) pushes[i] = s->prof_sp_n[i];
        s->prof_sp_ms[i] = 0.0;
        s->prof_sp_n[i] = 0;
    }
    return PIC_OK;
}

int pic_fields(pic_sim *s, int comp, double *host_out)
{
    if (!s) return PIC_ERR_ARG;
    if (comp < PIC_EX || comp > PIC_RHO || !host_out) return fail(s, PIC_ERR_ARG, "pic_fields: bad component");
    if (comp == PIC_RHO) {
        int rc = compute_rho(s);
        if (rc) return rc;
        return copy_comp_out<double>(s, s->rho, host_out);
    }
    if (s->precision == PIC_PREC_FP64_PLAIN)
        return copy_comp_out<double>(s, (const double *)s->F + comp * s->g.vol, host_out);
    return copy_comp_out<float>(s, (const float *)s->F + comp * s->g.vol, host_out);
}

int pic_field_device(pic_sim *s, int comp, pic_field_view *v)
{
    if (!s) return PIC_ERR_ARG;
    if (comp < PIC_EX || comp > PIC_JZ || !v) return fail(s, PIC_ERR_ARG, "pic_field_device: bad component");
    const Grid &g = s->g;
    const size_t R = rsize(s);
    v->data = (char *)s->F + (size_t)comp * g.vol * R;
    v->elem_bytes = (int)R;
    v->origin = g.origin;
    v->stride[0] = 1;
    v->stride[1] = g.sy;
    v->stride[2] = g.sz;
    for (int d = 0; d < 3; d++) {
        v->lo[d] = -g.G[d];
        v->hi[d] = g.n[d] + g.G[d] - 1;
    }
    return PIC_OK;
}

int64_t pic_particle_count(pic_sim *s, int sp)
{
    if (!s || sp < 0 || sp >= s->nsp) return -1;
    long long n = 0;
    if (read_count(s, sp, &n)) return -1;
    return n;
}

int pic_get_particles(pic_sim *s, int sp, int64_t cap, int64_t *n, double *x, double *y, double *z, double *ux,
                      double *uy, double *uz, uint8_t *alive)
{
    if (!s) return PIC_ERR_ARG;
    if (sp < 0 || sp >= s->nsp || !n) return fail(s, PIC_ERR_ARG, "pic_get_particles: bad arguments");
    long long cnt = 0;
    int rc = read_count(s, sp, &cnt);
    if (rc) return rc;
    *n = cnt;
    if (cnt > cap) return fail(s, PIC_ERR_CAPACITY, "pic_get_particles: %lld particles, room for %lld", cnt, (long long)cap);
    if (cnt == 0) return PIC_OK;
    SpeciesState &p = s->sp[sp];
    double *dtmp = nullptr;
    uint8_t *dal = nullptr;
    if (int rc_ = talloc(s, (void **)&dtmp, (size_t)cnt * 6 * sizeof(double))) return rc_;
    if (int rc_ = talloc(s, (void **)&dal, (size_t)cnt)) {
        tfree(s, dtmp);
        return rc_;
    }
    cudaError_t e = cudaSuccess;
    double *dx_[3] = {dtmp, dtmp + cnt, dtmp + 2 * cnt};
    double *du_[3] = {dtmp + 3 * cnt, dtmp + 4 * cnt, dtmp + 5 * cnt};
    if (s->precision == PIC_PREC_FP64_PLAIN) launch_unload_f64(view64(s, sp, p.cur), s->g, dx_, du_, dal, s->st);
    else launch_unload_f32(view32(s, sp, p.cur), s->g, dx_, du_, dal, s->st);
    e = cudaGetLastError();
    double *hs[6] = {x, y, z, ux, uy, uz};
    double *ds[6] = {dx_[0], dx_[1], dx_[2], du_[0], du_[1], du_[2]};
    for (int q = 0; q < 6 && e == cudaSuccess; q++)
        if (hs[q]) e = cudaMemcpyAsync(hs[q], ds[q], cnt * sizeof(double), cudaMemcpyDeviceToHost, s->st);
    if (e == cudaSuccess && alive) e = cudaMemcpyAsync(alive, dal, cnt, cudaMemcpyDeviceToHost, s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    tfree(s, dtmp);
    tfree(s, dal);
    if (e != cudaSuccess) return fail(s, PIC_ERR_CUDA, "pic_get_particles: %s", cudaGetErrorString(e));
    return PIC_OK;
}

int pic_get_cells(pic_sim *s, int sp, int64_t cap, uint32_t *cells, int *bits)
{
    if (!s) return PIC_ERR_ARG;
    if (sp < 0 || sp >= s->nsp || !cells) return fail(s, PIC_ERR_ARG, "pic_get_cells: bad arguments");
    long long cnt = 0;
    int rc = read_count(s, sp, &cnt);
    if (rc) return rc;
    if (cnt > cap) return fail(s, PIC_ERR_CAPACITY, "pic_get_cells: capacity");
    if (bits)
        for (int d = 0; d < 3; d++) bits[d] = s->g.bits[d];
    if (cnt == 0) return PIC_OK;
    SpeciesState &p = s->sp[sp];
    CK(cudaMemcpyAsync(cells, p.cell[p.cur], cnt * 4, cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    return PIC_OK;
}

int pic_gather(pic_sim *s, int sp, int64_t cap, double *out6)
{
    if (!s) return PIC_ERR_ARG;
    if (sp < 0 || sp >= s->nsp || !out6) return fail(s, PIC_ERR_ARG, "pic_gather: bad arguments");
    long long cnt = 0;
    int rc = read_count(s, sp, &cnt);
    if (rc) return rc;
    if (cnt > cap) return fail(s, PIC_ERR_CAPACITY, "pic_gather: capacity");
    if (cnt == 0) return PIC_OK;
    SpeciesState &p = s->sp[sp];
    double *d = nullptr;
    if (int rc_ = talloc(s, (void **)&d, (size_t)cnt * 6 * sizeof(double))) return rc_;
    if (s->precision == PIC_PREC_FP64_PLAIN)
        launch_gather_f64(view64(s, sp, p.cur), (const double *)s->F, s->g, d, s->st);
    else
        launch_gather_f32(view32(s, sp, p.cur), (const float *)s->F, s->g, d, s->st);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(out6, d, cnt * 6 * sizeof(double), cudaMemcpyDeviceToHost, s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    tfree(s, d);
    if (e != cudaSuccess) return fail(s, PIC_ERR_CUDA, "pic_gather: %s", cudaGetErrorString(e));
    return PIC_OK;
}

int pic_diagnostics(pic_sim *s, pic_diag *d)
{
    if (!s || !d) return PIC_ERR_ARG;
    const Grid &g = s->g;
    std::memset(d, 0, sizeof *d);
    double dV = 1.0, vol = 1.0;
    for (int a = 0; a < g.dim; a++) {
        dV *= g.dx[a];
        vol *= g.dx[a] * g.n[a];
    }
    double h[16] = {0};
    // field energy
    if (s->precision == PIC_PREC_FP64_PLAIN)
        diag_field_energy<double>((const double *)s->F, g, s->diag_scratch, s->diag_out, s->st);
    else
        diag_field_energy<float>((const float *)s->F, g, s->diag_scratch, s->diag_out, s->st);
    CK(cudaMemcpyAsync(h, s->diag_out, 2 * sizeof(double), cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    d->U_E = 0.5 * h[0] * dV;
    d->U_B = 0.5 * h[1] * dV;
    double charge = 0.0;
    for (int i = 0; i < s->nsp; i++) {
        SpeciesState &p = s->sp[i];
        if (s->precision == PIC_PREC_FP64_PLAIN)
            diag_kinetic_f64(view64(s, i, p.cur), p.kind == PIC_KIND_PHOTON, s->diag_scratch, s->diag_out, s->st);
        else
            diag_kinetic_f32(view32(s, i, p.cur), p.kind == PIC_KIND_PHOTON, s->diag_scratch, s->diag_out, s->st);
        CK(cudaMemcpyAsync(h, s->diag_out, 2 * sizeof(double), cudaMemcpyDeviceToHost, s->st));
        CK(cudaStreamSynchronize(s->st));
        d->U_kin[i] = h[0] * p.w * (p.kind == PIC_KIND_PHOTON ? 1.0 : p.m) * dV;
        d->n_alive[i] = (int64_t)llround(h[1]);
        charge += p.q * p.w * h[1] * dV;
    }
    d->charge = charge + s->rho_bg * vol;
    int rc = compute_rho(s);
    if (rc) return rc;
    if (s->precision == PIC_PREC_FP64_PLAIN)
        diag_gauss<double>((const double *)s->F, s->rho, g, s->rho_bg, s->diag_scratch, s->diag_out, s->st);
    else
        diag_gauss<float>((const float *)s->F, s->rho, g, s->rho_bg, s->diag_scratch, s->diag_out, s->st);
    CK(cudaMemcpyAsync(h, s->diag_out, sizeof(double), cudaMemcpyDeviceToHost, s->st));
    CK(cudaMemcpyAsync(h + 1, s->d_eabs, sizeof(double), cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    CK(cudaGetLastError());
    d->gauss_max = h[0];
    d->E_absorbed = h[1];
    CK(cudaMemcpy(&d->E_photon_lost, s->d_elost, sizeof(double), cudaMemcpyDeviceToHost));
    d->step = s->step;
    d->t = (double)s->step * g.dt;
    bool finite = std::isfinite(d->U_E) && std::isfinite(d->U_B) && std::isfinite(d->gauss_max);
    for (int i = 0; i < s->nsp; i++) finite = finite && std::isfinite(d->U_kin[i]);
    if (!finite) return fail(s, PIC_ERR_NONFINITE, "pic_diagnostics: non-finite value");
    return PIC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------
// surrogate network: device state and training orchestration
// ---------------------------------------------------------------------
namespace {

static_assert(PIC_MLP_NPARAMS == kMlpNParams, "parameter count of the C ABI");

int mlp_net_alloc(pic_sim *s, MlpNet &net)
{
    if (net.img) return PIC_OK;
    const size_t pb = (size_t)kMlpNParams * sizeof(float);
    void *img = nullptr, *buf = nullptr;
    int rc = dalloc(s, &img, sizeof(MlpImage));
    if (!rc) rc = dalloc(s, &buf, 4 * pb);
    if (rc) return rc;
    CK(cudaMemsetAsync(img, 0, sizeof(MlpImage), s->st));
    CK(cudaMemsetAsync(buf, 0, 4 * pb, s->st));
    net.img = (MlpImage *)img;
    net.P = (float *)buf;
    net.M = net.P + kMlpNParams;
    net.V = net.M + kMlpNParams;
    net.G = net.V + kMlpNParams;
    return PIC_OK;
}

int mlp_scratch(pic_sim *s, long long B)
{
    MlpScratch &S = s->ms;
    if (!S.it) {
        void *small = nullptr;
        int rc = dalloc(s, &small, 64 + kMlpValAcc * sizeof(double));
        if (rc) return rc;
        S.loss = (float *)small;                  // 2 floats
        S.it = (int *)((char *)small + 16);
        S.acc = (double *)((char *)small + 64);   // kMlpValAcc doubles
    }
    if (B <= S.B) return PIC_OK;
    void *buf = nullptr;
    const size_t per_row = (size_t)(3 * 2 + 6 * kMlpH) * sizeof(float);
    int rc = dalloc(s, &buf, per_row * (size_t)B + mlp_partial_floats(B) * sizeof(float));
    if (rc) return rc;
    float *f = (float *)buf;
    S.X = f;
    S.T = f + 2 * B;
    S.Y = f + 4 * B;
    for (int l = 0; l < 3; l++) {
        S.Z.z[l] = f + 6 * B + (size_t)l * kMlpH * B;
        S.D.z[l] = f + 6 * B + (size_t)(3 + l) * kMlpH * B;
    }
    S.partials = f + 6 * B + (size_t)6 * kMlpH * B;
    S.B = B;
    return PIC_OK;
}

// ln G (+ 8/(3 chi) for pairs) from the FP64 tables at two values of chi
int mlp_table_lnG(pic_sim *s, int p, const double chi[2], double out[2])
{
    double *d = nullptr;
    if (int rc_ = talloc(s, (void **)&d, 4 * sizeof(double))) return rc_;
    cudaError_t e = cudaMemcpyAsync(d, chi, 2 * sizeof(double), cudaMemcpyHostToDevice, s->st);
    if (e == cudaSuccess) {
        launch_qed_eval(s->T, true, p, 2, d, nullptr, d + 2, s->st);
        e = cudaGetLastError();
    }
    double G[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(G, d + 2, 2 * sizeof(double), cudaMemcpyDeviceToHost, s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    tfree(s, d);
    if (e != cudaSuccess) return fail(s, PIC_ERR_CUDA, "mlp: table evaluation: %s", cudaGetErrorString(e));
    for (int i = 0; i < 2; i++) out[i] = std::log(G[i]) + (p == QED_PAIR ? 8.0 / (3.0 * chi[i]) : 0.0);
    return PIC_OK;
}

void mlp_norm_set(MlpNorm &n, double chi_min, double chi_max, double mu, double sd)
{
    n.lnchi_lo = std::log(chi_min);
    n.lnchi_hi = std::log(chi_max);
    n.x0a = (float)(2.0 / (n.lnchi_hi - n.lnchi_lo));
    n.x0b = (float)(-(n.lnchi_hi + n.lnchi_lo) / (n.lnchi_hi - n.lnchi_lo));
    n.mu = (float)mu;
    n.sd = (float)sd;
}

// initial parameters: W ~ N(0, 1/fan_in), biases 0
void mlp_init_params(std::vector<float> &P, uint64_t seed)
{
    std::mt19937_64 rng(seed ^ 0x6d6c7020696e6974ull);
    std::normal_distribution<double> nd(0.0, 1.0);
    P.assign(kMlpNParams, 0.f);
    auto fill = [&](int off, int n_out, int n_in) {
        for (int i = 0; i < n_out * n_in; i++) P[off + i] = (float)(nd(rng) / std::sqrt((double)n_in));
    };
    fill(kOffW0, kMlpH, 2);
    fill(kOffW1, kMlpH, kMlpH);
    fill(kOffW2, kMlpH, kMlpH);
    fill(kOffW3, 2, kMlpH);
}

int mlp_check(pic_sim *s, int process)
{
    if (process != PIC_QED_EMISSION && process != PIC_QED_PAIR) return fail(s, PIC_ERR_ARG, "mlp: bad process");
    if (!s->qed_tables) return fail(s, PIC_ERR_STATE, "mlp: call pic_set_qed first (the tables)");
    return PIC_OK;
}

int mlp_validate(pic_sim *s, int p, pic_mlp_report *rep)
{
    MlpNet &net = s->net[p];
    int rc = mlp_scratch(s, 0);
    if (rc) return rc;
    CK(cudaMemsetAsync(s->ms.acc, 0, kMlpValAcc * sizeof(double), s->st));
    launch_mlp_validate(net.img, net.nrm, s->T, p, kMlpValRows, kMlpValRows, s->ms.acc, s->st);
    CK(cudaGetLastError());
    double acc[kMlpValAcc];
    CK(cudaMemcpyAsync(acc, s->ms.acc, sizeof acc, cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    rep->max_err_lnG = acc[0];
    rep->max_err_s = acc[1];
    rep->rms_err_s = std::sqrt(acc[2] / ((double)kMlpValRows * kMlpValRows));
    rep->max_err_mean = 0.0;
    for (int r = 0; r < kMlpValRows; r++) {
        const double fn = acc[4 + 2 * r], ft = acc[5 + 2 * r];
        if (ft > 0.0) rep->max_err_mean = std::max(rep->max_err_mean, std::fabs(fn / ft - 1.0));
    }
    rep->table_bytes = (int64_t)(qed_table_bytes() / 2);
    rep->net_bytes = kMlpStageBytes;
    return PIC_OK;
}

}  // namespace

extern "C" {

int pic_mlp_train(pic_sim *s, int p, const pic_mlp_train_opts *o, pic_mlp_report *rep)
{
    if (!s || !o) return PIC_ERR_ARG;
    int rc = mlp_check(s, p);
    if (rc) return rc;
    const long long iters = o->iterations > 0 ? o->iterations : 40000;
    const long long B = o->batch > 0 ? o->batch : 16384;
    // default ranges: emission from chi = 1e-3 (below, the tables' classical
    // limit); pairs from chi = 0.1, where G_pair = 3e-13 makes W dt ~ 1e-13 per
    // step -- below it the tables give the rate and no event is expected
    const double chi_min = o->chi_min > 0 ? o->chi_min : (p == QED_PAIR ? 1e-1 : 1e-3);
    const double chi_max = o->chi_max > 0 ? o->chi_max : 1e2;
    if (B % 128 || B > (1ll << 22) || o->iterations < 0 || !(chi_max > chi_min) || chi_min < 1e-4 || chi_max > 1e3 ||
        o->lr < 0 || o->lr_final < 0 || o->rate_weight < 0)
        return fail(s, PIC_ERR_ARG, "pic_mlp_train: bad options (batch a multiple of 128, chi range in [1e-4, 1e3])");
    MlpNet &net = s->net[p];
    const bool fresh = !net.img || !o->keep;
    if ((rc = mlp_net_alloc(s, net)) || (rc = mlp_scratch(s, B))) return rc;
    double lg[2];
    const double ends[2] = {chi_min, chi_max};
    if ((rc = mlp_table_lnG(s, p, ends, lg))) return rc;
    mlp_norm_set(net.nrm, chi_min, chi_max, 0.5 * (lg[0] + lg[1]), std::max(0.5 * std::fabs(lg[1] - lg[0]), 1.0));
    if (fresh) {
        std::vector<float> P0;
        mlp_init_params(P0, o->seed + (uint64_t)p);
        CK(cudaMemcpyAsync(net.P, P0.data(), P0.size() * sizeof(float), cudaMemcpyHostToDevice, s->st));
        CK(cudaMemsetAsync(net.M, 0, 3 * (size_t)kMlpNParams * sizeof(float), s->st));  // M, V, G
    }
    launch_mlp_image(net.P, net.img, s->st);
    CK(cudaMemsetAsync(s->ms.it, 0, sizeof(int), s->st));
    CK(cudaMemsetAsync(s->ms.loss, 0, 2 * sizeof(float), s->st));
    CK(cudaStreamSynchronize(s->st));
    MlpAdam a{iters, o->lr > 0 ? o->lr : 1e-2, o->lr_final > 0 ? o->lr_final : 1e-4, 0.9f, 0.999f, 1e-8f};
    const float w_rate = (float)(o->rate_weight > 0 ? o->rate_weight : 4.0);
    const uint32_t key[2] = {(uint32_t)o->seed, (uint32_t)(o->seed >> 32)};
    // one iteration captured as a graph on a private stream, replayed
    cudaStream_t ts = nullptr;
    cudaGraph_t gr = nullptr;
    cudaGraphExec_t ge = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(ts, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        mlp_train_iteration(net, s->ms, s->T, p, key, a, w_rate, ts);
        e = cudaStreamEndCapture(ts, &gr);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, gr, 0);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0, ts);
    for (long long i = 0; i < iters && e == cudaSuccess; i++) e = cudaGraphLaunch(ge, ts);
    note_launch(7 * (iters - 1));  // the captured iteration counted its seven launches once
    if (e == cudaSuccess) e = cudaEventRecord(e1, ts);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ts);
    float ms = 0.f, loss[2] = {0.f, 0.f};
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) e = cudaMemcpy(loss, s->ms.loss, sizeof loss, cudaMemcpyDeviceToHost);
    if (ge) cudaGraphExecDestroy(ge);
    if (gr) cudaGraphDestroy(gr);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (ts) cudaStreamDestroy(ts);
    if (e != cudaSuccess) return fail(s, PIC_ERR_CUDA, "pic_mlp_train: %s", cudaGetErrorString(e));
    net.ready = true;
    pic_mlp_report r{};
    if ((rc = mlp_validate(s, p, &r))) return rc;
    r.loss = loss[1];
    r.ms = ms;
    r.iterations = iters;
    if (rep) *rep = r;
    return PIC_OK;
}

int pic_mlp_validate(pic_sim *s, int p, pic_mlp_report *rep)
{
    if (!s || !rep) return PIC_ERR_ARG;
    int rc = mlp_check(s, p);
    if (rc) return rc;
    if (!s->net[p].ready) return fail(s, PIC_ERR_STATE, "pic_mlp_validate: no network");
    *rep = pic_mlp_report{};
    return mlp_validate(s, p, rep);
}

int pic_mlp_get(pic_sim *s, int p, float *params, pic_mlp_info *info)
{
    if (!s) return PIC_ERR_ARG;
    if (p != PIC_QED_EMISSION && p != PIC_QED_PAIR) return fail(s, PIC_ERR_ARG, "pic_mlp_get: bad process");
    const MlpNet &net = s->net[p];
    if (!net.ready) return fail(s, PIC_ERR_STATE, "pic_mlp_get: no network");
    if (params) {
        CK(cudaMemcpyAsync(params, net.P, (size_t)kMlpNParams * sizeof(float), cudaMemcpyDeviceToHost, s->st));
        CK(cudaStreamSynchronize(s->st));
    }
    if (info) {
        info->chi_min = std::exp(net.nrm.lnchi_lo);
        info->chi_max = std::exp(net.nrm.lnchi_hi);
        info->mu = net.nrm.mu;
        info->sd = net.nrm.sd;
    }
    return PIC_OK;
}

int pic_mlp_set(pic_sim *s, int p, const float *params, const pic_mlp_info *info)
{
    if (!s || !params || !info) return PIC_ERR_ARG;
    if (p != PIC_QED_EMISSION && p != PIC_QED_PAIR) return fail(s, PIC_ERR_ARG, "pic_mlp_set: bad process");
    if (!(info->chi_max > info->chi_min) || !(info->chi_min > 0.0) || !(info->sd > 0.0))
        return fail(s, PIC_ERR_ARG, "pic_mlp_set: bad range or normalisation");
    MlpNet &net = s->net[p];
    int rc = mlp_net_alloc(s, net);
    if (rc) return rc;
    mlp_norm_set(net.nrm, info->chi_min, info->chi_max, info->mu, info->sd);
    CK(cudaMemcpyAsync(net.P, params, (size_t)kMlpNParams * sizeof(float), cudaMemcpyHostToDevice, s->st));
    CK(cudaMemsetAsync(net.M, 0, 3 * (size_t)kMlpNParams * sizeof(float), s->st));
    launch_mlp_image(net.P, net.img, s->st);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s->st));
    net.ready = true;
    return PIC_OK;
}

int pic_mlp_eval(pic_sim *s, int p, int64_t n, const float *x, float *y)
{
    if (!s) return PIC_ERR_ARG;
    if ((p != PIC_QED_EMISSION && p != PIC_QED_PAIR) || n < 0 || (n && (!x || !y)))
        return fail(s, PIC_ERR_ARG, "pic_mlp_eval: bad arguments");
    const MlpNet &net = s->net[p];
    if (!net.ready) return fail(s, PIC_ERR_STATE, "pic_mlp_eval: no network");
    if (n == 0) return PIC_OK;
    float *d = nullptr;
    if (int rc_ = talloc(s, (void **)&d, (size_t)n * 4 * sizeof(float))) return rc_;
    cudaError_t e = cudaMemcpyAsync(d, x, (size_t)n * 2 * sizeof(float), cudaMemcpyHostToDevice, s->st);
    if (e == cudaSuccess) {
        launch_mlp_eval(net.img, n, d, d + 2 * n, s->st);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(y, d + 2 * n, (size_t)n * 2 * sizeof(float), cudaMemcpyDeviceToHost, s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    tfree(s, d);
    if (e != cudaSuccess) return fail(s, PIC_ERR_CUDA, "pic_mlp_eval: %s", cudaGetErrorString(e));
    return PIC_OK;
}

int pic_mlp_eval_tc(pic_sim *s, int p, int64_t n, const float *x, float *y)
{
    if (!s) return PIC_ERR_ARG;
    if ((p != PIC_QED_EMISSION && p != PIC_QED_PAIR) || n < 0 || (n && (!x || !y)))
        return fail(s, PIC_ERR_ARG, "pic_mlp_eval_tc: bad arguments");
    const MlpNet &net = s->net[p];
    if (!net.ready) return fail(s, PIC_ERR_STATE, "pic_mlp_eval_tc: no network");
    if (n == 0) return PIC_OK;
    float *d = nullptr;
    if (int rc_ = talloc(s, (void **)&d, (size_t)n * 4 * sizeof(float))) return rc_;
    cudaError_t e = cudaMemcpyAsync(d, x, (size_t)n * 2 * sizeof(float), cudaMemcpyHostToDevice, s->st);
    if (e == cudaSuccess) {
        launch_mlp_eval_tc(net.img, n, d, d + 2 * n, s->d_err, s->st);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(y, d + 2 * n, (size_t)n * 2 * sizeof(float), cudaMemcpyDeviceToHost, s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    tfree(s, d);
    if (e != cudaSuccess) return fail(s, PIC_ERR_CUDA, "pic_mlp_eval_tc: %s", cudaGetErrorString(e));
    return check_flags(s);
}

int pic_mlp_grad(pic_sim *s, int p, int64_t n, const float *x, const float *t, float *grad, double *loss)
{
    if (!s) return PIC_ERR_ARG;
    if ((p != PIC_QED_EMISSION && p != PIC_QED_PAIR) || n <= 0 || n % 32 || n > (1 << 20) || !x || !t || !grad)
        return fail(s, PIC_ERR_ARG, "pic_mlp_grad: bad arguments (n a positive multiple of 32)");
    MlpNet &net = s->net[p];
    if (!net.ready) return fail(s, PIC_ERR_STATE, "pic_mlp_grad: no network");
    int rc = mlp_scratch(s, n);
    if (rc) return rc;
    MlpScratch &S = s->ms;
    CK(cudaMemcpyAsync(S.X, x, (size_t)n * 2 * sizeof(float), cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(S.T, t, (size_t)n * 2 * sizeof(float), cudaMemcpyHostToDevice, s->st));
    CK(cudaMemsetAsync(net.G, 0, (size_t)kMlpNParams * sizeof(float), s->st));
    CK(cudaMemsetAsync(S.loss, 0, sizeof(float), s->st));
    launch_mlp_forward(net.img, n, S.X, S.Z, S.Y, s->st);
    launch_mlp_backward(net.img, n, S.X, S.T, S.Y, S.Z, S.D, S.partials, net.G, 1.0f, S.loss, s->st);
    CK(cudaGetLastError());
    float l = 0.f;
    CK(cudaMemcpyAsync(grad, net.G, (size_t)kMlpNParams * sizeof(float), cudaMemcpyDeviceToHost, s->st));
    CK(cudaMemcpyAsync(&l, S.loss, sizeof(float), cudaMemcpyDeviceToHost, s->st));
    CK(cudaMemsetAsync(net.G, 0, (size_t)kMlpNParams * sizeof(float), s->st));
    CK(cudaStreamSynchronize(s->st));
    if (loss) *loss = l;
    return PIC_OK;
}

}  // extern "C"
