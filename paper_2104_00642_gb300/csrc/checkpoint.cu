// checkpoint.cu -- pic_save / pic_restore: the whole state of a simulation
// in one host-endian binary file.
//
// Layout: a header (magic, version), the configuration signature (grid, dt,
// precision, species, sort interval, tiles, pusher, seed) that pic_restore
// compares with the simulation it restores into, then the state in a fixed
// order: step and tallies, laser, QED set-up, field arrays with their ghost
// layers (raw, in the simulation's precision), per species the live count
// and the live particles in array order with the tile index of the last sort,
// and the surrogate networks.  Everything a later step reads is there, so a
// restored run continues with the same Philox counters, the same sort phase
// and the same particle order as the run that wrote the file.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "sim.cuh"

using namespace pic;

namespace {

constexpr char kMagic[8] = {'P', 'I', 'C', 'C', 'K', 'P', 'T', '1'};
constexpr uint32_t kVersion = 1;

// configuration the state depends on: restore only into an equal one
struct Signature {
    int dim, precision, nsp, sort_interval, pusher, order;
    int n[3], bc[3], tile_log2[3];
    double dx[3], dt;
    uint64_t seed;
    double q[PIC_MAX_SPECIES], m[PIC_MAX_SPECIES], w[PIC_MAX_SPECIES];
    long long cap[PIC_MAX_SPECIES];
    int kind[PIC_MAX_SPECIES], qed[PIC_MAX_SPECIES];
};

Signature signature(const pic_sim *s)
{
    Signature z;
    std::memset(&z, 0, sizeof z);  // padding bytes too: the struct is compared with memcmp
    z.dim = s->g.dim;
    z.precision = s->precision;
    z.nsp = s->nsp;
    z.sort_interval = s->sort_interval;
    z.pusher = s->pusher;
    z.order = s->g.order;
    for (int d = 0; d < 3; d++) {
        z.n[d] = s->g.n[d];
        z.bc[d] = s->g.bc[d];
        z.tile_log2[d] = s->g.tile_log2[d];
        z.dx[d] = s->g.dx[d];
    }
    z.dt = s->g.dt;
    z.seed = s->seed;
    for (int i = 0; i < s->nsp; i++) {
        z.q[i] = s->sp[i].q;
        z.m[i] = s->sp[i].m;
        z.w[i] = s->sp[i].w;
        z.cap[i] = s->sp[i].cap;
        z.kind[i] = s->sp[i].kind;
        z.qed[i] = s->sp[i].qed;
    }
    return z;
}

struct File {
    FILE *f = nullptr;
    bool ok = true;
    ~File()
    {
        if (f) fclose(f);
    }
    void put(const void *p, size_t n)
    {
        if (ok && n && fwrite(p, 1, n, f) != n) ok = false;
    }
    void get(void *p, size_t n)
    {
        if (ok && n && fread(p, 1, n, f) != n) ok = false;
    }
    template <typename T>
    void put(const T &v) { put(&v, sizeof v); }
    template <typename T>
    void get(T &v) { get(&v, sizeof v); }
};

// device <-> file through one host buffer
int dev_put(pic_sim *s, File &F, const void *dev, size_t bytes, std::vector<char> &h)
{
    if (!bytes) return PIC_OK;
    h.resize(bytes);
    CK(cudaMemcpyAsync(h.data(), dev, bytes, cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    F.put(h.data(), bytes);
    return PIC_OK;
}

int dev_get(pic_sim *s, File &F, void *dev, size_t bytes, std::vector<char> &h)
{
    if (!bytes) return PIC_OK;
    h.resize(bytes);
    F.get(h.data(), bytes);
    if (!F.ok) return fail(s, PIC_ERR_ARG, "pic_restore: the file ends early");
    CK(cudaMemcpyAsync(dev, h.data(), bytes, cudaMemcpyHostToDevice, s->st));
    CK(cudaStreamSynchronize(s->st));
    return PIC_OK;
}

// the per-particle arrays of one species buffer, with their element sizes
int species_arrays(pic_sim *s, int i, void **ptr, size_t *esz)
{
    SpeciesState &p = s->sp[i];
    const int b = p.cur;
    int k = 0;
    ptr[k] = p.cell[b];
    esz[k++] = 4;
    for (int d = 0; d < s->g.dim; d++) {
        ptr[k] = s->precision == PIC_PREC_FP64_PLAIN ? (void *)p.x[b][d] : (void *)p.off[b][d];
        esz[k++] = rsize(s);
    }
    for (int d = 0; d < 3; d++) {
        ptr[k] = s->precision == PIC_PREC_FP64_PLAIN ? (void *)p.ud[b][d] : (void *)p.uf[b][d];
        esz[k++] = rsize(s);
    }
    if (p.has_qed_arrays()) {
        ptr[k] = p.tau[b];
        esz[k++] = 8;
        ptr[k] = p.id[b];
        esz[k++] = 8;
    }
    return k;
}

}  // namespace

extern "C" {

int pic_save(pic_sim *s, const char *path)
{
    if (!s) return PIC_ERR_ARG;
    if (!path) return fail(s, PIC_ERR_ARG, "pic_save: null path");
    CK(cudaStreamSynchronize(s->st));
    File F;
    F.f = fopen(path, "wb");
    if (!F.f) return fail(s, PIC_ERR_ARG, "pic_save: cannot open %s for writing", path);
    std::vector<char> h;
    F.put(kMagic, sizeof kMagic);
    F.put(kVersion);
    const Signature sig = signature(s);
    F.put(sig);
    // step and tallies
    F.put(s->step);
    double tally[2] = {0.0, 0.0};
    CK(cudaMemcpyAsync(&tally[0], s->d_eabs, 8, cudaMemcpyDeviceToHost, s->st));
    CK(cudaMemcpyAsync(&tally[1], s->d_elost, 8, cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
    F.put(tally);
    F.put(s->rho_bg);
    // laser and QED set-up (their device parts are rebuilt from these)
    F.put(s->laser.on);
    F.put(s->lp);
    const int qed_on = s->qed_on ? 1 : 0;
    F.put(qed_on);
    F.put(s->qed);
    // fields and currents with ghosts
    if (int rc = dev_put(s, F, s->F, (size_t)NCOMP * s->g.vol * rsize(s), h)) return rc;
    // species
    for (int i = 0; i < s->nsp; i++) {
        SpeciesState &p = s->sp[i];
        long long cnt = 0;
        CK(cudaMemcpyAsync(&cnt, p.d_count, 8, cudaMemcpyDeviceToHost, s->st));
        CK(cudaStreamSynchronize(s->st));
        F.put(cnt);
        F.put(p.n_hi);
        void *ptr[10];
        size_t esz[10];
        const int na = species_arrays(s, i, ptr, esz);
        for (int a = 0; a < na; a++)
            if (int rc = dev_put(s, F, ptr[a], (size_t)cnt * esz[a], h)) return rc;
        // the tile index of the last sort (the tiled push walks it until the next one)
        if (int rc = dev_put(s, F, p.tile_start, (size_t)(s->g.ntiles + 1) * 4, h)) return rc;
        const int items = p.items && p.items_valid ? 1 : 0;
        F.put(items);
        if (items) {
            uint32_t nit = 0;
            CK(cudaMemcpyAsync(&nit, p.nitems, 4, cudaMemcpyDeviceToHost, s->st));
            CK(cudaStreamSynchronize(s->st));
            F.put(nit);
            if (int rc = dev_put(s, F, p.items, (size_t)nit * sizeof(TileItem), h)) return rc;
        }
    }
    // surrogate networks: master parameters, Adam moments, normalisation
    for (int q = 0; q < 2; q++) {
        const MlpNet &net = s->net[q];
        const int ready = net.ready ? 1 : 0;
        F.put(ready);
        if (ready) {
            if (int rc = dev_put(s, F, net.P, 3 * (size_t)kMlpNParams * sizeof(float), h)) return rc;
            F.put(net.nrm);
        }
    }
    F.put(kMagic, sizeof kMagic);
    if (!F.ok) return fail(s, PIC_ERR_ARG, "pic_save: write to %s failed", path);
    if (fclose(F.f) != 0) {
        F.f = nullptr;
        return fail(s, PIC_ERR_ARG, "pic_save: closing %s failed", path);
    }
    F.f = nullptr;
    return PIC_OK;
}

int pic_restore(pic_sim *s, const char *path)
{
    if (!s) return PIC_ERR_ARG;
    if (!path) return fail(s, PIC_ERR_ARG, "pic_restore: null path");
    CK(cudaStreamSynchronize(s->st));
    File F;
    F.f = fopen(path, "rb");
    if (!F.f) return fail(s, PIC_ERR_ARG, "pic_restore: cannot open %s", path);
    std::vector<char> h;
    char magic[8];
    uint32_t version = 0;
    F.get(magic, sizeof magic);
    F.get(version);
    if (!F.ok || std::memcmp(magic, kMagic, sizeof kMagic) || version != kVersion)
        return fail(s, PIC_ERR_ARG, "pic_restore: %s is not a checkpoint of this version", path);
    Signature sig;
    F.get(sig);
    const Signature mine = signature(s);
    if (!F.ok || std::memcmp(&sig, &mine, sizeof sig))
        return fail(s, PIC_ERR_ARG, "pic_restore: %s was written by a simulation of another configuration", path);
    long long step = 0;
    double tally[2], rho_bg = 0.0;
    int laser_on = 0, qed_on = 0;
    pic_laser lp{};
    pic_qed qed{};
    F.get(step);
    F.get(tally);
    F.get(rho_bg);
    F.get(laser_on);
    F.get(lp);
    F.get(qed_on);
    F.get(qed);
    if (!F.ok) return fail(s, PIC_ERR_ARG, "pic_restore: the file ends early");
    if (laser_on) {
        if (int rc = pic_set_laser(s, &lp)) return rc;
    } else {
        s->laser.on = 0;
    }
    if (qed_on) {
        if (int rc = pic_set_qed(s, &qed)) return rc;
    } else {
        s->qed_on = false;
    }
    if (int rc = dev_get(s, F, s->F, (size_t)NCOMP * s->g.vol * rsize(s), h)) return rc;
    for (int i = 0; i < s->nsp; i++) {
        SpeciesState &p = s->sp[i];
        long long cnt = 0, n_hi = 0;
        F.get(cnt);
        F.get(n_hi);
        if (!F.ok || cnt < 0 || cnt > p.cap || n_hi < cnt || n_hi > p.cap)
            return fail(s, PIC_ERR_ARG, "pic_restore: bad particle count of species %d", i);
        void *ptr[10];
        size_t esz[10];
        const int na = species_arrays(s, i, ptr, esz);
        for (int a = 0; a < na; a++)
            if (int rc = dev_get(s, F, ptr[a], (size_t)cnt * esz[a], h)) return rc;
        // slots past the live count up to the host bound read as dead
        if (n_hi > cnt) CK(cudaMemsetAsync(p.cell[p.cur] + cnt, 0xFF, (size_t)(n_hi - cnt) * 4, s->st));
        CK(cudaMemcpyAsync(p.d_count, &cnt, 8, cudaMemcpyHostToDevice, s->st));
        if (int rc = dev_get(s, F, p.tile_start, (size_t)(s->g.ntiles + 1) * 4, h)) return rc;
        int items = 0;
        F.get(items);
        p.items_valid = false;
        if (items) {
            uint32_t nit = 0;
            F.get(nit);
            if (!F.ok || !p.items || (long long)nit > p.items_cap)
                return fail(s, PIC_ERR_ARG, "pic_restore: bad tile index of species %d", i);
            if (int rc = dev_get(s, F, p.items, (size_t)nit * sizeof(TileItem), h)) return rc;
            CK(cudaMemcpyAsync(p.nitems, &nit, 4, cudaMemcpyHostToDevice, s->st));
            p.items_valid = true;
        }
        CK(cudaStreamSynchronize(s->st));
        p.n_hi = n_hi;
    }
    for (int q = 0; q < 2; q++) {
        int ready = 0;
        F.get(ready);
        if (!F.ok) return fail(s, PIC_ERR_ARG, "pic_restore: the file ends early");
        if (!ready) {
            s->net[q].ready = false;
            continue;
        }
        std::vector<float> P(3 * (size_t)kMlpNParams);
        MlpNorm nrm{};
        F.get(P.data(), P.size() * sizeof(float));
        F.get(nrm);
        if (!F.ok) return fail(s, PIC_ERR_ARG, "pic_restore: the file ends early");
        // allocates the network and builds its BF16 image from the parameters
        pic_mlp_info info{std::exp(nrm.lnchi_lo), std::exp(nrm.lnchi_hi), nrm.mu, nrm.sd};
        if (int rc = pic_mlp_set(s, q, P.data(), &info)) return rc;
        MlpNet &net = s->net[q];
        net.nrm = nrm;  // bit-exact normalisation, not the round trip through exp/log
        CK(cudaMemcpyAsync(net.M, P.data() + kMlpNParams, 2 * (size_t)kMlpNParams * sizeof(float),
                           cudaMemcpyHostToDevice, s->st));
        CK(cudaStreamSynchronize(s->st));
    }
    char tail[8];
    F.get(tail, sizeof tail);
    if (!F.ok || std::memcmp(tail, kMagic, sizeof kMagic))
        return fail(s, PIC_ERR_ARG, "pic_restore: %s is truncated or corrupt", path);
    CK(cudaMemcpyAsync(s->d_eabs, &tally[0], 8, cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(s->d_elost, &tally[1], 8, cudaMemcpyHostToDevice, s->st));
    CK(cudaMemsetAsync(s->d_err, 0, sizeof(int), s->st));
    CK(cudaStreamSynchronize(s->st));
    s->step = step;
    s->rho_bg = rho_bg;
    return PIC_OK;
}

}  // extern "C"
