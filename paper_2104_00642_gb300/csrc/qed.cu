// qed.cu -- QED tables (built on the host in FP64 from Eqs. (23), (24)),
// the table-evaluation entry points, and the kernels that append emitted
// photons and created pairs to their species.
//
// Tables.  The Bessel functions enter only through K_{2/3}(y) and
// Int_y^inf K_{1/3}; both are tabulated once on a fine logarithmic y grid
// from their integral representations
//   K_nu(y) = Int_0^inf exp(-y cosh t) cosh(nu t) dt,
//   Int_y^inf K_{1/3} = Int_0^inf exp(-y cosh t) cosh(t/3) / cosh t dt,
// and interpolated (cubic in ln y).  For every chi of the table grid the
// spectrum is integrated cumulatively on a fine grid of s = fraction^(1/3)
// (removing the u^{-2/3} behaviour of Eq. (23) at small u), giving the
// total G(chi) and, by inverse interpolation, the inverse CDF.
#include <cmath>
#include <mutex>
#include <vector>

#include "qed.cuh"
#include "qed_host.cuh"
#include "scan_dev.cuh"
#include "sort.cuh"

namespace pic {

namespace {

constexpr int kNchi = 256;
constexpr double kChiMin = 1e-4, kChiMax = 1e3;
constexpr int kNr = 512;
constexpr int kNs = 4096;
constexpr int kNy = 8001;
constexpr double kYmin = 1e-10, kYmax = 700.0;

// ln K + y is tabulated (not ln K): K ~ exp(-y) at large y, and ln K + y is
// smooth in ln y over the whole range
struct BesselTable {
    double lny0, dlny;
    std::vector<double> lnk23, lnik13;  // ln K_{2/3}(y) + y, ln Int_y K_{1/3} + y
};

double trap_bessel(double nu, double y, bool over_cosh)
{
    // exp(-y cosh t) falls below e^-800 at t_max; the integrand is analytic
    // in a strip, so the trapezoid rule converges exponentially in 1/h
    const double tmax = std::acosh(std::max(800.0 / y, 1.0)) + 0.5;
    const int n = std::max(64, (int)std::ceil(tmax / 0.04));
    const double h = tmax / n;
    double s = 0.0;
    for (int i = 0; i <= n; i++) {
        const double t = i * h, ch = std::cosh(t);
        double f = std::exp(-y * ch) * std::cosh(nu * t);
        if (over_cosh) f /= ch;
        s += (i == 0 || i == n) ? 0.5 * f : f;
    }
    return s * h;
}

const BesselTable &bessel_table()
{
    static BesselTable B;
    static std::once_flag once;
    std::call_once(once, [] {
        B.lny0 = std::log(kYmin);
        B.dlny = (std::log(kYmax) - B.lny0) / (kNy - 1);
        B.lnk23.resize(kNy);
        B.lnik13.resize(kNy);
        for (int i = 0; i < kNy; i++) {
            const double y = std::exp(B.lny0 + i * B.dlny);
            B.lnk23[i] = std::log(trap_bessel(2.0 / 3.0, y, false)) + y;
            B.lnik13[i] = std::log(trap_bessel(1.0 / 3.0, y, true)) + y;
        }
    });
    return B;
}

// the host view of the Bessel table in the layout the device reads
QedTables bessel_view()
{
    const BesselTable &B = bessel_table();
    QedTables T{};
    T.bes_k23 = B.lnk23.data();
    T.bes_ik13 = B.lnik13.data();
    T.nbes = kNy;
    T.bes_lny0 = B.lny0;
    T.bes_dlny = B.dlny;
    T.bes_ymin = kYmin;
    T.bes_ymax = kYmax;
    return T;
}

// K_{2/3}(y) and Int_y^inf K_{1/3}: the same evaluation the device makes
// (qed_bessel: below the table the leading small-argument behaviour, exact
// to O(y^{4/3}); zero beyond kYmax)
void bessel(double y, double &k23, double &ik13)
{
    static const QedTables T = bessel_view();
    qed_bessel(T, y, k23, ik13);
}

// Eq. (23): ((1-u) + 1/(1-u)) K_{2/3}(y) - Int_y^inf K_{1/3}, y = 2u / (3 chi (1-u))
double spec_rad(double u, double chi)
{
    if (u <= 0.0 || u >= 1.0) return 0.0;
    double k, ik;
    bessel(2.0 * u / (3.0 * chi * (1.0 - u)), k, ik);
    return ((1.0 - u) + 1.0 / (1.0 - u)) * k - ik;
}

// Eq. (24): ((v^2 + (1-v)^2) / (v (1-v))) K_{2/3}(y) + Int_y^inf K_{1/3}, y = 2 / (3 chi v (1-v))
double spec_pair(double v, double chi)
{
    if (v <= 0.0 || v >= 1.0) return 0.0;
    double k, ik;
    bessel(2.0 / (3.0 * chi * v * (1.0 - v)), k, ik);
    return ((v * v + (1.0 - v) * (1.0 - v)) / (v * (1.0 - v))) * k + ik;
}

struct HostTables {
    std::vector<double> lnG[2], inv[2];
};

// Cumulative integral of a spectrum on a grid of fractions f_k, built from
// cells in a local variable where the integrand is smooth:
//   emission, f <= 1/2: f = s^3 (the u^{-2/3} behaviour at small u);
//   emission, f >= 1/2: 1 - f = t^3 (the (1-u)^{-1/3} peak of width ~1/(3 chi)
//     below u = 1 at large chi);
//   pairs, f <= 1/2: f = t^3 (v^{-1/3} above the cut-off at large chi).
// Two-point Gauss per cell.  f[k] increases; C[k] = Int_0^{f_k} F.
void cumulate(int p, double chi, std::vector<double> &f, std::vector<double> &C)
{
    const int n = p == QED_RAD ? 2 * kNs : kNs;
    f.assign(n + 1, 0.0);
    C.assign(n + 1, 0.0);
    const double g = 0.5 / std::sqrt(3.0), w_half = std::cbrt(0.5);
    const double h = w_half / kNs;
    for (int k = 0; k < n; k++) {
        double acc = 0.0;
        for (int q = 0; q < 2; q++) {
            const double z = (q ? g : -g);
            if (p == QED_PAIR || k < kNs) {  // f = w^3, w in [0, (1/2)^(1/3)]
                const double w = (k + 0.5 + z) * h, fr = w * w * w;
                acc += 3.0 * w * w * (p == QED_RAD ? spec_rad(fr, chi) : spec_pair(fr, chi));
            } else {  // 1 - f = t^3, t from (1/2)^(1/3) down to 0
                const double t = w_half - (k - kNs + 0.5 + z) * h, fr = 1.0 - t * t * t;
                acc += 3.0 * t * t * spec_rad(fr, chi);
            }
        }
        C[k + 1] = C[k] + 0.5 * h * acc;
        if (p == QED_PAIR || k < kNs) {
            const double w = (k + 1) * h;
            f[k + 1] = w * w * w;
        } else {
            const double t = w_half - (k + 1 - kNs) * h;
            f[k + 1] = 1.0 - t * t * t;
        }
    }
    if (p == QED_RAD) f[n] = 1.0;
    else f[n] = 0.5;
}

const HostTables &host_tables()
{
    static HostTables H;
    static std::once_flag once;
    std::call_once(once, [] {
        std::vector<double> f, C;
        for (int p = 0; p < 2; p++) {
            H.lnG[p].resize(kNchi);
            H.inv[p].resize((size_t)kNchi * kNr);
        }
        const double lc0 = std::log(kChiMin), dlc = (std::log(kChiMax) - lc0) / (kNchi - 1);
        for (int i = 0; i < kNchi; i++) {
            const double chi = std::exp(lc0 + i * dlc);
            for (int p = 0; p < 2; p++) {
                cumulate(p, chi, f, C);
                const int n = (int)C.size() - 1;
                const double tot = C[n];
                const double G = p == QED_RAD ? tot : 2.0 * tot;  // pairs: symmetric about v = 1/2
                // pairs: ln G + 8/(3 chi) (the exponential small-chi factor removed);
                // underflowed nodes are filled below by linear extrapolation
                H.lnG[p][i] = G > 1e-300 ? std::log(G) + (p == QED_PAIR ? 8.0 / (3.0 * chi) : 0.0) : NAN;
                int k = 0;
                for (int j = 0; j < kNr; j++) {
                    // r grids dense where the inverse is singular: near r = 1
                    // for emission (the high-energy tail), near r = 0 for pairs
                    const double tj = (double)j / (kNr - 1);
                    const double rj = p == QED_RAD ? 1.0 - (1.0 - tj) * (1.0 - tj) : 0.5 * tj * tj;
                    const double target = rj * G;
                    double fr;
                    if (!(tot > 0.0)) fr = f[n] * j / (kNr - 1);
                    else if (j == kNr - 1) fr = f[n];
                    else {
                        while (k < n - 1 && C[k + 1] < target) k++;
                        const double dC = C[k + 1] - C[k];
                        const double a = std::min(std::max(dC > 0.0 ? (target - C[k]) / dC : 0.0, 0.0), 1.0);
                        // interpolate in the cell's local variable, as integrated
                        if (p == QED_PAIR || k < kNs) {
                            const double w0 = std::cbrt(f[k]), w1 = std::cbrt(f[k + 1]), w = w0 + a * (w1 - w0);
                            fr = w * w * w;
                        } else {
                            const double t0 = std::cbrt(1.0 - f[k]), t1 = std::cbrt(1.0 - f[k + 1]);
                            const double t = t0 + a * (t1 - t0);
                            fr = 1.0 - t * t * t;
                        }
                    }
                    H.inv[p][(size_t)i * kNr + j] = std::cbrt(fr);
                }
            }
        }
        for (int p = 0; p < 2; p++) {
            int first = 0;
            while (first < kNchi - 1 && std::isnan(H.lnG[p][first])) first++;
            for (int i = first - 1; i >= 0; i--) H.lnG[p][i] = 2.0 * H.lnG[p][i + 1] - H.lnG[p][i + 2];
        }
    });
    return H;
}

}  // namespace

void qed_spectra(int p, double frac, double chi, double *F) { *F = p == QED_RAD ? spec_rad(frac, chi) : spec_pair(frac, chi); }

size_t qed_table_bytes()
{
    return 2 * ((size_t)kNchi + (size_t)kNchi * kNr) * (sizeof(float) + sizeof(double)) + 2 * (size_t)kNy * 8;
}

// fill a device buffer (qed_table_bytes) and the table view pointing into it
int qed_upload_tables(void *dev, QedTables *T, cudaStream_t st)
{
    const HostTables &H = host_tables();
    std::vector<float> hf;
    std::vector<double> hd;
    for (int p = 0; p < 2; p++) {
        hd.insert(hd.end(), H.lnG[p].begin(), H.lnG[p].end());
        hd.insert(hd.end(), H.inv[p].begin(), H.inv[p].end());
    }
    hf.assign(hd.begin(), hd.end());
    char *base = (char *)dev;
    if (cudaMemcpyAsync(base, hd.data(), hd.size() * 8, cudaMemcpyHostToDevice, st) != cudaSuccess) return -1;
    if (cudaMemcpyAsync(base + hd.size() * 8, hf.data(), hf.size() * 4, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return -1;
    if (cudaStreamSynchronize(st) != cudaSuccess) return -1;
    // the Bessel table after the rate and inverse-CDF tables
    const BesselTable &B = bessel_table();
    char *bes = base + hd.size() * 8 + hf.size() * 4;
    if (cudaMemcpyAsync(bes, B.lnk23.data(), (size_t)kNy * 8, cudaMemcpyHostToDevice, st) != cudaSuccess) return -1;
    if (cudaMemcpyAsync(bes + (size_t)kNy * 8, B.lnik13.data(), (size_t)kNy * 8, cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
        return -1;
    if (cudaStreamSynchronize(st) != cudaSuccess) return -1;
    const double *d = (const double *)base;
    const float *f = (const float *)(base + hd.size() * 8);
    size_t off = 0;
    for (int p = 0; p < 2; p++) {
        T->lnG_d[p] = d + off;
        T->lnG_f[p] = f + off;
        off += kNchi;
        T->inv_d[p] = d + off;
        T->inv_f[p] = f + off;
        off += (size_t)kNchi * kNr;
    }
    T->nchi = kNchi;
    T->nr = kNr;
    T->bes_k23 = (const double *)bes;
    T->bes_ik13 = (const double *)bes + kNy;
    T->nbes = kNy;
    T->bes_lny0 = B.lny0;
    T->bes_dlny = B.dlny;
    T->bes_ymin = kYmin;
    T->bes_ymax = kYmax;
    T->lnchi0 = std::log(kChiMin);
    T->dlnchi = (std::log(kChiMax) - T->lnchi0) / (kNchi - 1);
    T->lnchi0_f = (float)T->lnchi0;
    T->inv_dlnchi_f = (float)(1.0 / T->dlnchi);
    return 0;
}

// ---------------------------------------------------------------------
// table evaluation (inspection entry points)
// ---------------------------------------------------------------------
template <typename R>
__global__ void k_qed_eval(QedTables T, int p, long long n, const double *chi, const double *r, double *out)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if constexpr (sizeof(R) == 4)  // the FP32 form's own FP32 arithmetic, as its pushes evaluate it
        out[i] = r ? (double)qed_sample_f32(T, p, (float)chi[i], (float)r[i]) : (double)qed_rate_f32(T, p, (float)chi[i]);
    else
        out[i] = r ? qed_sample<R>(T, p, chi[i], r[i]) : qed_rate<R>(T, p, chi[i]);
}

void launch_qed_eval(const QedTables &T, bool f64, int p, long long n, const double *chi, const double *r, double *out,
                     cudaStream_t st)
{
    if (n <= 0) return;
    note_launch();
    if (f64) k_qed_eval<double><<<div_up(n, 256), 256, 0, st>>>(T, p, n, chi, r, out);
    else k_qed_eval<float><<<div_up(n, 256), 256, 0, st>>>(T, p, n, chi, r, out);
}

// ---------------------------------------------------------------------
// spawning: the events of a species are ranked in array order and the
// children appended at the end of their species (deterministic order).  The
// ranks come in two passes over the flags: the sums of blocks of kScanItems
// flags, scanned (scan_block_sums), then the spawn kernel itself, which
// strides over the blocks of flags: a block whose scanned sums show no event
// is skipped without reading its flags; otherwise the 256 threads read 16
// flags each, scan them and add the block's offset.
// ---------------------------------------------------------------------
constexpr int kSpawnThreads = 256, kSpawnPer = kScanItems / kSpawnThreads;

inline int spawn_grid(long long m)
{
    static int nsm = 0;
    if (!nsm) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    }
    return (int)std::min<long long>(scan_blocks(m), 4ll * nsm);
}

// the flags (0 or 1) of block b, kSpawnPer per thread from p0, as a bit mask,
// and the rank of this thread's first event; false (block-uniform) when the
// block has no event.  m: the flags' end (the parents' device count: the
// slots past it count as no event, as in the block sums)
__device__ __forceinline__ bool spawn_ranks(const uint32_t *__restrict__ ev, long long m,
                                            const uint32_t *__restrict__ bsum, long long b, long long &p0,
                                            uint32_t &bits, uint32_t &run)
{
    __shared__ uint32_t sh[32];
    if (bsum[b + 1] == bsum[b]) return false;
    p0 = b * kScanItems + (long long)threadIdx.x * kSpawnPer;
    bits = 0;
    if (p0 + kSpawnPer <= m && (reinterpret_cast<uintptr_t>(ev) & 15u) == 0) {
#pragma unroll
        for (int k = 0; k < kSpawnPer; k += 4) {
            const uint4 v = *reinterpret_cast<const uint4 *>(ev + p0 + k);
            bits |= (v.x ? 1u : 0u) << k | (v.y ? 2u : 0u) << k | (v.z ? 4u : 0u) << k | (v.w ? 8u : 0u) << k;
        }
    } else {
#pragma unroll
        for (int k = 0; k < kSpawnPer; k++)
            if (p0 + k < m && ev[p0 + k]) bits |= 1u << k;
    }
    uint32_t tot;
    run = block_excl_scan<kSpawnThreads>((uint32_t)__popc(bits), sh, tot) + bsum[b];
    return true;
}

__global__ void __launch_bounds__(kSpawnThreads) k_spawn_photons_f32(PartF32 parent, const uint32_t *__restrict__ bsum,
                                    const uint32_t *__restrict__ total, long long m, QedParams q, PartF32 ph, double *ph_tau,
                                    uint64_t *ph_id, uint32_t *ph_ev, long long *ph_count, long long ph_cap, int dim,
                                    int *err)
{
    const long long base = *ph_count;
    if (blockIdx.x == 0 && threadIdx.x == 0 && base + *total > ph_cap) atomicOr(err, ERR_CAPACITY);
    m = min(m, *parent.dn);  // (past the parents' device count: no event)
    const long long nb = (m + kScanItems - 1) / kScanItems;
    for (long long b = blockIdx.x; b < nb; b += gridDim.x) {
        long long p0;
        uint32_t bits, run;
        if (!spawn_ranks(q.ev, m, bsum, b, p0, bits, run)) continue;
        for (; bits; bits &= bits - 1) {
            const long long p = p0 + (__ffs(bits) - 1);
            const uint32_t rank = run++;
            const long long dst = base + rank;
            if (dst >= ph_cap) continue;
            uint32_t w[4];
            const uint64_t pid = q.id[p];
            philox4x32_10((uint32_t)pid, (uint32_t)(pid >> 32), q.step, QP_EMIT, q.key[0], q.key[1], w);
            const uint64_t cid = ((uint64_t)w[3] << 32) | w[2];
            ph.cell[dst] = parent.cell[p];  // the parent's x^{n+1}
#pragma unroll
            for (int d = 0; d < 3; d++)
                if (d < dim) ph.off[d][dst] = parent.off[d][p];  // (constant indices: the views stay in registers)
            ph.u[0][dst] = q.evk[4 * p];
            ph.u[1][dst] = q.evk[4 * p + 1];
            ph.u[2][dst] = q.evk[4 * p + 2];
            ph_id[dst] = cid;
            ph_tau[dst] = initial_tau_f32(cid, q.key);
            ph_ev[dst] = 0;
        }
    }
}

__global__ void __launch_bounds__(kSpawnThreads) k_spawn_pairs_f32(PartF32 phot, const uint32_t *__restrict__ bsum, const uint32_t *__restrict__ total, long long m,
                                  QedParams q, PartF32 el, double *el_tau, uint64_t *el_id, uint32_t *el_ev,
                                  long long *el_count, long long el_cap, PartF32 po, double *po_tau, uint64_t *po_id,
                                  uint32_t *po_ev, long long *po_count, long long po_cap, int dim, int *err)
{
    const long long be = *el_count, bp = *po_count;
    if (blockIdx.x == 0 && threadIdx.x == 0 && (be + *total > el_cap || bp + *total > po_cap))
        atomicOr(err, ERR_CAPACITY);
    m = min(m, *phot.dn);  // (past the photons' device count: no event)
    const long long nb = (m + kScanItems - 1) / kScanItems;
    for (long long b = blockIdx.x; b < nb; b += gridDim.x) {
        long long p0;
        uint32_t bits, run;
        if (!spawn_ranks(q.ev, m, bsum, b, p0, bits, run)) continue;
        for (; bits; bits &= bits - 1) {
            const long long p = p0 + (__ffs(bits) - 1);
            const uint32_t rank = run++;
            const long long de = be + rank, dp = bp + rank;
            if (de >= el_cap || dp >= po_cap) continue;
            uint32_t w[4];
            const uint64_t pid = q.id[p];
            philox4x32_10((uint32_t)pid, (uint32_t)(pid >> 32), q.step, QP_PAIR, q.key[0], q.key[1], w);
            const uint64_t eid = ((uint64_t)w[3] << 32) | w[2], pid2 = eid + 1;
            // event data: the photon's momentum k and the positron fraction v
            const double kx = q.evk[4 * p], ky = q.evk[4 * p + 1], kz = q.evk[4 * p + 2], v = q.evk[4 * p + 3];
            const double k = sqrt(kx * kx + ky * ky + kz * kz);
            // the pair is born where the photon converted (its x^{n+1}); the photon dies
            const uint32_t cell = phot.cell[p];
#pragma unroll
            for (int d = 0; d < 3; d++) {
                if (d >= dim) break;
                el.off[d][de] = phot.off[d][p];
                po.off[d][dp] = phot.off[d][p];
            }
            el.cell[de] = cell;
            po.cell[dp] = cell;
            phot.cell[p] = kDead;
            const double ep = v * k, em = (1.0 - v) * k;  // eps_+ and eps_- (m c^2)
            const double pm = sqrt(fmax(em * em - 1.0, 0.0)), pp = sqrt(fmax(ep * ep - 1.0, 0.0));
            const double inv = k > 0.0 ? 1.0 / k : 0.0;
            el.u[0][de] = (float)(pm * kx * inv);
            el.u[1][de] = (float)(pm * ky * inv);
            el.u[2][de] = (float)(pm * kz * inv);
            po.u[0][dp] = (float)(pp * kx * inv);
            po.u[1][dp] = (float)(pp * ky * inv);
            po.u[2][dp] = (float)(pp * kz * inv);
            el_id[de] = eid;
            po_id[dp] = pid2;
            el_tau[de] = initial_tau_f32(eid, q.key);
            po_tau[dp] = initial_tau_f32(pid2, q.key);
            el_ev[de] = 0;
            po_ev[dp] = 0;
        }
    }
}

// FP64 plain form: absolute positions, event data as 4 doubles per particle
__global__ void __launch_bounds__(kSpawnThreads) k_spawn_photons_f64(PartF64 parent, const uint32_t *__restrict__ bsum,
                                    const uint32_t *__restrict__ total, long long m, QedParams q, PartF64 ph, double *ph_tau,
                                    uint64_t *ph_id, uint32_t *ph_ev, long long *ph_count, long long ph_cap, int dim,
                                    int *err)
{
    const long long base = *ph_count;
    if (blockIdx.x == 0 && threadIdx.x == 0 && base + *total > ph_cap) atomicOr(err, ERR_CAPACITY);
    m = min(m, *parent.dn);  // (past the parents' device count: no event)
    const long long nb = (m + kScanItems - 1) / kScanItems;
    for (long long b = blockIdx.x; b < nb; b += gridDim.x) {
        long long p0;
        uint32_t bits, run;
        if (!spawn_ranks(q.ev, m, bsum, b, p0, bits, run)) continue;
        for (; bits; bits &= bits - 1) {
            const long long p = p0 + (__ffs(bits) - 1);
            const uint32_t rank = run++;
            const long long dst = base + rank;
            if (dst >= ph_cap) continue;
            uint32_t w[4];
            const uint64_t pid = q.id[p];
            philox4x32_10((uint32_t)pid, (uint32_t)(pid >> 32), q.step, QP_EMIT, q.key[0], q.key[1], w);
            const uint64_t cid = ((uint64_t)w[3] << 32) | w[2];
            const double4 e = reinterpret_cast<const double4 *>(q.evk)[p];
            ph.cell[dst] = parent.cell[p];
#pragma unroll
            for (int d = 0; d < 3; d++)
                if (d < dim) ph.x[d][dst] = parent.x[d][p];
            ph.u[0][dst] = e.x;
            ph.u[1][dst] = e.y;
            ph.u[2][dst] = e.z;
            ph_id[dst] = cid;
            ph_tau[dst] = initial_tau(cid, q.key);
            ph_ev[dst] = 0;
        }
    }
}

__global__ void __launch_bounds__(kSpawnThreads) k_spawn_pairs_f64(PartF64 phot, const uint32_t *__restrict__ bsum, const uint32_t *__restrict__ total, long long m,
                                  QedParams q, PartF64 el, double *el_tau, uint64_t *el_id, uint32_t *el_ev,
                                  long long *el_count, long long el_cap, PartF64 po, double *po_tau, uint64_t *po_id,
                                  uint32_t *po_ev, long long *po_count, long long po_cap, int dim, int *err)
{
    const long long be = *el_count, bp = *po_count;
    if (blockIdx.x == 0 && threadIdx.x == 0 && (be + *total > el_cap || bp + *total > po_cap))
        atomicOr(err, ERR_CAPACITY);
    m = min(m, *phot.dn);  // (past the photons' device count: no event)
    const long long nb = (m + kScanItems - 1) / kScanItems;
    for (long long b = blockIdx.x; b < nb; b += gridDim.x) {
        long long p0;
        uint32_t bits, run;
        if (!spawn_ranks(q.ev, m, bsum, b, p0, bits, run)) continue;
        for (; bits; bits &= bits - 1) {
            const long long p = p0 + (__ffs(bits) - 1);
            const uint32_t rank = run++;
            const long long de = be + rank, dp = bp + rank;
            if (de >= el_cap || dp >= po_cap) continue;
            uint32_t w[4];
            const uint64_t pid = q.id[p];
            philox4x32_10((uint32_t)pid, (uint32_t)(pid >> 32), q.step, QP_PAIR, q.key[0], q.key[1], w);
            const uint64_t eid = ((uint64_t)w[3] << 32) | w[2], pid2 = eid + 1;
            const double4 e = reinterpret_cast<const double4 *>(q.evk)[p];
            const double k = sqrt(e.x * e.x + e.y * e.y + e.z * e.z);
            const uint32_t cell = phot.cell[p];
#pragma unroll
            for (int d = 0; d < 3; d++) {
                if (d >= dim) break;
                el.x[d][de] = phot.x[d][p];
                po.x[d][dp] = phot.x[d][p];
            }
            el.cell[de] = cell;
            po.cell[dp] = cell;
            phot.cell[p] = kDead;
            const double ep = e.w * k, em = (1.0 - e.w) * k;
            const double pm = sqrt(fmax(em * em - 1.0, 0.0)), pp = sqrt(fmax(ep * ep - 1.0, 0.0));
            const double inv = k > 0.0 ? 1.0 / k : 0.0;
            el.u[0][de] = pm * e.x * inv;
            el.u[1][de] = pm * e.y * inv;
            el.u[2][de] = pm * e.z * inv;
            po.u[0][dp] = pp * e.x * inv;
            po.u[1][dp] = pp * e.y * inv;
            po.u[2][dp] = pp * e.z * inv;
            el_id[de] = eid;
            po_id[dp] = pid2;
            el_tau[de] = initial_tau(eid, q.key);
            po_tau[dp] = initial_tau(pid2, q.key);
            el_ev[de] = 0;
            po_ev[dp] = 0;
        }
    }
}

__global__ void k_add_count(long long *count, const uint32_t *total, long long cap)
{
    const long long c = *count + *total;
    *count = c > cap ? cap : c;
}

// a pair is created only where both its electron and its positron find room
// (the spawn kernels skip the rest), so both counts advance by the same number
__global__ void k_add_pair_counts(long long *el_count, long long *po_count, const uint32_t *total, long long el_cap,
                                  long long po_cap)
{
    long long n = *total;
    n = min(n, el_cap - *el_count);
    n = min(n, po_cap - *po_count);
    if (n < 0) n = 0;
    *el_count += n;
    *po_count += n;
}

__global__ void k_init_qed(long long first, long long n, uint64_t id0, uint64_t *id, double *tau, uint32_t k0,
                           uint32_t k1)
{
    const long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    const uint64_t v = id0 + (uint64_t)(first + a);
    id[first + a] = v;
    const uint32_t key[2] = {k0, k1};
    tau[first + a] = initial_tau(v, key);
}

void launch_init_qed(long long first, long long n, uint64_t id0, uint64_t *id, double *tau, const uint32_t *key,
                     cudaStream_t st)
{
    if (n <= 0) return;
    note_launch();
    k_init_qed<<<div_up(n, 256), 256, 0, st>>>(first, n, id0, id, tau, key[0], key[1]);
}

void launch_spawn_photons(const PartF32 &parent, const uint32_t *bsum, const uint32_t *total, long long m,
                          const QedParams &q,
                          const PartF32 &ph, double *ph_tau, uint64_t *ph_id, uint32_t *ph_ev, long long *ph_count,
                          long long ph_cap, int dim, int *err, cudaStream_t st)
{
    if (parent.n == 0 || m <= 0) return;
    note_launch(2);
    k_spawn_photons_f32<<<spawn_grid(m), kSpawnThreads, 0, st>>>(parent, bsum, total, m, q, ph, ph_tau, ph_id, ph_ev,
                                                              ph_count, ph_cap, dim, err);
    k_add_count<<<1, 1, 0, st>>>(ph_count, total, ph_cap);
}

void launch_spawn_pairs(const PartF32 &phot, const uint32_t *bsum, const uint32_t *total, long long m,
                        const QedParams &q,
                        const PartF32 &el, double *el_tau, uint64_t *el_id, uint32_t *el_ev, long long *el_count,
                        long long el_cap, const PartF32 &po, double *po_tau, uint64_t *po_id, uint32_t *po_ev,
                        long long *po_count, long long po_cap, int dim, int *err, cudaStream_t st)
{
    if (phot.n == 0 || m <= 0) return;
    note_launch(2);
    k_spawn_pairs_f32<<<spawn_grid(m), kSpawnThreads, 0, st>>>(phot, bsum, total, m, q, el, el_tau, el_id, el_ev, el_count,
                                                          el_cap, po, po_tau, po_id, po_ev, po_count, po_cap, dim, err);
    k_add_pair_counts<<<1, 1, 0, st>>>(el_count, po_count, total, el_cap, po_cap);
}

void launch_spawn_photons(const PartF64 &parent, const uint32_t *bsum, const uint32_t *total, long long m,
                          const QedParams &q,
                          const PartF64 &ph, double *ph_tau, uint64_t *ph_id, uint32_t *ph_ev, long long *ph_count,
                          long long ph_cap, int dim, int *err, cudaStream_t st)
{
    if (parent.n == 0 || m <= 0) return;
    note_launch(2);
    k_spawn_photons_f64<<<spawn_grid(m), kSpawnThreads, 0, st>>>(parent, bsum, total, m, q, ph, ph_tau, ph_id, ph_ev,
                                                              ph_count, ph_cap, dim, err);
    k_add_count<<<1, 1, 0, st>>>(ph_count, total, ph_cap);
}

void launch_spawn_pairs(const PartF64 &phot, const uint32_t *bsum, const uint32_t *total, long long m,
                        const QedParams &q,
                        const PartF64 &el, double *el_tau, uint64_t *el_id, uint32_t *el_ev, long long *el_count,
                        long long el_cap, const PartF64 &po, double *po_tau, uint64_t *po_id, uint32_t *po_ev,
                        long long *po_count, long long po_cap, int dim, int *err, cudaStream_t st)
{
    if (phot.n == 0 || m <= 0) return;
    note_launch(2);
    k_spawn_pairs_f64<<<spawn_grid(m), kSpawnThreads, 0, st>>>(phot, bsum, total, m, q, el, el_tau, el_id, el_ev, el_count,
                                                          el_cap, po, po_tau, po_id, po_ev, po_count, po_cap, dim, err);
    k_add_pair_counts<<<1, 1, 0, st>>>(el_count, po_count, total, el_cap, po_cap);
}

}  // namespace pic
