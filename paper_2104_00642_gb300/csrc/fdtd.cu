// fdtd.cu -- Yee FDTD half steps (Eqs. (9), (10) over dt/2), the Mur
// absorbing faces with the laser entering through x-min, and the current
// fold of the ghost layers.
//
// One thread per padded cell, x fastest: every row is read and written with
// unit stride (coalesced), each thread updates the three components of its
// cell.  Along periodic axes the ghost layers are computed directly (a
// neighbour that falls off the padded box is taken one period away), so they
// stay bit-identical copies of their images without a separate exchange.
#include "fdtd.cuh"

namespace pic {

// offset of the neighbour one cell along axis d (dir = +1/-1) of the cell
// at padded coordinate p, taken one period away at the padded edge
__device__ __forceinline__ long long nb_off(const Grid &g, int d, int p, int dir)
{
    long long s = d == 0 ? 1 : (d == 1 ? g.sy : g.sz);
    int q = p + dir;
    if (q < -g.G[d]) q += g.n[d];
    else if (q >= g.n[d] + g.G[d]) q -= g.n[d];
    return (long long)(q - p) * s;
}

// is component c updated at padded coordinate (i,j,k)?
__device__ __forceinline__ bool updated(const Grid &g, int c, int i, int j, int k)
{
    int p[3] = {i, j, k};
#pragma unroll
    for (int d = 0; d < 3; d++) {
        if (d >= g.dim || g.bc[d] == PERIODIC) continue;
        int hi = stag(c, d) ? g.n[d] - 1 : g.n[d];
        if (p[d] < 0 || p[d] > hi) return false;
    }
    return true;
}

__device__ __forceinline__ void cell_of_thread(const Grid &g, long long t, int &i, int &j, int &k)
{
    long long e0 = g.ext[0], e1 = g.ext[1];
    i = (int)(t % e0) - g.G[0];
    long long r = t / e0;
    j = (int)(r % e1) - g.G[1];
    k = (int)(r / e1) - g.G[2];
}

// E += h (curl B - J); optionally J = 0 afterwards (J^n is not needed once
// the first half step of step n has used it).
template <typename R, int DIM>
__global__ void k_update_E(R *__restrict__ F, Grid g, R h, int zeroJ)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long tot = (long long)g.ext[0] * g.ext[1] * g.ext[2];
    if (t >= tot) return;
    int i, j, k;
    cell_of_thread(g, t, i, j, k);
    long long o = goff(g, i, j, k);
    const long long V = g.vol;
    const R *Bx = F + BX * V, *By = F + BY * V, *Bz = F + BZ * V;
    R *Ex = F + EX * V, *Ey = F + EY * V, *Ez = F + EZ * V;
    R *Jx = F + JX * V, *Jy = F + JY * V, *Jz = F + JZ * V;
    const R rdx = R(1.0 / g.dx[0]), rdy = R(1.0 / g.dx[1]), rdz = R(1.0 / g.dx[2]);
    R cx = 0, cy = 0, cz = 0;
    long long mx = nb_off(g, 0, i, -1);
    cy -= (Bz[o] - Bz[o + mx]) * rdx;
    cz += (By[o] - By[o + mx]) * rdx;
    if (DIM >= 2) {
        long long my = nb_off(g, 1, j, -1);
        cx += (Bz[o] - Bz[o + my]) * rdy;
        cz -= (Bx[o] - Bx[o + my]) * rdy;
    }
    if (DIM >= 3) {
        long long mz = nb_off(g, 2, k, -1);
        cx -= (By[o] - By[o + mz]) * rdz;
        cy += (Bx[o] - Bx[o + mz]) * rdz;
    }
    R jx = Jx[o], jy = Jy[o], jz = Jz[o];
    if (updated(g, EX, i, j, k)) Ex[o] += h * (cx - jx);
    if (updated(g, EY, i, j, k)) Ey[o] += h * (cy - jy);
    if (updated(g, EZ, i, j, k)) Ez[o] += h * (cz - jz);
    if (zeroJ) { Jx[o] = 0; Jy[o] = 0; Jz[o] = 0; }
}

// laser field at the x-min face at time t and transverse (y, z):
// out[0] = E_y, out[1] = E_z (paraxial Gaussian beam, Gaussian intensity
// envelope with full width at half maximum fwhm)
__device__ inline void laser_face(const Laser &L, int dim, double t, double y, double z, double *out)
{
    double r2 = 0.0, amp = 1.0, wxi = 1.0, rinv = 0.0, gouy = 0.0;
    if (dim >= 2) {
        double xr = 0.5 * L.waist * L.waist;
        double xi = -L.x_focus;
        wxi = L.waist * sqrt(1.0 + (xi / xr) * (xi / xr));
        rinv = xi / (xi * xi + xr * xr);
        gouy = atan(xi / xr);
        r2 = (y - L.yc) * (y - L.yc);
        if (dim == 3) r2 += (z - L.zc) * (z - L.zc);
        amp = dim == 3 ? L.waist / wxi : sqrt(L.waist / wxi);
        if (dim == 2) gouy *= 0.5;
    }
    double tau = (t - L.t_peak) / L.fwhm;
    double env = exp(-2.0 * 0.69314718055994530942 * tau * tau);
    double trans = dim >= 2 ? exp(-r2 / (wxi * wxi)) : 1.0;
    double ph = (t - L.t_peak) - 0.5 * r2 * rinv + gouy;
    double a = L.a0 * amp * trans * env;
    double s, c;
    sincos(ph, &s, &c);
    out[0] = a * s;
    out[1] = L.pol == 1 ? a * c : 0.0;
}

// incident B of the laser (a +x wave: Bz = Ey, By = -Ez) a distance xoff
// from the face; (j, k) are wrapped to the interior so that periodic ghost
// rows see the same laser as their images
__device__ inline double incident_B(const Grid &g, const Laser &L, int c, double xoff, double t, int j, int k)
{
    if (g.dim >= 2 && g.bc[1] == PERIODIC) { j %= g.n[1]; if (j < 0) j += g.n[1]; }
    if (g.dim >= 3 && g.bc[2] == PERIODIC) { k %= g.n[2]; if (k < 0) k += g.n[2]; }
    double y = g.dim >= 2 ? (j + (stag(c, 1) ? 0.5 : 0.0)) * g.dx[1] : 0.0;
    double z = g.dim >= 3 ? (k + (stag(c, 2) ? 0.5 : 0.0)) * g.dx[2] : 0.0;
    double e[2];
    laser_face(L, g.dim, t - xoff, y, z, e);
    return c == BZ ? e[0] : (c == BY ? -e[1] : 0.0);
}

// B -= h curl E, then the Mur ghosts of the tangential B on absorbing
// faces: for the scattered part s = B - B_inc of an outgoing wave,
// s_ghost(new) = s_inner(old) + (a-1)/(a+1) (s_inner(new) - s_ghost(old)),
// a = h/dx.  The thread owning the first inner value writes the ghost.
template <typename R, int DIM>
__global__ void k_update_B(R *__restrict__ F, Grid g, R h, double t_new, Laser L)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long tot = (long long)g.ext[0] * g.ext[1] * g.ext[2];
    if (t >= tot) return;
    int i, j, k;
    cell_of_thread(g, t, i, j, k);
    long long o = goff(g, i, j, k);
    const long long V = g.vol;
    const R *Ex = F + EX * V, *Ey = F + EY * V, *Ez = F + EZ * V;
    R *B[3] = {F + BX * V, F + BY * V, F + BZ * V};
    const R rdx = R(1.0 / g.dx[0]), rdy = R(1.0 / g.dx[1]), rdz = R(1.0 / g.dx[2]);
    R cx = 0, cy = 0, cz = 0;
    long long px = nb_off(g, 0, i, +1);
    cy -= (Ez[o + px] - Ez[o]) * rdx;
    cz += (Ey[o + px] - Ey[o]) * rdx;
    if (DIM >= 2) {
        long long py = nb_off(g, 1, j, +1);
        cx += (Ez[o + py] - Ez[o]) * rdy;
        cz -= (Ex[o + py] - Ex[o]) * rdy;
    }
    if (DIM >= 3) {
        long long pz = nb_off(g, 2, k, +1);
        cx -= (Ey[o + pz] - Ey[o]) * rdz;
        cy += (Ex[o + pz] - Ex[o]) * rdz;
    }
    R cur[3] = {cx, cy, cz};
    R oldv[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        oldv[c] = B[c][o];
        if (updated(g, BX + c, i, j, k)) B[c][o] = oldv[c] - h * cur[c];
    }
    int p[3] = {i, j, k};
#pragma unroll
    for (int d = 0; d < DIM; d++) {
        if (g.bc[d] != ABSORB) continue;
        bool lo = p[d] == 0, hi = p[d] == g.n[d] - 1;
        if (!lo && !hi) continue;
        // the transverse position must itself be a swept (updated) one
        bool ok = true;
#pragma unroll
        for (int e = 0; e < DIM; e++)
            if (e != d && g.bc[e] == ABSORB && (p[e] < 0 || p[e] > g.n[e])) ok = false;
        if (!ok) continue;
        double a = (double)h / g.dx[d];
        double c1 = (a - 1.0) / (a + 1.0);
        long long s = d == 0 ? 1 : (d == 1 ? g.sy : g.sz);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            if (!stag(BX + c, d)) continue;
            for (int face = 0; face < 2; face++) {
                if ((face == 0 && !lo) || (face == 1 && !hi)) continue;
                long long og = o + (face == 0 ? -s : s);
                double ig_new = 0, ig_old = 0, ii_new = 0, ii_old = 0;
                if (face == 0 && d == 0 && L.on) {
                    double hx = 0.5 * g.dx[0], t_old = t_new - (double)h;
                    ig_new = incident_B(g, L, BX + c, -hx, t_new, j, k);
                    ig_old = incident_B(g, L, BX + c, -hx, t_old, j, k);
                    ii_new = incident_B(g, L, BX + c, hx, t_new, j, k);
                    ii_old = incident_B(g, L, BX + c, hx, t_old, j, k);
                }
                double sg_old = (double)B[c][og] - ig_old;
                double si_old = (double)oldv[c] - ii_old;
                double si_new = (double)B[c][o] - ii_new;
                B[c][og] = (R)(ig_new + si_old + c1 * (si_new - sg_old));
            }
        }
    }
}

// A set of ncomp arrays (base + q*stride) with per-component staggering
// masks (bit d set = half node along axis d), e.g. Jx,Jy,Jz or rho.
struct FoldSet {
    int ncomp;
    long long stride;
    int mask[3];
};

// periodic fold along axis d: what was deposited into a ghost belongs to
// its image; both end up holding the sum (image + ghost, fixed order)
template <typename R>
__global__ void k_fold_periodic(R *__restrict__ base, FoldSet fs, Grid g, int d)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int G = g.G[d], N = g.n[d];
    long long e[3] = {g.ext[0], g.ext[1], g.ext[2]};
    e[d] = 2 * G;
    long long tot = e[0] * e[1] * e[2];
    if (t >= tot) return;
    int p[3];
    p[0] = (int)(t % e[0]);
    long long r = t / e[0];
    p[1] = (int)(r % e[1]);
    p[2] = (int)(r / e[1]);
    for (int a = 0; a < 3; a++) p[a] -= (a == d) ? 0 : g.G[a];
    int s = p[d];
    int in = s < G ? s : N - 2 * G + s;
    int partner = in < G ? in + N : in - N;
    p[d] = in;
    long long oi = goff(g, p[0], p[1], p[2]);
    p[d] = partner;
    long long op = goff(g, p[0], p[1], p[2]);
    for (int q = 0; q < fs.ncomp; q++) {
        R *J = base + q * fs.stride;
        R v = J[oi] + J[op];
        J[oi] = v;
        J[op] = v;
    }
}

// absorbing axis d: what was deposited outside the physical range leaves
// the domain and is discarded
template <typename R>
__global__ void k_discard_absorb(R *__restrict__ base, FoldSet fs, Grid g, int d)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int G = g.G[d], N = g.n[d];
    long long e[3] = {g.ext[0], g.ext[1], g.ext[2]};
    e[d] = 2 * G;
    long long tot = e[0] * e[1] * e[2];
    if (t >= tot) return;
    int p[3];
    p[0] = (int)(t % e[0]);
    long long r = t / e[0];
    p[1] = (int)(r % e[1]);
    p[2] = (int)(r / e[1]);
    for (int a = 0; a < 3; a++) p[a] -= (a == d) ? 0 : g.G[a];
    int s = p[d];
    p[d] = s < G ? s - G : N + (s - G);  // [-G,0) and [N, N+G)
    long long o = goff(g, p[0], p[1], p[2]);
    for (int q = 0; q < fs.ncomp; q++) {
        int hi = ((fs.mask[q] >> d) & 1) ? N - 1 : N;
        if (p[d] < 0 || p[d] > hi) base[q * fs.stride + o] = 0;
    }
}

// ---------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------

template <typename R>
void launch_update_E(R *F, const Grid &g, double h, bool zeroJ, cudaStream_t st)
{
    long long tot = (long long)g.ext[0] * g.ext[1] * g.ext[2];
    int bs = 256, nb = div_up(tot, bs);
    note_launch();
    if (g.dim == 1) k_update_E<R, 1><<<nb, bs, 0, st>>>(F, g, (R)h, zeroJ);
    else if (g.dim == 2) k_update_E<R, 2><<<nb, bs, 0, st>>>(F, g, (R)h, zeroJ);
    else k_update_E<R, 3><<<nb, bs, 0, st>>>(F, g, (R)h, zeroJ);
}

template <typename R>
void launch_update_B(R *F, const Grid &g, double h, double t_new, const Laser &L, cudaStream_t st)
{
    long long tot = (long long)g.ext[0] * g.ext[1] * g.ext[2];
    int bs = 256, nb = div_up(tot, bs);
    note_launch();
    if (g.dim == 1) k_update_B<R, 1><<<nb, bs, 0, st>>>(F, g, (R)h, t_new, L);
    else if (g.dim == 2) k_update_B<R, 2><<<nb, bs, 0, st>>>(F, g, (R)h, t_new, L);
    else k_update_B<R, 3><<<nb, bs, 0, st>>>(F, g, (R)h, t_new, L);
}

template <typename R>
void launch_fold_set(R *base, const FoldSet &fs, const Grid &g, cudaStream_t st)
{
    for (int d = 0; d < g.dim; d++) {
        long long e[3] = {g.ext[0], g.ext[1], g.ext[2]};
        e[d] = 2 * g.G[d];
        long long tot = e[0] * e[1] * e[2];
        int bs = 256, nb = div_up(tot, bs);
        note_launch();
        if (g.bc[d] == PERIODIC) k_fold_periodic<R><<<nb, bs, 0, st>>>(base, fs, g, d);
        else k_discard_absorb<R><<<nb, bs, 0, st>>>(base, fs, g, d);
    }
}

template <typename R>
void launch_fold(R *F, const Grid &g, cudaStream_t st)
{
    FoldSet fs{3, g.vol, {1, 2, 4}};
    launch_fold_set<R>(F + JX * g.vol, fs, g, st);
}

void launch_fold_rho(double *rho, const Grid &g, cudaStream_t st)
{
    FoldSet fs{1, 0, {0, 0, 0}};
    launch_fold_set<double>(rho, fs, g, st);
}

template void launch_update_E<float>(float *, const Grid &, double, bool, cudaStream_t);
template void launch_update_E<double>(double *, const Grid &, double, bool, cudaStream_t);
template void launch_update_B<float>(float *, const Grid &, double, double, const Laser &, cudaStream_t);
template void launch_update_B<double>(double *, const Grid &, double, double, const Laser &, cudaStream_t);
template void launch_fold<float>(float *, const Grid &, cudaStream_t);
template void launch_fold<double>(double *, const Grid &, cudaStream_t);

}  // namespace pic
