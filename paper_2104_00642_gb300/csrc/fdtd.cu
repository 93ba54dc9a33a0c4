// fdtd.cu -- Yee FDTD half steps (Eqs. (9), (10) over dt/2), the Mur
// absorbing faces with the laser entering through x-min, and the current
// fold of the ghost layers.
//
// One thread per padded cell on a (x, y, z) thread grid, x fastest: rows are
// read and written with unit stride (coalesced) and no thread does integer
// division.  Each thread updates the three components of its cell.  Along
// periodic axes the ghost layers are computed directly (a neighbour that
// falls off the padded box is taken one period away), so they stay
// bit-identical copies of their images without a separate exchange.
//
// E update modes: a half step (dt/2), or the second half step of step n
// fused with the first half step of step n+1 -- both use the same curl B and
// the same J^{n+1}, applied twice in registers, which gives the same bits as
// two separate launches while reading and writing E once.
#include "fdtd.cuh"

namespace pic {

// offset of the neighbour one cell along axis d (dir = +1/-1) of the cell
// at padded coordinate p, taken one period away at the padded edge
__device__ __forceinline__ int nb_off(const Grid &g, int d, int p, int dir)
{
    int s = d == 0 ? 1 : (d == 1 ? (int)g.sy : (int)g.sz);
    int q = p + dir;
    if (q < -g.G[d]) q += g.n[d];
    else if (q >= g.n[d] + g.G[d]) q -= g.n[d];
    return (q - p) * s;
}

// per-thread masks: bit d of `half_ok` / `node_ok` = the coordinate along
// axis d lies in the physical half-node / node range (always on periodic or
// inactive axes); component c is updated when every axis agrees
struct Phys {
    int half_ok, node_ok;
    __device__ __forceinline__ bool comp(int c) const
    {
        int ok = 1;
#pragma unroll
        for (int d = 0; d < 3; d++) ok &= stag(c, d) ? (half_ok >> d) : (node_ok >> d);
        return ok & 1;
    }
};

__device__ __forceinline__ Phys phys_of(const Grid &g, int i, int j, int k)
{
    int p[3] = {i, j, k};
    Phys r{7, 7};
#pragma unroll
    for (int d = 0; d < 3; d++) {
        if (d >= g.dim || g.bc[d] == PERIODIC) continue;
        if (p[d] < 0 || p[d] > g.n[d] - 1) r.half_ok &= ~(1 << d);
        if (p[d] < 0 || p[d] > g.n[d]) r.node_ok &= ~(1 << d);
    }
    return r;
}

__device__ __forceinline__ bool thread_cell(const Grid &g, int &i, int &j, int &k)
{
    i = blockIdx.x * blockDim.x + threadIdx.x;
    j = blockIdx.y * blockDim.y + threadIdx.y;
    k = blockIdx.z;
    if (i >= g.ext[0] || j >= g.ext[1]) return false;
    i -= g.G[0];
    j -= g.G[1];
    k -= g.G[2];
    return true;
}

__device__ __forceinline__ int loff(const Grid &g, int i, int j, int k)
{
    return (int)g.origin + k * (int)g.sz + j * (int)g.sy + i;
}

// E += h (curl B - J), once (mode 0) or twice (mode 1); then J = 0 when
// zeroJ (J^n is no longer needed once the first half step of step n used it)
template <typename R, int DIM>
__global__ void __launch_bounds__(256) k_update_E(R *__restrict__ F, Grid g, R h, int twice, int zeroJ)
{
    int i, j, k;
    if (!thread_cell(g, i, j, k)) return;
    const int o = loff(g, i, j, k);
    const long long V = g.vol;
    const R *__restrict__ Bx = F + BX * V;
    const R *__restrict__ By = F + BY * V;
    const R *__restrict__ Bz = F + BZ * V;
    R *Ex = F + EX * V, *Ey = F + EY * V, *Ez = F + EZ * V;
    R *Jx = F + JX * V, *Jy = F + JY * V, *Jz = F + JZ * V;
    const R rdx = pic::rdx<R>(g, 0), rdy = pic::rdx<R>(g, 1), rdz = pic::rdx<R>(g, 2);
    R cx = 0, cy = 0, cz = 0;
    const int mx = nb_off(g, 0, i, -1);
    cy -= (Bz[o] - Bz[o + mx]) * rdx;
    cz += (By[o] - By[o + mx]) * rdx;
    if (DIM >= 2) {
        const int my = nb_off(g, 1, j, -1);
        cx += (Bz[o] - Bz[o + my]) * rdy;
        cz -= (Bx[o] - Bx[o + my]) * rdy;
    }
    if (DIM >= 3) {
        const int mz = nb_off(g, 2, k, -1);
        cx -= (By[o] - By[o + mz]) * rdz;
        cy += (Bx[o] - Bx[o + mz]) * rdz;
    }
    const R jx = Jx[o], jy = Jy[o], jz = Jz[o];
    const Phys ph = phys_of(g, i, j, k);
    const R ax = h * (cx - jx), ay = h * (cy - jy), az = h * (cz - jz);
    if (ph.comp(EX)) { R e = Ex[o] + ax; if (twice) e += ax; Ex[o] = e; }
    if (ph.comp(EY)) { R e = Ey[o] + ay; if (twice) e += ay; Ey[o] = e; }
    if (ph.comp(EZ)) { R e = Ez[o] + az; if (twice) e += az; Ez[o] = e; }
    if (zeroJ) { Jx[o] = 0; Jy[o] = 0; Jz[o] = 0; }
}

// incident B of the laser (a +x wave: Bz = Ey, By = -Ez) at time point q
// (see Laser); (j, k) are wrapped to the interior so that periodic ghost rows
// see the same laser as their images.  Rows outside the profile get none.
__device__ __forceinline__ float sin_r(float x) { return sinf(x); }
__device__ __forceinline__ double sin_r(double x) { return sin(x); }
__device__ __forceinline__ float cos_r(float x) { return cosf(x); }
__device__ __forceinline__ double cos_r(double x) { return cos(x); }

template <typename R>
__device__ inline R incident_B(const Grid &g, const Laser &L, int c, int q, int j, int k)
{
    if (g.dim >= 2 && g.bc[1] == PERIODIC) { j %= g.n[1]; if (j < 0) j += g.n[1]; }
    if (g.dim >= 3 && g.bc[2] == PERIODIC) { k %= g.n[2]; if (k < 0) k += g.n[2]; }
    if (g.dim < 2) j = 0;
    if (g.dim < 3) k = 0;
    if (j < 0 || j >= L.nty || k < 0 || k >= L.ntz) return R(0);
    const int t = k * L.nty + j;
    const R ph = (R)L.ph0[q];
    const R env = (R)L.env[q];
    if (c == BZ) {
        const R *A = (const R *)L.A[0], *P = (const R *)L.PHI[0];
        return A[t] * env * sin_r(ph + P[t]);
    }
    if (c == BY && L.pol == 1) {
        const R *A = (const R *)L.A[1], *P = (const R *)L.PHI[1];
        return -A[t] * env * cos_r(ph + P[t]);
    }
    return R(0);
}

// B -= h curl E, then the Mur ghosts of the tangential B on absorbing
// faces: for the scattered part s = B - B_inc of an outgoing wave,
// s_ghost(new) = s_inner(old) + (a-1)/(a+1) (s_inner(new) - s_ghost(old)),
// a = h/dx.  The thread owning the first inner value writes the ghost.
template <typename R, int DIM>
__global__ void __launch_bounds__(256) k_update_B(R *__restrict__ F, Grid g, R h, double t_new, Laser L)
{
    int i, j, k;
    if (!thread_cell(g, i, j, k)) return;
    const int o = loff(g, i, j, k);
    const long long V = g.vol;
    const R *__restrict__ Ex = F + EX * V;
    const R *__restrict__ Ey = F + EY * V;
    const R *__restrict__ Ez = F + EZ * V;
    R *B[3] = {F + BX * V, F + BY * V, F + BZ * V};
    const R rdx = pic::rdx<R>(g, 0), rdy = pic::rdx<R>(g, 1), rdz = pic::rdx<R>(g, 2);
    R cx = 0, cy = 0, cz = 0;
    const int px = nb_off(g, 0, i, +1);
    cy -= (Ez[o + px] - Ez[o]) * rdx;
    cz += (Ey[o + px] - Ey[o]) * rdx;
    if (DIM >= 2) {
        const int py = nb_off(g, 1, j, +1);
        cx += (Ez[o + py] - Ez[o]) * rdy;
        cz -= (Ex[o + py] - Ex[o]) * rdy;
    }
    if (DIM >= 3) {
        const int pz = nb_off(g, 2, k, +1);
        cx -= (Ey[o + pz] - Ey[o]) * rdz;
        cy += (Ex[o + pz] - Ex[o]) * rdz;
    }
    const R cur[3] = {cx, cy, cz};
    const Phys ph = phys_of(g, i, j, k);
    R oldv[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        oldv[c] = B[c][o];
        if (ph.comp(BX + c)) B[c][o] = oldv[c] - h * cur[c];
    }
    int p[3] = {i, j, k};
#pragma unroll
    for (int d = 0; d < DIM; d++) {
        if (g.bc[d] != ABSORB) continue;
        const bool lo = p[d] == 0, hi = p[d] == g.n[d] - 1;
        if (!lo && !hi) continue;
        // the transverse position must itself be a swept (updated) one
        bool ok = true;
#pragma unroll
        for (int e = 0; e < DIM; e++)
            if (e != d && g.bc[e] == ABSORB && (p[e] < 0 || p[e] > g.n[e])) ok = false;
        if (!ok) continue;
        const R a = h * pic::rdx<R>(g, d);
        const R c1 = (a - R(1)) / (a + R(1));
        const int s = d == 0 ? 1 : (d == 1 ? (int)g.sy : (int)g.sz);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            if (!stag(BX + c, d)) continue;
            for (int face = 0; face < 2; face++) {
                if ((face == 0 && !lo) || (face == 1 && !hi)) continue;
                const int og = o + (face == 0 ? -s : s);
                R ig_new = 0, ig_old = 0, ii_new = 0, ii_old = 0;
                if (face == 0 && d == 0 && L.on) {
                    ig_new = incident_B<R>(g, L, BX + c, 0, j, k);
                    ig_old = incident_B<R>(g, L, BX + c, 1, j, k);
                    ii_new = incident_B<R>(g, L, BX + c, 2, j, k);
                    ii_old = incident_B<R>(g, L, BX + c, 3, j, k);
                }
                const R sg_old = B[c][og] - ig_old;
                const R si_old = oldv[c] - ii_old;
                const R si_new = B[c][o] - ii_new;
                B[c][og] = ig_new + si_old + c1 * (si_new - sg_old);
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

// thread grid over the padded box with axis d replaced by its 2G shell
__device__ __forceinline__ bool shell_cell(const Grid &g, int d, int *p)
{
    int e[3] = {g.ext[0], g.ext[1], g.ext[2]};
    e[d] = 2 * g.G[d];
    p[0] = blockIdx.x * blockDim.x + threadIdx.x;
    p[1] = blockIdx.y * blockDim.y + threadIdx.y;
    p[2] = blockIdx.z;
    if (p[0] >= e[0] || p[1] >= e[1]) return false;
    for (int a = 0; a < 3; a++) p[a] -= (a == d) ? 0 : g.G[a];
    return true;
}

// periodic fold along axis d: what was deposited into a ghost belongs to
// its image; both end up holding the sum (image + ghost, fixed order)
template <typename R>
__global__ void k_fold_periodic(R *__restrict__ base, FoldSet fs, Grid g, int d)
{
    int p[3];
    if (!shell_cell(g, d, p)) return;
    const int G = g.G[d], N = g.n[d];
    const int s = p[d];
    const int in = s < G ? s : N - 2 * G + s;
    const int partner = in < G ? in + N : in - N;
    p[d] = in;
    const long long oi = goff(g, p[0], p[1], p[2]);
    p[d] = partner;
    const long long op = goff(g, p[0], p[1], p[2]);
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
    int p[3];
    if (!shell_cell(g, d, p)) return;
    const int G = g.G[d], N = g.n[d];
    const int s = p[d];
    p[d] = s < G ? s - G : N + (s - G);  // [-G,0) and [N, N+G)
    const long long o = goff(g, p[0], p[1], p[2]);
    for (int q = 0; q < fs.ncomp; q++) {
        int hi = ((fs.mask[q] >> d) & 1) ? N - 1 : N;
        if (p[d] < 0 || p[d] > hi) base[q * fs.stride + o] = 0;
    }
}

// ---------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------

static void grid_dims(const Grid &g, int e0, int e1, int e2, dim3 &blk, dim3 &grd)
{
    if (g.dim == 1) blk = dim3(256, 1, 1);
    else blk = dim3(64, 4, 1);
    grd = dim3((unsigned)div_up(e0, blk.x), (unsigned)div_up(e1, blk.y), (unsigned)e2);
}

template <typename R>
void launch_update_E(R *F, const Grid &g, double h, bool twice, bool zeroJ, cudaStream_t st)
{
    dim3 b, n;
    grid_dims(g, g.ext[0], g.ext[1], g.ext[2], b, n);
    note_launch();
    if (g.dim == 1) k_update_E<R, 1><<<n, b, 0, st>>>(F, g, (R)h, twice, zeroJ);
    else if (g.dim == 2) k_update_E<R, 2><<<n, b, 0, st>>>(F, g, (R)h, twice, zeroJ);
    else k_update_E<R, 3><<<n, b, 0, st>>>(F, g, (R)h, twice, zeroJ);
}

template <typename R>
void launch_update_B(R *F, const Grid &g, double h, double t_new, const Laser &L, cudaStream_t st)
{
    dim3 b, n;
    grid_dims(g, g.ext[0], g.ext[1], g.ext[2], b, n);
    note_launch();
    if (g.dim == 1) k_update_B<R, 1><<<n, b, 0, st>>>(F, g, (R)h, t_new, L);
    else if (g.dim == 2) k_update_B<R, 2><<<n, b, 0, st>>>(F, g, (R)h, t_new, L);
    else k_update_B<R, 3><<<n, b, 0, st>>>(F, g, (R)h, t_new, L);
}

template <typename R>
void launch_fold_set(R *base, const FoldSet &fs, const Grid &g, cudaStream_t st)
{
    for (int d = 0; d < g.dim; d++) {
        int e[3] = {g.ext[0], g.ext[1], g.ext[2]};
        e[d] = 2 * g.G[d];
        dim3 b, n;
        grid_dims(g, e[0], e[1], e[2], b, n);
        note_launch();
        if (g.bc[d] == PERIODIC) k_fold_periodic<R><<<n, b, 0, st>>>(base, fs, g, d);
        else k_discard_absorb<R><<<n, b, 0, st>>>(base, fs, g, d);
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

template void launch_update_E<float>(float *, const Grid &, double, bool, bool, cudaStream_t);
template void launch_update_E<double>(double *, const Grid &, double, bool, bool, cudaStream_t);
template void launch_update_B<float>(float *, const Grid &, double, double, const Laser &, cudaStream_t);
template void launch_update_B<double>(double *, const Grid &, double, double, const Laser &, cudaStream_t);
template void launch_fold<float>(float *, const Grid &, cudaStream_t);
template void launch_fold<double>(double *, const Grid &, cudaStream_t);

}  // namespace pic
