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

template <typename R, int DIM>
__device__ __forceinline__ void mur_faces(R *const *B, const Grid &g, R h, const Laser &L, int i, int j, int k, int o,
                                          const R *oldv);

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
    mur_faces<R, DIM>(B, g, h, L, i, j, k, o, oldv);
}

// the Mur ghosts of cell (i, j, k) at offset o, after its B update (oldv:
// its B before the update)
template <typename R, int DIM>
__device__ __forceinline__ void mur_faces(R *const *B, const Grid &g, R h, const Laser &L, int i, int j, int k, int o,
                                          const R *oldv)
{
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

// ---------------------------------------------------------------------
// FP32, four cells per thread along x (float4 loads and stores; the padded
// rows start 16-byte aligned and hold a multiple of 4 cells when n_x is a
// multiple of 4).  Same arithmetic, in the same order, as the one-cell
// kernels above.  A component is stored as a vector when all four cells are
// physical for it, else cell by cell (ghost cells on absorbing axes belong
// to the Mur update).
// ---------------------------------------------------------------------
__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void st4(float *p, const float (&v)[4])
{
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void unpack4(const float4 &a, float (&v)[4])
{
    v[0] = a.x;
    v[1] = a.y;
    v[2] = a.z;
    v[3] = a.w;
}

__device__ __forceinline__ bool thread_cell4(const Grid &g, int &i, int &j, int &k)
{
    i = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    j = blockIdx.y * blockDim.y + threadIdx.y;
    k = blockIdx.z;
    if (i >= g.ext[0] || j >= g.ext[1]) return false;
    i -= g.G[0];
    j -= g.G[1];
    k -= g.G[2];
    return true;
}

__device__ __forceinline__ void store_phys(float *A, int o, const float (&v)[4], const Phys (&ph)[4], int c)
{
    const bool all = ph[0].comp(c) && ph[1].comp(c) && ph[2].comp(c) && ph[3].comp(c);
    if (all) {
        st4(A + o, v);
    } else {
#pragma unroll
        for (int e = 0; e < 4; e++)
            if (ph[e].comp(c)) A[o + e] = v[e];
    }
}

template <int DIM>
__global__ void __launch_bounds__(256) k_update_E4(float *__restrict__ F, Grid g, float h, int twice, int zeroJ)
{
    int i, j, k;
    if (!thread_cell4(g, i, j, k)) return;
    const int o = loff(g, i, j, k);
    const long long V = g.vol;
    const float *__restrict__ Bx = F + BX * V;
    const float *__restrict__ By = F + BY * V;
    const float *__restrict__ Bz = F + BZ * V;
    float *E[3] = {F + EX * V, F + EY * V, F + EZ * V};
    float *J[3] = {F + JX * V, F + JY * V, F + JZ * V};
    const float rdx = g.rdx_f[0], rdy = g.rdx_f[1], rdz = g.rdx_f[2];
    float bz[4], by[4];
    unpack4(ld4(Bz + o), bz);
    unpack4(ld4(By + o), by);
    const int mx = nb_off(g, 0, i, -1);
    const float bzl = Bz[o + mx], byl = By[o + mx];
    float cx[4] = {0.f, 0.f, 0.f, 0.f}, cy[4] = {0.f, 0.f, 0.f, 0.f}, cz[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int e = 0; e < 4; e++) {
        cy[e] -= (bz[e] - (e ? bz[e - 1] : bzl)) * rdx;
        cz[e] += (by[e] - (e ? by[e - 1] : byl)) * rdx;
    }
    float bx[4];
    if (DIM >= 2) {
        const int my = nb_off(g, 1, j, -1);
        float bzm[4], bxm[4];
        unpack4(ld4(Bx + o), bx);
        unpack4(ld4(Bz + o + my), bzm);
        unpack4(ld4(Bx + o + my), bxm);
#pragma unroll
        for (int e = 0; e < 4; e++) {
            cx[e] += (bz[e] - bzm[e]) * rdy;
            cz[e] -= (bx[e] - bxm[e]) * rdy;
        }
    }
    if (DIM >= 3) {
        const int mz = nb_off(g, 2, k, -1);
        float bym[4], bxm[4];
        unpack4(ld4(By + o + mz), bym);
        unpack4(ld4(Bx + o + mz), bxm);
#pragma unroll
        for (int e = 0; e < 4; e++) {
            cx[e] -= (by[e] - bym[e]) * rdz;
            cy[e] += (bx[e] - bxm[e]) * rdz;
        }
    }
    Phys ph[4];
#pragma unroll
    for (int e = 0; e < 4; e++) ph[e] = phys_of(g, i + e, j, k);
    const float *cur[3] = {cx, cy, cz};
#pragma unroll
    for (int c = 0; c < 3; c++) {
        float jv[4], ev[4];
        unpack4(ld4(J[c] + o), jv);
        unpack4(ld4(E[c] + o), ev);
#pragma unroll
        for (int e = 0; e < 4; e++) {
            const float a = h * (cur[c][e] - jv[e]);
            ev[e] += a;
            if (twice) ev[e] += a;
        }
        store_phys(E[c], o, ev, ph, EX + c);
    }
    if (zeroJ) {
        const float z[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int c = 0; c < 3; c++) st4(J[c] + o, z);
    }
}

template <int DIM>
__global__ void __launch_bounds__(256) k_update_B4(float *__restrict__ F, Grid g, float h, Laser L)
{
    int i, j, k;
    if (!thread_cell4(g, i, j, k)) return;
    const int o = loff(g, i, j, k);
    const long long V = g.vol;
    const float *__restrict__ Ex = F + EX * V;
    const float *__restrict__ Ey = F + EY * V;
    const float *__restrict__ Ez = F + EZ * V;
    float *B[3] = {F + BX * V, F + BY * V, F + BZ * V};
    const float rdx = g.rdx_f[0], rdy = g.rdx_f[1], rdz = g.rdx_f[2];
    float ez[4], ey[4];
    unpack4(ld4(Ez + o), ez);
    unpack4(ld4(Ey + o), ey);
    const int px = nb_off(g, 0, i + 3, +1);
    const float ezr = Ez[o + 3 + px], eyr = Ey[o + 3 + px];
    float cx[4] = {0.f, 0.f, 0.f, 0.f}, cy[4] = {0.f, 0.f, 0.f, 0.f}, cz[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int e = 0; e < 4; e++) {
        cy[e] -= ((e < 3 ? ez[e + 1] : ezr) - ez[e]) * rdx;
        cz[e] += ((e < 3 ? ey[e + 1] : eyr) - ey[e]) * rdx;
    }
    float ex[4];
    if (DIM >= 2) {
        const int py = nb_off(g, 1, j, +1);
        float ezp[4], exp_[4];
        unpack4(ld4(Ex + o), ex);
        unpack4(ld4(Ez + o + py), ezp);
        unpack4(ld4(Ex + o + py), exp_);
#pragma unroll
        for (int e = 0; e < 4; e++) {
            cx[e] += (ezp[e] - ez[e]) * rdy;
            cz[e] -= (exp_[e] - ex[e]) * rdy;
        }
    }
    if (DIM >= 3) {
        const int pz = nb_off(g, 2, k, +1);
        float eyp[4], exp_[4];
        unpack4(ld4(Ey + o + pz), eyp);
        unpack4(ld4(Ex + o + pz), exp_);
#pragma unroll
        for (int e = 0; e < 4; e++) {
            cx[e] -= (eyp[e] - ey[e]) * rdz;
            cy[e] += (exp_[e] - ex[e]) * rdz;
        }
    }
    Phys ph[4];
#pragma unroll
    for (int e = 0; e < 4; e++) ph[e] = phys_of(g, i + e, j, k);
    const float *cur[3] = {cx, cy, cz};
    float oldv[3][4];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        float nv[4];
        unpack4(ld4(B[c] + o), oldv[c]);
#pragma unroll
        for (int e = 0; e < 4; e++) nv[e] = oldv[c][e] - h * cur[c][e];
        store_phys(B[c], o, nv, ph, BX + c);
    }
    // Mur ghosts: only groups that touch an absorbing face
    bool face = false;
#pragma unroll
    for (int d = 0; d < DIM; d++) {
        if (g.bc[d] != ABSORB) continue;
        const int lo = d == 0 ? i : (d == 1 ? j : k), hi = d == 0 ? i + 3 : lo;
        face |= (lo <= 0 && hi >= 0) || (lo <= g.n[d] - 1 && hi >= g.n[d] - 1);
    }
    if (face) {
#pragma unroll
        for (int e = 0; e < 4; e++) {
            const float ov[3] = {oldv[0][e], oldv[1][e], oldv[2][e]};
            mur_faces<float, DIM>(B, g, h, L, i + e, j, k, o + e, ov);
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

static bool vec4_ok(const Grid &g) { return g.n[0] % 4 == 0 && g.G[0] % 4 == 0; }

template <typename R>
void launch_update_E(R *F, const Grid &g, double h, bool twice, bool zeroJ, cudaStream_t st)
{
    dim3 b, n;
    note_launch();
    if constexpr (sizeof(R) == 4) {
        if (vec4_ok(g)) {
            grid_dims(g, g.ext[0] / 4, g.ext[1], g.ext[2], b, n);
            if (g.dim == 1) k_update_E4<1><<<n, b, 0, st>>>(F, g, (float)h, twice, zeroJ);
            else if (g.dim == 2) k_update_E4<2><<<n, b, 0, st>>>(F, g, (float)h, twice, zeroJ);
            else k_update_E4<3><<<n, b, 0, st>>>(F, g, (float)h, twice, zeroJ);
            return;
        }
    }
    grid_dims(g, g.ext[0], g.ext[1], g.ext[2], b, n);
    if (g.dim == 1) k_update_E<R, 1><<<n, b, 0, st>>>(F, g, (R)h, twice, zeroJ);
    else if (g.dim == 2) k_update_E<R, 2><<<n, b, 0, st>>>(F, g, (R)h, twice, zeroJ);
    else k_update_E<R, 3><<<n, b, 0, st>>>(F, g, (R)h, twice, zeroJ);
}

template <typename R>
void launch_update_B(R *F, const Grid &g, double h, double t_new, const Laser &L, cudaStream_t st)
{
    dim3 b, n;
    note_launch();
    if constexpr (sizeof(R) == 4) {
        if (vec4_ok(g)) {
            grid_dims(g, g.ext[0] / 4, g.ext[1], g.ext[2], b, n);
            if (g.dim == 1) k_update_B4<1><<<n, b, 0, st>>>(F, g, (float)h, L);
            else if (g.dim == 2) k_update_B4<2><<<n, b, 0, st>>>(F, g, (float)h, L);
            else k_update_B4<3><<<n, b, 0, st>>>(F, g, (float)h, L);
            return;
        }
    }
    grid_dims(g, g.ext[0], g.ext[1], g.ext[2], b, n);
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
