// diag.cu -- FP64 diagnostics: field energy, kinetic energy per species,
// live counts, the particle charge density averaged over the two half-step
// positions that bracket the integer step, and the Gauss residual
// max |div E - rho - rho_bg| (Eq. (1) in the units of Eq. (8)).
//
// Sums use a fixed reduction tree: a fixed grid of blocks, each reducing a
// fixed strided set of elements in a fixed shuffle order into one partial,
// then one block summing the partials in index order, so results do not
// depend on scheduling.
#include "diag.cuh"
#include "push_dev.cuh"

namespace pic {

constexpr int kRedBlocks = 1024;
constexpr int kRedThreads = 256;

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// NV values per thread reduced to partial[blockIdx.x * NV + q]
template <int NV, bool MAX>
__device__ __forceinline__ void block_reduce_store(double *v, double *partial)
{
    __shared__ double sh[NV][kRedThreads / 32];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; q++) {
        double x = MAX ? warp_max(v[q]) : warp_sum(v[q]);
        if (lane == 0) sh[q][warp] = x;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
#pragma unroll
        for (int q = 0; q < NV; q++) {
            double x = lane < kRedThreads / 32 ? sh[q][lane] : (MAX ? 0.0 : 0.0);
            x = MAX ? warp_max(x) : warp_sum(x);
            if (lane == 0) partial[blockIdx.x * NV + q] = x;
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(kRedThreads) k_field_energy(const R *__restrict__ F, Grid g, double *partial)
{
    long long tot = (long long)g.n[0] * g.n[1] * g.n[2];
    double v[2] = {0.0, 0.0};
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < tot;
         t += (long long)gridDim.x * blockDim.x) {
        int i = (int)(t % g.n[0]);
        long long r = t / g.n[0];
        int j = (int)(r % g.n[1]);
        int k = (int)(r / g.n[1]);
        long long o = goff(g, i, j, k);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            double e = (double)F[(EX + c) * g.vol + o], b = (double)F[(BX + c) * g.vol + o];
            v[0] += e * e;
            v[1] += b * b;
        }
    }
    block_reduce_store<2, false>(v, partial);
}

// sum of (gamma - 1) = u^2 / (gamma + 1) per particle, or of |k| for photons
__global__ void __launch_bounds__(kRedThreads) k_kinetic_f32(PartF32 P, int photon, double *partial)
{
    double v[2] = {0.0, 0.0};
    long long n = *P.dn;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        if (P.cell[p] == kDead) continue;
        double ux = P.u[0][p], uy = P.u[1][p], uz = P.u[2][p];
        double uu = ux * ux + uy * uy + uz * uz;
        v[0] += photon ? sqrt(uu) : uu / (sqrt(1.0 + uu) + 1.0);
        v[1] += 1.0;
    }
    block_reduce_store<2, false>(v, partial);
}

__global__ void __launch_bounds__(kRedThreads) k_kinetic_f64(PartF64 P, int photon, double *partial)
{
    double v[2] = {0.0, 0.0};
    long long n = *P.dn;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        if (P.cell[p] == kDead) continue;
        double ux = P.u[0][p], uy = P.u[1][p], uz = P.u[2][p];
        double uu = ux * ux + uy * uy + uz * uz;
        v[0] += photon ? sqrt(uu) : uu / (sqrt(1.0 + uu) + 1.0);
        v[1] += 1.0;
    }
    block_reduce_store<2, false>(v, partial);
}

// sums partial[b*NV + q] over b in index order (one block, fixed tree)
template <int NV, bool MAX>
__global__ void __launch_bounds__(kRedThreads) k_final(const double *__restrict__ partial, int nparts, double *out)
{
    double v[NV];
#pragma unroll
    for (int q = 0; q < NV; q++) v[q] = 0.0;
    for (int b = threadIdx.x; b < nparts; b += blockDim.x)
#pragma unroll
        for (int q = 0; q < NV; q++) v[q] = MAX ? fmax(v[q], partial[b * NV + q]) : v[q] + partial[b * NV + q];
    __shared__ double sh[NV][kRedThreads / 32];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; q++) {
        double x = MAX ? warp_max(v[q]) : warp_sum(v[q]);
        if (lane == 0) sh[q][warp] = x;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
#pragma unroll
        for (int q = 0; q < NV; q++) {
            double x = lane < kRedThreads / 32 ? sh[q][lane] : 0.0;
            x = MAX ? warp_max(x) : warp_sum(x);
            if (lane == 0) out[q] = x;
        }
    }
}

// charge density of one species: q w W (W_2 or W_4, the shape the deposit
// uses) at x -/+ (dt/2) v, half each
template <int DIM, int ORDER>
__device__ __forceinline__ void rho_add(double *rho, const Grid &g, const double *X, double qw2)
{
    constexpr int P = ORDER + 1, H = ORDER / 2;
    // a non-finite position has no node; the pushes remove particles whose
    // momentum became non-finite, so this only guards the index arithmetic
#pragma unroll
    for (int d = 0; d < DIM; d++)
        if (!isfinite(X[d])) return;
    int ic[3] = {0, 0, 0};
    double w[3][P];
#pragma unroll
    for (int d = 0; d < 3; d++) {
        if (d < DIM) {
            ic[d] = (int)floor(X[d] + 0.5);
            if constexpr (ORDER == 4) w4<double>(X[d] - (double)ic[d], w[d]);
            else w2<double>(X[d] - (double)ic[d], w[d]);
        } else {
#pragma unroll
            for (int a = 0; a < P; a++) w[d][a] = a == H ? 1.0 : 0.0;
        }
    }
#pragma unroll
    for (int c = 0; c < (DIM > 2 ? P : 1); c++)
#pragma unroll
        for (int b = 0; b < (DIM > 1 ? P : 1); b++)
#pragma unroll
            for (int a = 0; a < P; a++) {
                int jb = DIM > 1 ? b : H, kc = DIM > 2 ? c : H;
                double wt = w[0][a] * w[1][jb] * w[2][kc];
                atomicAdd(rho + goff(g, ic[0] + a - H, DIM > 1 ? ic[1] + b - H : 0, DIM > 2 ? ic[2] + c - H : 0),
                          qw2 * wt);
            }
}

template <int DIM, int ORDER>
__global__ void k_rho_f32(PartF32 P, Grid g, double hdt, double qw2, double *rho)
{
    long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= *P.dn) return;
    uint32_t cp = P.cell[p];
    if (cp == kDead) return;
    int c[3];
    unpack_cell(g, cp, c[0], c[1], c[2]);
    double ux = P.u[0][p], uy = P.u[1][p], uz = P.u[2][p];
    double ig = 1.0 / sqrt(1.0 + ux * ux + uy * uy + uz * uz);
    double u[3] = {ux, uy, uz};
    for (int side = -1; side <= 1; side += 2) {
        double X[3] = {0, 0, 0};
        for (int d = 0; d < DIM; d++) X[d] = (double)c[d] + (double)P.off[d][p] + side * hdt * u[d] * ig / g.dx[d];
        rho_add<DIM, ORDER>(rho, g, X, qw2);
    }
}

template <int DIM, int ORDER>
__global__ void k_rho_f64(PartF64 P, Grid g, double hdt, double qw2, double *rho)
{
    long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= *P.dn) return;
    if (P.cell[p] == kDead) return;
    double ux = P.u[0][p], uy = P.u[1][p], uz = P.u[2][p];
    double ig = 1.0 / sqrt(1.0 + ux * ux + uy * uy + uz * uz);
    double u[3] = {ux, uy, uz};
    for (int side = -1; side <= 1; side += 2) {
        double X[3] = {0, 0, 0};
        for (int d = 0; d < DIM; d++) X[d] = (P.x[d][p] + side * hdt * u[d] * ig) / g.dx[d];
        rho_add<DIM, ORDER>(rho, g, X, qw2);
    }
}

// max over interior nodes of |div E - rho - rho_bg|
template <typename R>
__global__ void __launch_bounds__(kRedThreads) k_gauss(const R *__restrict__ F, const double *__restrict__ rho, Grid g,
                                                       double rho_bg, double *partial)
{
    long long tot = (long long)g.n[0] * g.n[1] * g.n[2];
    double v[1] = {0.0};
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < tot;
         t += (long long)gridDim.x * blockDim.x) {
        int i = (int)(t % g.n[0]);
        long long r = t / g.n[0];
        int j = (int)(r % g.n[1]);
        int k = (int)(r / g.n[1]);
        long long o = goff(g, i, j, k);
        const R *Ex = F + EX * g.vol, *Ey = F + EY * g.vol, *Ez = F + EZ * g.vol;
        double div = ((double)Ex[o] - (double)Ex[o - 1]) / g.dx[0];
        if (g.dim > 1) div += ((double)Ey[o] - (double)Ey[o - g.sy]) / g.dx[1];
        if (g.dim > 2) div += ((double)Ez[o] - (double)Ez[o - g.sz]) / g.dx[2];
        v[0] = fmax(v[0], fabs(div - rho[o] - rho_bg));
    }
    block_reduce_store<1, true>(v, partial);
}

// ---------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------
size_t diag_scratch_doubles() { return (size_t)kRedBlocks * 4 + 64; }

template <typename R>
void diag_field_energy(const R *F, const Grid &g, double *scratch, double *out2, cudaStream_t st)
{
    k_field_energy<R><<<kRedBlocks, kRedThreads, 0, st>>>(F, g, scratch);
    k_final<2, false><<<1, kRedThreads, 0, st>>>(scratch, kRedBlocks, out2);
}
template void diag_field_energy<float>(const float *, const Grid &, double *, double *, cudaStream_t);
template void diag_field_energy<double>(const double *, const Grid &, double *, double *, cudaStream_t);

void diag_kinetic_f32(const PartF32 &P, bool photon, double *scratch, double *out2, cudaStream_t st)
{
    k_kinetic_f32<<<kRedBlocks, kRedThreads, 0, st>>>(P, photon ? 1 : 0, scratch);
    k_final<2, false><<<1, kRedThreads, 0, st>>>(scratch, kRedBlocks, out2);
}
void diag_kinetic_f64(const PartF64 &P, bool photon, double *scratch, double *out2, cudaStream_t st)
{
    k_kinetic_f64<<<kRedBlocks, kRedThreads, 0, st>>>(P, photon ? 1 : 0, scratch);
    k_final<2, false><<<1, kRedThreads, 0, st>>>(scratch, kRedBlocks, out2);
}

void diag_rho_f32(const PartF32 &P, const Grid &g, double qw, double *rho, cudaStream_t st)
{
    if (P.n == 0) return;
    int nb = div_up(P.n, 256);
    double h = 0.5 * g.dt;
    if (g.order == 4) {
        if (g.dim == 1) k_rho_f32<1, 4><<<nb, 256, 0, st>>>(P, g, h, 0.5 * qw, rho);
        else if (g.dim == 2) k_rho_f32<2, 4><<<nb, 256, 0, st>>>(P, g, h, 0.5 * qw, rho);
        else k_rho_f32<3, 4><<<nb, 256, 0, st>>>(P, g, h, 0.5 * qw, rho);
        return;
    }
    if (g.dim == 1) k_rho_f32<1, 2><<<nb, 256, 0, st>>>(P, g, h, 0.5 * qw, rho);
    else if (g.dim == 2) k_rho_f32<2, 2><<<nb, 256, 0, st>>>(P, g, h, 0.5 * qw, rho);
    else k_rho_f32<3, 2><<<nb, 256, 0, st>>>(P, g, h, 0.5 * qw, rho);
}
void diag_rho_f64(const PartF64 &P, const Grid &g, double qw, double *rho, cudaStream_t st)
{
    if (P.n == 0) return;
    int nb = div_up(P.n, 256);
    double h = 0.5 * g.dt;
    if (g.order == 4) {
        if (g.dim == 1) k_rho_f64<1, 4><<<nb, 256, 0, st>>>(P, g, h, 0.5 * qw, rho);
        else if (g.dim == 2) k_rho_f64<2, 4><<<nb, 256, 0, st>>>(P, g, h, 0.5 * qw, rho);
        else k_rho_f64<3, 4><<<nb, 256, 0, st>>>(P, g, h, 0.5 * qw, rho);
        return;
    }
    if (g.dim == 1) k_rho_f64<1, 2><<<nb, 256, 0, st>>>(P, g, h, 0.5 * qw, rho);
    else if (g.dim == 2) k_rho_f64<2, 2><<<nb, 256, 0, st>>>(P, g, h, 0.5 * qw, rho);
    else k_rho_f64<3, 2><<<nb, 256, 0, st>>>(P, g, h, 0.5 * qw, rho);
}

template <typename R>
void diag_gauss(const R *F, const double *rho, const Grid &g, double rho_bg, double *scratch, double *out1,
                cudaStream_t st)
{
    k_gauss<R><<<kRedBlocks, kRedThreads, 0, st>>>(F, rho, g, rho_bg, scratch);
    k_final<1, true><<<1, kRedThreads, 0, st>>>(scratch, kRedBlocks, out1);
}
template void diag_gauss<float>(const float *, const double *, const Grid &, double, double *, double *, cudaStream_t);
template void diag_gauss<double>(const double *, const double *, const Grid &, double, double *, double *,
                                 cudaStream_t);

}  // namespace pic
