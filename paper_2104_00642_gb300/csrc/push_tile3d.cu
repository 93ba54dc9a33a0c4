// push_tile3d.cu -- tiled particle push for 3D grids (FP32 cell+offset
// form): the scheme of push_tile.cu with a 3D box.
#include <algorithm>
#include <cstring>

#include "push_qed_dev.cuh"
#include "push_tile_dev.cuh"
#include "tma.cuh"

namespace pic {

// ---------------------------------------------------------------------
// 3D: tiles of T^3 cells, the same scheme with a 3D box
//   x: [t0-4, t0+T+4) (float4-aligned rows), y and z: [t0-3, t0+T+3);
// the box of a tile that touches the domain edge stays inside the padded
// field box (ghost layers of 4), so staging and flush need no edge tests.
// Consecutive lanes take consecutive particles of an item (coalesced loads
// of the particle state, which is not staged in 3D).
// ---------------------------------------------------------------------
template <int T>
struct Box3 {
    static constexpr int WX = T + 8, WY = T + 6, WZ = T + 6;
    static constexpr int RS = WX, PS = WX * WY, N = WX * WY * WZ;
    static constexpr int SMEM = 9 * N * (int)sizeof(float);  // fields (6) + current (3)
};

// element k of a small register array without dynamic indexing (selects)
__device__ __forceinline__ float sel3(const float *v, int k) { return k == 0 ? v[0] : (k == 1 ? v[1] : v[2]); }
__device__ __forceinline__ float sel4(const float *v, int k)
{
    return k == 0 ? v[0] : (k == 1 ? v[1] : (k == 2 ? v[2] : v[3]));
}

// Eq. (19) in 3D on the shared box.  The z loop is kept rolled: the 3D push
// body is large, and a fully unrolled one stalls on instruction fetch.
template <int T>
__device__ __forceinline__ void gather3d_box(const float *__restrict__ P, const int *o0, const int *icn,
                                             const float (*wn)[3], const int *ich, const float (*wh)[3], float *eb)
{
    using B = Box3<T>;
#pragma unroll
    for (int c = 0; c < 6; c++) {
        const int sx = stag(c, 0), sy = stag(c, 1), sz = stag(c, 2);
        const int ix = (sx ? ich[0] : icn[0]) - 1 - o0[0];
        const int iy = (sy ? ich[1] : icn[1]) - 1 - o0[1];
        const int iz = (sz ? ich[2] : icn[2]) - 1 - o0[2];
        const float *wx = sx ? wh[0] : wn[0];
        const float *wy = sy ? wh[1] : wn[1];
        const float *wz = sz ? wh[2] : wn[2];
        const float *q = P + c * B::N + iz * B::PS + iy * B::RS + ix;
        float acc = 0.f;
#pragma unroll 1
        for (int cz = 0; cz < 3; cz++) {
            float sb = 0.f;
#pragma unroll
            for (int b = 0; b < 3; b++) {
                const float *r = q + cz * B::PS + b * B::RS;
                float s = wx[0] * r[0];
                s += wx[1] * r[1];
                s += wx[2] * r[2];
                sb += wy[b] * s;
            }
            acc += sel3(wz, cz) * sb;
        }
        eb[c] = acc;
    }
}

// Esirkepov in 3D on the union window (Eqs. (20)-(22)): W_x = dSx (ty tz +
// dSy dSz / 12) with t = S0 + dS/2 (= S0y S0z + (dSy S0z + S0y dSz)/2 +
// dSy dSz/3), cyclic for y and z; J_d is cJ_d times the prefix sum of W_d
// along d (three nonzero nodes of the four).  Shared int32 fixed point.
template <int T>
__device__ __forceinline__ void esirkepov3d_box(int *base, const float (*S0)[4], const float (*dS)[4], float cjx,
                                                float cjy, float cjz, float scale)
{
    using B = Box3<T>;
    float t[3][4], p[3][3];
#pragma unroll
    for (int d = 0; d < 3; d++) {
#pragma unroll
        for (int k = 0; k < 4; k++) t[d][k] = S0[d][k] + 0.5f * dS[d][k];
        p[d][0] = dS[d][0];
        p[d][1] = p[d][0] + dS[d][1];
        p[d][2] = p[d][1] + dS[d][2];
    }
    const float cj[3] = {cjx * scale, cjy * scale, cjz * scale};
    const float r12 = 1.0f / 12.0f;
    // the outermost loop of each component stays rolled (code size, as in
    // gather3d_box); its index picks the z (or y) shape by selects
#pragma unroll 1
    for (int c = 0; c < 4; c++) {
        const float tzc = sel4(t[2], c), dzc = sel4(dS[2], c) * r12;
        int *bc = base + c * B::PS;
#pragma unroll
        for (int b = 0; b < 4; b++) {
            const float wx = fmaf(t[1][b], tzc, dS[1][b] * dzc) * cj[0];
#pragma unroll
            for (int a = 0; a < 3; a++) atomicAdd(bc + b * B::RS + a, __float2int_rn(p[0][a] * wx));
        }
#pragma unroll
        for (int a = 0; a < 4; a++) {
            const float wy = fmaf(t[0][a], tzc, dS[0][a] * dzc) * cj[1];
#pragma unroll
            for (int b = 0; b < 3; b++) atomicAdd(bc + B::N + b * B::RS + a, __float2int_rn(p[1][b] * wy));
        }
    }
#pragma unroll 1
    for (int b = 0; b < 4; b++) {
        const float tyb = sel4(t[1], b), dyb = sel4(dS[1], b) * r12;
        int *bb = base + 2 * B::N + b * B::RS;
#pragma unroll
        for (int a = 0; a < 4; a++) {
            const float wz = fmaf(t[0][a], tyb, dS[0][a] * dyb) * cj[2];
#pragma unroll
            for (int c = 0; c < 3; c++) atomicAdd(bb + c * B::PS + a, __float2int_rn(p[2][c] * wz));
        }
    }
}

// the QED variants' slow paths, out of line (rare: a particle that drifted
// out of its tile's box since the sort): the gather from HBM and the
// deposit with global atomics on the 5-node window
static __device__ __noinline__ void gather3d_global(const float *F, const Grid &g, const int *icn,
                                                   const float (*wn)[3], const int *ich, const float (*wh)[3],
                                                   float *eb)
{
    gather<float, 3>(F, g, icn, wn, ich, wh, eb);
}

static __device__ __noinline__ bool deposit3d_global(float *F, const Grid &g, const PushConst &pc, const int *ch,
                                                     const float *oh, const int *c, const float *o, float uy,
                                                     float uz, float ig1)
{
    float S0[3][5], dS[3][5];
    int base[3];
    bool ok = true;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        int i0, i1;
        float w0[3], w1[3];
        axis_wn_f32(ch[d], oh[d], i0, w0);
        axis_wn_f32(c[d], o[d], i1, w1);
        ok &= window5<float>(i0, w0, i1, w1, S0[d], dS[d]);
        base[d] = i0 - 2;
    }
    if (!ok) return false;
    const float cJ[3] = {pc.cJ_f[0], pc.cJ_f[1], pc.cJ_f[2]};
    deposit_global<float, 3>(F, g, base, S0, dS, cJ, pc.qw_f * uy * ig1, pc.qw_f * uz * ig1);
    return true;
}

// A particle whose stencil leaves its tile's box (it drifted since the sort)
// is not pushed here (QM == 0): its index goes to a list, and the list is
// pushed afterwards on the global path (launch_push_list_f32).  Nothing of
// the particle is written before that decision, and a warp never waits on
// one lane's slow path.
//
// QM (QED leptons): 1 = the Monte Carlo of Sec. IV with the tables, 2 = with
// the surrogate network (its image after the boxes), as in the 2D kernel;
// a particle whose stencil left the box takes the global gather and deposit
// in place (its optical depth has moved on).  Particles are taken in
// block-wide passes so that the network's warp-collective evaluation sees
// every lane; the event flag of every particle of the items is written.
template <int T, int QM>
__global__ void __launch_bounds__(kTileThreads, QM == 2 ? 3 : 5)
    k_push_tile3d(PartF32 P, const TileItem *__restrict__ items, const uint32_t *__restrict__ nitems,
                  float *__restrict__ F, Grid g, PushConst pc, int *err, double *e_abs, uint32_t *defer,
                  uint32_t *ndefer, const __grid_constant__ CUtensorMap tmap, int use_tma, QedParams q)
{
    using B = Box3<T>;
    extern __shared__ __align__(16) float smem_raw[];
    __shared__ uint64_t mbar;
    // the TMA destination starts on a 128-byte boundary
    // (offset from the shared array itself, so that the compiler keeps every
    // access below in the shared address space)
    float *smem = smem_raw + ((128u - ((uint32_t)__cvta_generic_to_shared(smem_raw) & 127u)) & 127u) / 4u;
    float *sF = smem;                                    // 6 components
    int *sJ = reinterpret_cast<int *>(smem + 6 * B::N);  // 3 components, fixed point
    unsigned char *sNet = reinterpret_cast<unsigned char *>(smem) + B::SMEM;  // QM == 2: the network
    if constexpr (QM == 2) mlp_stage(sNet, q.net, kMlpStageBytes);
    const int nit = (int)*nitems;
    const long long V = g.vol;
    const float hdx[3] = {pc.hdx_f[0], pc.hdx_f[1], pc.hdx_f[2]};
    const float k = pc.qmdt2_f;
    const float cjx = pc.cJ_f[0], cjy = pc.cJ_f[1], cjz = pc.cJ_f[2];
    // fixed-point unit of the shared current box: 2^20 units per C, C the
    // largest value one particle adds to a node (see AccShared)
    const float cmax = fmaxf(fmaxf(fabsf(cjx), fabsf(cjy)), fabsf(cjz));
    const float jscale = 1048576.0f / fmaxf(cmax, 1e-30f);
    const float junit = 1.0f / jscale;
    float *Fg = F + g.origin;
    const int rs = (int)g.sy, ps = (int)g.sz;
    if (use_tma && threadIdx.x == 0) mbar_init(&mbar, 1);
    __syncthreads();
    uint32_t phase = 0;
    for (int it = blockIdx.x; it < nit; it += gridDim.x) {
        const TileItem m = items[it];
        const int tx = m.tile % g.ntile[0], ty = (m.tile / g.ntile[0]) % g.ntile[1],
                  tz = m.tile / (g.ntile[0] * g.ntile[1]);
        const int o0[3] = {tx * T - 4, ty * T - 3, tz * T - 3};
        // 1-2. stage fields (one TMA tile: x padded coordinate tx*T, a
        // multiple of 4 floats; else float4 rows), zero the current box
        if (use_tma) {
            if (threadIdx.x == 0) {
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&mbar, 6 * B::N * (int)sizeof(float));
                tma_load_4d(sF, &tmap, o0[0] + g.G[0], o0[1] + g.G[1], o0[2] + g.G[2], 0, &mbar);
            }
        } else {
            for (int e4 = threadIdx.x; e4 < 6 * B::N / 4; e4 += blockDim.x) {
                const int e = 4 * e4;
                const int c = e / B::N, r = e - c * B::N;
                const int z = r / B::PS, y = (r - z * B::PS) / B::RS, x = r - z * B::PS - y * B::RS;
                const float *src = Fg + c * V + (long long)(o0[2] + z) * ps + (long long)(o0[1] + y) * rs + o0[0] + x;
                reinterpret_cast<float4 *>(sF)[e4] = __ldg(reinterpret_cast<const float4 *>(src));
            }
        }
        for (int e4 = threadIdx.x; e4 < 3 * B::N / 4; e4 += blockDim.x)
            reinterpret_cast<int4 *>(sJ)[e4] = make_int4(0, 0, 0, 0);
        bool landed = true;
        if (use_tma) {
            landed = mbar_wait(&mbar, phase, 1 << 22);
            phase ^= 1u;
        }
        if (__syncthreads_or(!landed)) {
            if (threadIdx.x == 0) atomicOr(err, ERR_TIMEOUT);
            return;
        }
        // 3. particles, in block-wide passes (warp-uniform), consecutive lanes
        // on consecutive particles: the particle state is read straight from
        // HBM, coalesced (lane striding, as in 2D, measured 5 % slower here:
        // without a staging buffer its loads scatter)
        for (int pbase = 0; pbase < m.count; pbase += blockDim.x) {
            const int li = pbase + threadIdx.x;
            const int p = m.start + li;
            const bool mine = li < m.count;
            const uint32_t cp = mine ? P.cell[p] : kDead;
            bool act = cp != kDead;
            int c[3] = {0, 0, 0}, ch[3] = {0, 0, 0}, c1[3] = {0, 0, 0};
            float o[3] = {0.f, 0.f, 0.f}, oh[3] = {0.f, 0.f, 0.f}, o1[3] = {0.f, 0.f, 0.f};
            float ux = 0.f, uy = 0.f, uz = 0.f, ig1 = 0.f;
            float eb[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (act) {
                unpack_cell(g, cp, c[0], c[1], c[2]);
                o[0] = P.off[0][p];
                o[1] = P.off[1][p];
                o[2] = P.off[2][p];
                ux = P.u[0][p];
                uy = P.u[1][p];
                uz = P.u[2][p];
                const float ig = inv_gamma_fast(ux, uy, uz);
                const float u[3] = {ux, uy, uz};
#pragma unroll
                for (int d = 0; d < 3; d++) drift_f32(c[d], o[d], hdx[d] * u[d] * ig);
                int icn[3], ich[3];
                float wn[3][3], wh[3][3];
                bool gin = true;
#pragma unroll
                for (int d = 0; d < 3; d++) {
                    ch[d] = c[d];
                    oh[d] = o[d];
                    axis_w_f32(c[d], o[d], icn[d], wn[d], ich[d], wh[d]);
                    const int W = d == 0 ? B::WX : B::WY;
                    gin &= ch[d] - 1 >= o0[d] && ch[d] + 2 < o0[d] + W;
                }
                if (QM == 0 && !gin) {
                    defer[atomicAdd(ndefer, 1u)] = (uint32_t)p;
                    act = false;  // pushed by the list, from its unchanged state
                } else {
                    if (gin) gather3d_box<T>(sF, o0, icn, wn, ich, wh, eb);
                    else gather3d_global(F, g, icn, wn, ich, wh, eb);
                    if (pc.pusher) vay<float>(ux, uy, uz, k * eb[0], k * eb[1], k * eb[2], k * eb[3], k * eb[4], k * eb[5]);
                    else boris_fast(ux, uy, uz, k * eb[0], k * eb[1], k * eb[2], k * eb[3], k * eb[4], k * eb[5]);
                }
            }
            // QED (every lane of the block: the network's evaluation is warp-collective)
            uint32_t event = 0;
            float4 evd = make_float4(0.f, 0.f, 0.f, 0.f);
            if constexpr (QM != 0) qed_lepton_f32<QM == 2>(q, sNet, act, p, eb, ux, uy, uz, err, event, evd);
            bool dep = false;  // deposited (so the state is written)
            if (act) {
                ig1 = inv_gamma_fast(ux, uy, uz);
                const float dd[3] = {hdx[0] * ux * ig1, hdx[1] * uy * ig1, hdx[2] * uz * ig1};
#pragma unroll
                for (int d = 0; d < 3; d++) drift_f32(c[d], o[d], dd[d]);
#pragma unroll
                for (int d = 0; d < 3; d++) {
                    c1[d] = c[d];
                    o1[d] = o[d];
                }
#pragma unroll
                for (int d = 0; d < 3; d++) drift_f32(c[d], o[d], dd[d]);
                // Esirkepov on x^{n+1/2} -> x^{n+3/2}
                int i0[3], i1[3];
                float w0[3][3], w1[3][3];
                bool ok = true, din = true;
                float S0[3][4], dS[3][4];
                int u0[3];
#pragma unroll
                for (int d = 0; d < 3; d++) {
                    axis_wn_f32(ch[d], oh[d], i0[d], w0[d]);
                    axis_wn_f32(c[d], o[d], i1[d], w1[d]);
                    ok &= (i1[d] - i0[d] >= -1 && i1[d] - i0[d] <= 1);
                    u0[d] = union4(i0[d], w0[d], i1[d], w1[d], S0[d], dS[d]);
                    const int W = d == 0 ? B::WX : B::WY;
                    din &= u0[d] >= o0[d] && u0[d] + 3 < o0[d] + W;
                }
                // a non-finite momentum (a NaN or infinite field) is reported and the particle
                // removed before anything uses its position: NaN positions would give no valid
                // cell or node index to the gather, the deposit or the diagnostics (and would
                // otherwise be reported as a Courant violation)
                if (!isfinite(ux + uy + uz)) {
                    atomicOr(err, ERR_NONFINITE);
                    P.cell[p] = kDead;
                } else if (!ok) {
                    atomicOr(err, ERR_CFL);
                } else if (din) {
                    esirkepov3d_box<T>(sJ + (u0[2] - o0[2]) * B::PS + (u0[1] - o0[1]) * B::RS + (u0[0] - o0[0]), S0,
                                       dS, cjx, cjy, cjz, jscale);
                    dep = true;
                } else if (QM == 0) {
                    defer[atomicAdd(ndefer, 1u)] = (uint32_t)p;  // pushed by the list from its unchanged state
                } else {
                    dep = deposit3d_global(F, g, pc, ch, oh, c, o, uy, uz, ig1);
                    if (!dep) atomicOr(err, ERR_CFL);
                }
            }
            if (!dep) {
                if (QM != 0 && mine) q.ev[p] = 0;
                continue;
            }
            // boundaries
            int cc[3] = {c1[0], c1[1], c1[2]};
            bool dead = false;
#pragma unroll
            for (int d = 0; d < 3; d++) {
                if (g.bc[d] == PERIODIC) {
                    if (cc[d] < 0) cc[d] += g.n[d];
                    else if (cc[d] >= g.n[d]) cc[d] -= g.n[d];
                } else if (cc[d] < 0 || cc[d] >= g.n[d]) {
                    dead = true;
                }
            }
            if (dead) {
                P.cell[p] = kDead;
                double uu = (double)ux * ux + (double)uy * uy + (double)uz * uz;
                atomicAdd(e_abs, pc.wmdV * uu / (sqrt(1.0 + uu) + 1.0));
                event = 0;  // an emitter absorbed in the same step records no photon
            } else {
                P.cell[p] = pack_cell(g, cc[0], cc[1], cc[2]);
            }
#pragma unroll
            for (int d = 0; d < 3; d++) P.off[d][p] = o1[d];
            P.u[0][p] = ux;
            P.u[1][p] = uy;
            P.u[2][p] = uz;
            if constexpr (QM != 0) {
                q.ev[p] = event;
                if (event) reinterpret_cast<float4 *>(q.evk)[p] = evd;
            }
        }
        __syncthreads();
        // 4. flush the current box, four values at a time
        for (int e4 = threadIdx.x; e4 < 3 * B::N / 4; e4 += blockDim.x) {
            const int4 iv = reinterpret_cast<const int4 *>(sJ)[e4];
            if ((iv.x | iv.y | iv.z | iv.w) == 0) continue;
            const int e = 4 * e4;
            const int c = e / B::N, r = e - c * B::N;
            const int z = r / B::PS, y = (r - z * B::PS) / B::RS, x = r - z * B::PS - y * B::RS;
            float *dst = Fg + (JX + c) * V + (long long)(o0[2] + z) * ps + (long long)(o0[1] + y) * rs + o0[0] + x;
            atomicAdd(reinterpret_cast<float4 *>(dst), make_float4(iv.x * junit, iv.y * junit, iv.z * junit, iv.w * junit));
        }
        __syncthreads();
    }
}

template <int QM>
static void launch_tile3d_T(const PartF32 &P, const TileItem *items, const uint32_t *nitems, long long max_items,
                            float *F, const Grid &g, const PushConst &pc, int *err, double *e_abs, uint32_t *defer,
                            uint32_t *ndefer, cudaStream_t st, const QedParams &q)
{
    constexpr int T = 4;
    constexpr int smem = Box3<T>::SMEM + 128 + (QM == 2 ? kMlpStageBytes : 0);  // + alignment of the TMA destination
    static bool attr = false;
    static int nsm = 0, per_sm = 0;
    if (!attr) {
        cudaFuncSetAttribute(k_push_tile3d<T, QM>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_push_tile3d<T, QM>, kTileThreads, smem);
        if (per_sm < 1) per_sm = 1;
        attr = true;
    }
    // the six field components as one 4D tensor (x, y, z, component)
    CUtensorMap tmap;
    const int box[4] = {Box3<T>::WX, Box3<T>::WY, Box3<T>::WZ, 6};
    const bool tma = tma_encode_field_map3(&tmap, F, g.ext, g.sy, g.sz, g.vol, 6, box);
    if (!tma) memset(&tmap, 0, sizeof tmap);
    long long grid = std::min<long long>(max_items, (long long)nsm * per_sm);  // one resident wave
    if (grid < 1) grid = 1;
    note_launch();
    k_push_tile3d<T, QM><<<(int)grid, kTileThreads, smem, st>>>(P, items, nitems, F, g, pc, err, e_abs, defer, ndefer,
                                                                 tmap, tma ? 1 : 0, q);
}

void launch_push_tile3d(const PartF32 &P, const TileItem *items, const uint32_t *nitems, long long max_items,
                        float *F, const Grid &g, const PushConst &pc, int *err, double *e_abs, uint32_t *defer,
                        uint32_t *ndefer, cudaStream_t st, const QedParams *q)
{
    if (P.n == 0) return;
    if (q && q->on) {  // QED leptons: no deferral (see k_push_tile3d)
        if (q->net) launch_tile3d_T<2>(P, items, nitems, max_items, F, g, pc, err, e_abs, defer, ndefer, st, *q);
        else launch_tile3d_T<1>(P, items, nitems, max_items, F, g, pc, err, e_abs, defer, ndefer, st, *q);
        return;
    }
    cudaMemsetAsync(ndefer, 0, sizeof(uint32_t), st);
    const QedParams none{};
    launch_tile3d_T<0>(P, items, nitems, max_items, F, g, pc, err, e_abs, defer, ndefer, st, none);
    launch_push_list_f32(P, defer, ndefer, P.n, F, g, pc, err, e_abs, st);
}

bool tile3d_push_supported(const Grid &g)
{
    for (int d = 0; d < 3; d++)
        if (g.tile_log2[d] != 2 || g.n[d] % 4 != 0 || g.G[d] != 4) return false;
    return g.dim == 3;
}

}  // namespace pic
