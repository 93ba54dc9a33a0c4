// push_tile.cu -- tiled particle push for 2D grids (FP32 cell+offset form).
//
// Particles are counting-sorted by tile (T x T cells) every K steps.  Each
// work item is a chunk of at most kChunk particles that sat in one tile at the
// last sort.  A persistent CTA takes items in turn and, per item:
//   1. stages the six field components of the tile box [t0-4, t0+T+8) x
//      [t0-4, t0+T+5) into shared memory (rows are contiguous in HBM);
//   2. zeroes a shared current box of the same shape;
//   3. pushes every particle of the chunk (half drift, gather from shared
//      memory, Boris, two half drifts, Esirkepov on the 4-node union window
//      with shared-memory atomics);
//   4. flushes the current box to HBM with vector atomics (float4), once.
// A particle that drifted so far since the sort that its stencil leaves the
// box is handled on the global path (gather from HBM, global atomics), so the
// result does not depend on the sort interval.
#include <cstring>

#include "push_qed_dev.cuh"
#include "push_tile_dev.cuh"
#include "tma.cuh"

namespace pic {

// particle staging: slot (j, l) of particle i = l*S + j (lane l, segment
// position j < kChunk/32) sits at j*33 + l, so the 32 lanes of a read hit
// 32 banks
constexpr int kPSlot = 33 * (kChunk / 32);

template <int T>
struct Box2 {
    static constexpr int WX = T + 12;  // x: [t0-4, t0+T+8), a multiple of 4 floats
    static constexpr int WY = T + 9;   // y: [t0-4, t0+T+5)
    static constexpr int N = WX * WY;
    // fields (6) + current (3) boxes + staged particle state (6 arrays)
    static constexpr int SMEM = (9 * N + 6 * kPSlot) * (int)sizeof(float);
};

// Eq. (19) in 2D on a strided view: F_c(x, y) = P[c*cs + (y-oy)*rs + (x-ox)]
__device__ __forceinline__ void gather2d(const float *__restrict__ P, long long cs, int rs, int ox, int oy,
                                         const int *icn, const float (*wn)[3], const int *ich, const float (*wh)[3],
                                         float *eb)
{
#pragma unroll
    for (int c = 0; c < 6; c++) {
        const int sx = stag(c, 0), sy = stag(c, 1);
        const int ix = (sx ? ich[0] : icn[0]) - 1 - ox;
        const int iy = (sy ? ich[1] : icn[1]) - 1 - oy;
        const float *wx = sx ? wh[0] : wn[0];
        const float *wy = sy ? wh[1] : wn[1];
        const float *row = P + c * cs + (long long)iy * rs + ix;
        float acc = 0.f;
#pragma unroll
        for (int b = 0; b < 3; b++) {
            const float *r = row + (long long)b * rs;
            float s = wx[0] * r[0];
            s += wx[1] * r[1];
            s += wx[2] * r[2];
            acc += wy[b] * s;
        }
        eb[c] = acc;
    }
}

// Esirkepov in 2D on the union window (Eqs. (20)-(22)): W_x = dSx (S0y +
// dSy/2), W_y = dSy (S0x + dSx/2), and J_z = q w v_z times the time average
// of the node-shape product, S0xS0y + (dSx S0y + S0x dSy)/2 + dSx dSy/3,
// written as tx ty + dSx dSy/12 with tx = S0x + dSx/2, ty = S0y + dSy/2.
// `Acc` adds one value at window offset (a, b) of component c.
template <class Acc>
__device__ __forceinline__ void esirkepov2d(const float (*S0)[4], const float (*dS)[4], float cjx, float cjy,
                                            float jvz, Acc &acc)
{
    float tx[4], ty[4], dx12[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        tx[k] = S0[0][k] + 0.5f * dS[0][k];
        ty[k] = S0[1][k] + 0.5f * dS[1][k];
        dx12[k] = dS[0][k] * (1.0f / 12.0f);
    }
    float px[3], py[3];  // prefix sums of dS along x and y
    px[0] = dS[0][0];
    py[0] = dS[1][0];
#pragma unroll
    for (int k = 1; k < 3; k++) {
        px[k] = px[k - 1] + dS[0][k];
        py[k] = py[k - 1] + dS[1][k];
    }
#pragma unroll
    for (int b = 0; b < 4; b++)
#pragma unroll
        for (int a = 0; a < 3; a++) acc.add(0, a, b, cjx * px[a] * ty[b]);
#pragma unroll
    for (int b = 0; b < 3; b++)
#pragma unroll
        for (int a = 0; a < 4; a++) acc.add(1, a, b, cjy * py[b] * tx[a]);
#pragma unroll
    for (int b = 0; b < 4; b++)
#pragma unroll
        for (int a = 0; a < 4; a++) acc.add(2, a, b, jvz * (tx[a] * ty[b] + dx12[a] * dS[1][b]));
}

// current straight into HBM (particles whose window left the box)
struct AccGlobal {
    float *base;
    long long cs;
    int rs;
    __device__ __forceinline__ void add(int c, int a, int b, float v)
    {
        if (v != 0.f) atomicAdd(base + c * cs + (long long)b * rs + a, v);
    }
};

// warp-aggregated current into the shared box: the lanes of grp share the
// window origin; each value is summed over the group with one warp
// reduction and added by the group's first lane with one shared atomic
// (in the fixed-point units of AccShared; a group sum of at most 32
// particles stays far inside int32)
struct AccWarp {
    int *base;
    int cs, rs;
    float scale;
    unsigned grp;
    bool lead;
    __device__ __forceinline__ void add(int c, int a, int b, float v)
    {
        const int s = __reduce_add_sync(grp, __float2int_rn(v * scale));
        if (lead && s) atomicAdd(base + c * cs + b * rs + a, s);
    }
};

// With use_tma the field box of an item is one TMA tile copy (tmap: the six
// field components as a 3D tensor, x fastest), issued by one thread and
// overlapping the zeroing of the current box and the particle staging.
//
// AGG (warp-aggregated deposit): the 32 lanes of a warp take 32 consecutive
// particles of the item (the sort orders a tile's particles by cell, so they
// share cells: their gathers read the same nodes -- shared-memory broadcasts --
// and lanes with the same deposit window are summed before one atomic per
// value).  Without AGG lane l walks the l-th of 32 contiguous segments, so
// the lanes of an atomic hit different cells.
//
// QM (QED leptons): 1 = the Monte Carlo of Sec. IV with the
// tables (Method I or II), 2 = with the surrogate network inside its chi
// range (its image staged after the boxes); between the momentum update and
// the drifts, as in the one-thread-per-particle QED push.  The event flag
// of every particle of the items is written (0 for dead ones); particles
// appended after the sort are left to that kernel.
template <int T, bool AGG, int QM>
__global__ void __launch_bounds__(kTileThreads, QM == 2 ? 3 : kTileMinBlocks)
    k_push_tile2d(PartF32 P, const TileItem *__restrict__ items, const uint32_t *__restrict__ nitems,
                  float *__restrict__ F, Grid g, PushConst pc, int *err, double *e_abs,
                  const __grid_constant__ CUtensorMap tmap, int use_tma, QedParams q)
{
    using B = Box2<T>;
    extern __shared__ __align__(16) float smem_raw[];
    __shared__ uint64_t mbar;
    // the TMA destination starts on a 128-byte boundary
    // (offset from the shared array itself, so that the compiler keeps every
    // access below in the shared address space)
    float *smem = smem_raw + ((128u - ((uint32_t)__cvta_generic_to_shared(smem_raw) & 127u)) & 127u) / 4u;
    float *sF = smem;           // 6 components
    int *sJ = reinterpret_cast<int *>(smem + 6 * B::N);  // 3 components, fixed point
    float *sP = smem + 9 * B::N;                          // off_x, off_y, u_x, u_y, u_z
    uint32_t *sPc = reinterpret_cast<uint32_t *>(sP + 5 * kPSlot);  // packed cell
    unsigned char *sNet = reinterpret_cast<unsigned char *>(smem) + ((B::SMEM + 15) & ~15);  // QM == 2: the network
    if constexpr (QM == 2) mlp_stage(sNet, q.net, kMlpStageBytes);
    const int nit = (int)*nitems;
    const long long V = g.vol;
    const float hdx0 = pc.hdx_f[0], hdx1 = pc.hdx_f[1];
    const float k = pc.qmdt2_f;
    const float cjx = pc.cJ_f[0], cjy = pc.cJ_f[1], qw = pc.qw_f;
    // fixed-point unit of the shared current box: 2^20 units per C
    const float cmax = fabsf(qw) * fmaxf(fmaxf(fabsf(cjx), fabsf(cjy)) / fmaxf(fabsf(qw), 1e-30f), 1.0f);
    const float jscale = 1048576.0f / fmaxf(cmax, 1e-30f);
    const float junit = 1.0f / jscale;
    const float sjx = cjx * jscale, sjy = cjy * jscale;
    float *Fg = F + g.origin;  // interior origin
    const int rs = (int)g.sy;
    if (use_tma && threadIdx.x == 0) mbar_init(&mbar, 1);
    __syncthreads();
    uint32_t phase = 0;
    for (int it = blockIdx.x; it < nit; it += gridDim.x) {
        const TileItem m = items[it];
        const int tx = m.tile % g.ntile[0], ty = m.tile / g.ntile[0];
        const int bx0 = tx * T - 4, by0 = ty * T - 4;
        // 1-2. stage fields, zero the current box
        if (use_tma) {
            if (threadIdx.x == 0) {
                // padded coordinates of the box corner; x = tx*T is a multiple
                // of 4 floats (16 bytes) as the copy engine requires
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&mbar, 6 * B::N * (int)sizeof(float));
                tma_load_3d(sF, &tmap, bx0 + g.G[0], by0 + g.G[1], 0, &mbar);
            }
        } else {
            for (int e = threadIdx.x; e < 6 * B::N; e += blockDim.x) {
                const int c = e / B::N, r = e - c * B::N;
                const int y = r / B::WX, x = r - y * B::WX;
                const int gx = bx0 + x, gy = by0 + y;
                float v = 0.f;
                if (gx < g.n[0] + g.G[0] && gy < g.n[1] + g.G[1]) v = __ldg(Fg + c * V + (long long)gy * rs + gx);
                sF[e] = v;
            }
        }
        for (int e = threadIdx.x; e < 3 * B::N; e += blockDim.x) sJ[e] = 0;
        // Lane striding: the chunk is cut into 32 contiguous segments of S
        // particles and lane l of every warp walks segment l.  Sorted
        // particles of one cell are contiguous, so the 32 lanes of one
        // shared-memory atomic target 32 different cells (different current
        // addresses) instead of one, whatever the in-tile order.
        const int S = (m.count + 31) >> 5;
        // i / S for i < kChunk as a float product: (i + 1/2) / S lies at least
        // 1/(2S) from an integer, far beyond the product's rounding
        const float invS = 1.0f / (float)S;
        // stage the chunk's particle state: every thread issues all its loads
        // at once (coalesced), stored transposed to (segment position, lane)
        // (asynchronous 4-byte copies: no register round trip)
        for (int i = threadIdx.x; i < m.count; i += blockDim.x) {
            const int l = __float2int_rz(((float)i + 0.5f) * invS), j = i - l * S;
            const int pos = AGG ? i : j * 33 + l;
            const int p = m.start + i;  // capacities are below 2^31
            cp_async4(sPc + pos, P.cell + p);
            cp_async4(sP + 0 * kPSlot + pos, P.off[0] + p);
            cp_async4(sP + 1 * kPSlot + pos, P.off[1] + p);
            cp_async4(sP + 2 * kPSlot + pos, P.u[0] + p);
            cp_async4(sP + 3 * kPSlot + pos, P.u[1] + p);
            cp_async4(sP + 4 * kPSlot + pos, P.u[2] + p);
        }
        cp_async_wait_all();
        bool landed = true;
        if (use_tma) {
            // bounded wait: a copy that never lands sets an error flag and the
            // CTA stops, all its threads together (the host reports the flag)
            landed = mbar_wait(&mbar, phase, 1 << 22);
            phase ^= 1u;
        }
        if (__syncthreads_or(!landed)) {
            if (threadIdx.x == 0) atomicOr(err, ERR_TIMEOUT);
            return;
        }
        // 3. particles
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        constexpr int kWarps = kTileThreads / 32;
        // passes of the warp over the item: warp-uniform, so the lanes stay
        // together for the warp-collective deposit of AGG
        const int npass = AGG ? (m.count + kTileThreads - 1) / kTileThreads : (S + kWarps - 1) / kWarps;
        for (int pass = 0; pass < npass; pass++) {
            int li, pos;
            if (AGG) {
                li = pass * kTileThreads + warp * 32 + lane;
                pos = li;
            } else {
                const int j = pass * kWarps + warp;
                li = j < S ? lane * S + j : m.count;
                pos = j * 33 + lane;
            }
            const uint32_t cp = li < m.count ? sPc[pos] : kDead;
            bool act = cp != kDead;  // a live particle of this item
            int c[2] = {0, 0}, c1[2] = {0, 0}, u0[2] = {0, 0};
            float o[2] = {0.f, 0.f}, o1[2] = {0.f, 0.f};
            float ux = 0.f, uy = 0.f, uz = 0.f, ig1 = 0.f;
            float S0[2][4], dS[2][4];
            int ch[2] = {0, 0};
            float eb[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            int icn[2] = {0, 0};  // node shape at x^{n+1/2}: the gather's, and the deposit's start
            float wn[2][3];
            bool ok = true;
            if (act) {
                int dummy;
                unpack_cell(g, cp, c[0], c[1], dummy);
                o[0] = sP[pos];
                o[1] = sP[kPSlot + pos];
                ux = sP[2 * kPSlot + pos];
                uy = sP[3 * kPSlot + pos];
                uz = sP[4 * kPSlot + pos];
                float ig = inv_gamma_fast(ux, uy, uz);
                drift_f32(c[0], o[0], hdx0 * ux * ig);
                drift_f32(c[1], o[1], hdx1 * uy * ig);
                ch[0] = c[0];
                ch[1] = c[1];
                int ich[2];
                float wh[2][3];
                axis_w_f32(c[0], o[0], icn[0], wn[0], ich[0], wh[0]);
                axis_w_f32(c[1], o[1], icn[1], wn[1], ich[1], wh[1]);
                const bool gin =
                    ch[0] - 1 >= bx0 && ch[0] + 2 < bx0 + B::WX && ch[1] - 1 >= by0 && ch[1] + 2 < by0 + B::WY;
                if (gin) gather2d(sF, B::N, B::WX, bx0, by0, icn, wn, ich, wh, eb);
                else gather2d(Fg, V, rs, 0, 0, icn, wn, ich, wh, eb);
                if (pc.pusher) vay<float>(ux, uy, uz, k * eb[0], k * eb[1], k * eb[2], k * eb[3], k * eb[4], k * eb[5]);
                else boris_fast(ux, uy, uz, k * eb[0], k * eb[1], k * eb[2], k * eb[3], k * eb[4], k * eb[5]);
            }
            // QED (every lane of the warp: the network's evaluation is collective)
            const long long pg = (long long)m.start + li;
            uint32_t event = 0;
            float4 evd = make_float4(0.f, 0.f, 0.f, 0.f);
            if constexpr (QM != 0) qed_lepton_f32<QM == 2>(q, sNet, act, pg, eb, ux, uy, uz, err, event, evd);
            if (act) {
                ig1 = inv_gamma_fast(ux, uy, uz);
                const float d0 = hdx0 * ux * ig1, d1 = hdx1 * uy * ig1;
                drift_f32(c[0], o[0], d0);
                drift_f32(c[1], o[1], d1);
                c1[0] = c[0];
                c1[1] = c[1];
                o1[0] = o[0];
                o1[1] = o[1];
                drift_f32(c[0], o[0], d0);
                drift_f32(c[1], o[1], d1);
                // Esirkepov on x^{n+1/2} -> x^{n+3/2}
#pragma unroll
                for (int d = 0; d < 2; d++) {
                    int i1;
                    float w1[3];
                    axis_wn_f32(c[d], o[d], i1, w1);
                    ok &= (i1 - icn[d] >= -1 && i1 - icn[d] <= 1);
                    u0[d] = union4(icn[d], wn[d], i1, w1, S0[d], dS[d]);
                }
                // a non-finite momentum (a NaN or infinite field) is reported and the particle
                // removed before anything uses its position: NaN positions would give no valid
                // cell or node index to the gather, the deposit or the diagnostics (and would
                // otherwise be reported as a Courant violation)
                if (!isfinite(ux + uy + uz)) {
                    atomicOr(err, ERR_NONFINITE);
                    sPc[pos] = kDead;
                    act = false;
                } else if (!ok) {
                    atomicOr(err, ERR_CFL);
                    act = false;  // keeps its staged state
                }
            }
            const float jvz = qw * uz * ig1;
            const bool din = act && u0[0] >= bx0 && u0[0] + 3 < bx0 + B::WX && u0[1] >= by0 && u0[1] + 3 < by0 + B::WY;
            if (act && !din) {
                AccGlobal acc{Fg + JX * V + (long long)u0[1] * rs + u0[0], V, rs};
                esirkepov2d(S0, dS, cjx, cjy, jvz, acc);
            }
            if (AGG) {
                const unsigned smask = __ballot_sync(0xffffffffu, din);
                if (din) {
                    const int key = (u0[1] - by0) * B::WX + (u0[0] - bx0);
                    const unsigned grp = __match_any_sync(smask, key);
                    AccWarp acc{sJ + key, B::N, B::WX, jscale, grp, lane == __ffs(grp) - 1};
                    esirkepov2d(S0, dS, cjx, cjy, jvz, acc);
                }
            } else {
                // A warp whose 32 lanes all deposit on one window (a dense
                // beam: the whole chunk in one cell, so lane striding cannot
                // spread the lanes over cells) sums each value over the warp
                // with one reduction and adds it with one atomic; otherwise
                // every lane adds its own values (lanes on different cells).
                // The fixed-point scale is folded into the three coefficients.
                const int key = din ? (u0[1] - by0) * B::WX + (u0[0] - bx0) : -1;
                int same = 0;
                // (checked in the QED variants, whose beams are dense; a plain
                // plasma of tens of particles per cell never fills a warp's
                // lanes with one window, and the check costs ~3 % there)
                if constexpr (QM != 0) __match_all_sync(0xffffffffu, key, &same);
                if (same && key >= 0) {
                    AccWarpAll acc{sJ + key, B::N, B::WX, lane == 0};
                    esirkepov2d(S0, dS, sjx, sjy, jvz * jscale, acc);
                } else if (din) {
                    AccSharedUnits acc{sJ + key, B::N, B::WX};
                    esirkepov2d(S0, dS, sjx, sjy, jvz * jscale, acc);
                }
            }
            if (!act) {
                if (QM != 0 && li < m.count) q.ev[pg] = 0;
                continue;
            }
            // boundaries
            int cc[2] = {c1[0], c1[1]};
            bool dead = false;
#pragma unroll
            for (int d = 0; d < 2; d++) {
                if (g.bc[d] == PERIODIC) {
                    if (cc[d] < 0) cc[d] += g.n[d];
                    else if (cc[d] >= g.n[d]) cc[d] -= g.n[d];
                } else if (cc[d] < 0 || cc[d] >= g.n[d]) {
                    dead = true;
                }
            }
            if (dead) {
                sPc[pos] = kDead;
                double uu = (double)ux * ux + (double)uy * uy + (double)uz * uz;
                atomicAdd(e_abs, pc.wmdV * uu / (sqrt(1.0 + uu) + 1.0));
                event = 0;  // an emitter absorbed in the same step records no photon
            } else {
                sPc[pos] = pack_cell(g, cc[0], cc[1], 0);
            }
            if constexpr (QM != 0) {
                q.ev[pg] = event;
                if (event) reinterpret_cast<float4 *>(q.evk)[pg] = evd;
            }
            // the new state goes back to the particle's own staging slot and
            // leaves in array order below: lane-strided global stores would
            // touch 32 sectors per instruction
            sP[pos] = o1[0];
            sP[kPSlot + pos] = o1[1];
            sP[2 * kPSlot + pos] = ux;
            sP[3 * kPSlot + pos] = uy;
            sP[4 * kPSlot + pos] = uz;
        }
        __syncthreads();
        // 4a. write the chunk's state back, coalesced (particles skipped above
        // keep their staged values)
        for (int i = threadIdx.x; i < m.count; i += blockDim.x) {
            const int l = __float2int_rz(((float)i + 0.5f) * invS), j = i - l * S;
            const int pos = AGG ? i : j * 33 + l;
            const int p = m.start + i;
            P.cell[p] = sPc[pos];
            P.off[0][p] = sP[pos];
            P.off[1][p] = sP[kPSlot + pos];
            P.u[0][p] = sP[2 * kPSlot + pos];
            P.u[1][p] = sP[3 * kPSlot + pos];
            P.u[2][p] = sP[4 * kPSlot + pos];
        }
        // 4b. flush the current box, four values at a time
        for (int v4 = threadIdx.x; v4 < 3 * B::N / 4; v4 += blockDim.x) {
            const int4 iv = reinterpret_cast<const int4 *>(sJ)[v4];
            if ((iv.x | iv.y | iv.z | iv.w) == 0) continue;
            const float4 v = make_float4(iv.x * junit, iv.y * junit, iv.z * junit, iv.w * junit);
            const int e = 4 * v4;
            const int c = e / B::N, r = e - c * B::N;
            const int y = r / B::WX, x = r - y * B::WX;
            const int gx = bx0 + x, gy = by0 + y;
            if (gx < -g.G[0] || gx + 3 >= g.n[0] + g.G[0] || gy < -g.G[1] || gy >= g.n[1] + g.G[1]) {
                // partial vector at the edge of the padded box (holds zeros only
                // for accepted particles; kept exact for safety)
                float vv[4] = {v.x, v.y, v.z, v.w};
                for (int l = 0; l < 4; l++)
                    if (vv[l] != 0.f && gx + l >= -g.G[0] && gx + l < g.n[0] + g.G[0] && gy >= -g.G[1] &&
                        gy < g.n[1] + g.G[1])
                        atomicAdd(Fg + (JX + c) * V + (long long)gy * rs + gx + l, vv[l]);
                continue;
            }
            atomicAdd(reinterpret_cast<float4 *>(Fg + (JX + c) * V + (long long)gy * rs + gx), v);
        }
        __syncthreads();
    }
}

// The surrogate's candidate conversions (the thinned sampler of
// qed_photon_f32): the tiled photon push appends them to a queue, one slot
// per photon, and this kernel resolves them, 32 per network evaluation:
// the pair rate W and the positron fraction from one evaluation (from the
// tables for candidates below the network's chi range), a
// conversion with probability W / W_env (the candidate's draw of purpose
// QP_THIN), and the optical depth restarted from -ln r.  The network's
// registers stay out of the push, which then runs at the table push's
// occupancy.  Entries: (photon index, ln chi, W_env's G, chi); each
// candidate's outcome depends on its own entry and draws only, so the
// queue's order (that of the appends) does not change the result.
__global__ void __launch_bounds__(256) k_photon_resolve(QedParams q, PartF32 P, int *err)
{
    extern __shared__ __align__(16) unsigned char net[];
    mlp_stage(net, q.net, kMlpStageBytes);
    __syncthreads();
    const long long n = *q.cq_n;
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (long long wb = (long long)blockIdx.x * wpb + (threadIdx.x >> 5); wb * 32 < n; wb += (long long)gridDim.x * wpb) {
        const long long i = wb * 32 + lane;  // (warp-uniform loop: the evaluation is warp-collective)
        const bool mine = i < n;
        const float4 e = mine ? q.cq[i] : make_float4(0.f, 0.f, 1.f, 1.f);
        const long long p = (long long)(uint32_t)__float_as_int(e.x);
        const bool row = mine && e.y >= q.net_lo_f;  // inside the network's range (else the tables)
        uint32_t w[4] = {0u, 0u, 0u, 0u};
        float x0 = 0.f, x1 = 0.f, y0 = 0.f, y1 = 0.f;
        uint64_t id = 0;
        if (mine) {
            id = q.id[p];
            philox4x32_10((uint32_t)id, (uint32_t)(id >> 32), q.step, QP_PAIR, q.key[0], q.key[1], w);
            if (row) mlp_inputs_f32(q.nrm, QED_PAIR, e.y, uniform24_f32(w[0]), x0, x1);
        }
        if (__any_sync(0xffffffffu, row))
            mlp_eval_warp_sparse(*reinterpret_cast<const MlpImage *>(net), row, x0, x1, y0, y1);
        if (!mine) continue;
        const float G = row ? mlp_rate_f32(q.nrm, QED_PAIR, e.w, y1) : qed_rate_f32(q.T, QED_PAIR, e.w);
        const float pa = G / e.z;
        if (pa > 1.0f) atomicOr(err, ERR_QEDDT);
        uint32_t v[4];
        philox4x32_10((uint32_t)id, (uint32_t)(id >> 32), q.step, QP_THIN, q.key[0], q.key[1], v);
        const bool accept = uniform24_f32(v[0]) < pa;
        q.tau[p] = (double)neg_log_uniform24_f32(w[1]);
        q.ev[p] = accept ? 1u : 0u;
        if (accept) {
            const float r0 = uniform24_f32(w[0]);
            reinterpret_cast<float4 *>(q.evk)[p] = make_float4(
                P.u[0][p], P.u[1][p], P.u[2][p],
                row ? mlp_fraction_f32(QED_PAIR, y0, r0) : qed_sample_f32(q.T, QED_PAIR, e.w, r0));
        }
    }
}

// ---------------------------------------------------------------------
// Tiled photon push (2D, FP32).  Photons carry no current, so a work item
// only stages its tile's field box (one TMA copy) and walks its photons with
// consecutive lanes on consecutive photons: the particle traffic is
// coalesced and the gathers of photons of one cell are shared-memory
// broadcasts.  Each photon moves at c along k, its pair Monte Carlo is
// qed_photon_f32 (as in the one-thread-per-particle photon push), event
// flags are written for every photon of the items.  It runs over the sort's
// work items and over those of the photons appended since (k_tail_items).
// SURR: the thinned sampler up to the top of the network's chi range, its
// candidates appended to the queue that k_photon_resolve evaluates.
// ---------------------------------------------------------------------
template <int T, bool SURR>
__global__ void __launch_bounds__(kTileThreads, kTileMinBlocks)
    k_push_photon_tile2d(PartF32 P, const TileItem *__restrict__ items, const uint32_t *__restrict__ nitems,
                         const float *__restrict__ F, Grid g, PushConst pc, int *err,
                         const __grid_constant__ CUtensorMap tmap, int use_tma, QedParams q)
{
    using B = Box2<T>;
    extern __shared__ __align__(16) float smem_raw[];
    __shared__ uint64_t mbar;
    float *smem = smem_raw + ((128u - ((uint32_t)__cvta_generic_to_shared(smem_raw) & 127u)) & 127u) / 4u;
    float *sF = smem;  // 6 components
    // the item's photon state, staged by cp.async while the field box lands:
    // optical depth (FP64), cell, two offsets, three momentum components
    double *sTau = reinterpret_cast<double *>(smem + ((6 * B::N + 1) & ~1));
    uint32_t *sCell = reinterpret_cast<uint32_t *>(sTau + kChunk);
    float *sSt = reinterpret_cast<float *>(sCell + kChunk);  // off0, off1, k0, k1, k2: kChunk each
    const int lane = threadIdx.x & 31;
    const int nit = (int)*nitems;
    const long long V = g.vol;
    const float *Fg = F + g.origin;
    const int rs = (int)g.sy;
    const float hdx0 = pc.hdx_f[0], hdx1 = pc.hdx_f[1];
    if (use_tma && threadIdx.x == 0) mbar_init(&mbar, 1);
    __syncthreads();
    uint32_t phase = 0;
    for (int it = blockIdx.x; it < nit; it += gridDim.x) {
        const TileItem m = items[it];
        const int tx = m.tile % g.ntile[0], ty = m.tile / g.ntile[0];
        const int bx0 = tx * T - 4, by0 = ty * T - 4;
        if (use_tma) {
            if (threadIdx.x == 0) {
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&mbar, 6 * B::N * (int)sizeof(float));
                tma_load_3d(sF, &tmap, bx0 + g.G[0], by0 + g.G[1], 0, &mbar);
            }
        } else {
            for (int e = threadIdx.x; e < 6 * B::N; e += blockDim.x) {
                const int c = e / B::N, r = e - c * B::N;
                const int y = r / B::WX, x = r - y * B::WX;
                const int gx = bx0 + x, gy = by0 + y;
                float v = 0.f;
                if (gx < g.n[0] + g.G[0] && gy < g.n[1] + g.G[1]) v = __ldg(Fg + c * V + (long long)gy * rs + gx);
                sF[e] = v;
            }
        }
        for (int i = threadIdx.x; i < m.count; i += blockDim.x) {
            const int p = m.start + i;
            cp_async4(sCell + i, P.cell + p);
            cp_async4(sSt + i, P.off[0] + p);
            cp_async4(sSt + kChunk + i, P.off[1] + p);
            cp_async4(sSt + 2 * kChunk + i, P.u[0] + p);
            cp_async4(sSt + 3 * kChunk + i, P.u[1] + p);
            cp_async4(sSt + 4 * kChunk + i, P.u[2] + p);
            if (q.on) cp_async8(sTau + i, q.tau + p);
        }
        cp_async_wait_all();
        bool landed = true;
        if (use_tma) {
            landed = mbar_wait(&mbar, phase, 1 << 22);
            phase ^= 1u;
        }
        if (__syncthreads_or(!landed)) {
            if (threadIdx.x == 0) atomicOr(err, ERR_TIMEOUT);
            return;
        }
        // warp-uniform passes (the candidates' appends are warp-aggregated)
        const int npass = (m.count + kTileThreads - 1) / kTileThreads;
        for (int pass = 0; pass < npass; pass++) {
            const int li = pass * kTileThreads + threadIdx.x;
            const long long p = (long long)m.start + li;
            const uint32_t cp = li < m.count ? sCell[li] : kDead;
            const bool live = cp != kDead;
            int c[2] = {0, 0};
            float o[2] = {0.f, 0.f};
            float kx = 0.f, ky = 0.f, kz = 0.f;
            double tau0 = 0.0;
            if (live) {
                int dummy;
                unpack_cell(g, cp, c[0], c[1], dummy);
                o[0] = sSt[li];
                o[1] = sSt[kChunk + li];
                kx = sSt[2 * kChunk + li];
                ky = sSt[3 * kChunk + li];
                kz = sSt[4 * kChunk + li];
                if (q.on) tau0 = sTau[li];
            }
            const float km = sqrtf(kx * kx + ky * ky + kz * kz);
            const float ik = km > 0.f ? 1.0f / km : 0.f;
            const float d0 = hdx0 * kx * ik, d1 = hdx1 * ky * ik;
            drift_f32(c[0], o[0], d0);
            drift_f32(c[1], o[1], d1);
            uint32_t event = 0;
            float4 evd = make_float4(0.f, 0.f, 0.f, 0.f);
            bool cand = false;  // SURR: a candidate conversion, resolved by k_photon_resolve
            float4 centry = make_float4(0.f, 0.f, 0.f, 0.f);
            double tau = tau0;
            bool put_tau = false;  // SURR: store tau (thinned, not a candidate)
            if (q.on && live) {
                float eb[6];
                int icn[2], ich[2];
                float wn[2][3], wh[2][3];
                axis_w_f32(c[0], o[0], icn[0], wn[0], ich[0], wh[0]);
                axis_w_f32(c[1], o[1], icn[1], wn[1], ich[1], wh[1]);
                const bool gin =
                    c[0] - 1 >= bx0 && c[0] + 2 < bx0 + B::WX && c[1] - 1 >= by0 && c[1] + 2 < by0 + B::WY;
                if (gin) gather2d(sF, B::N, B::WX, bx0, by0, icn, wn, ich, wh, eb);
                else gather2d(Fg, V, rs, 0, 0, icn, wn, ich, wh, eb);
                if constexpr (SURR) {
                    // the thinned sampler of qed_photon_f32, with the network's
                    // evaluations gathered: candidates go to the queue that
                    // k_photon_resolve evaluates 32 at a time
                    const float chi = chi_f32(km, kx, ky, kz, eb[0], eb[1], eb[2], eb[3], eb[4], eb[5], q.inv_Es_f);
                    float lnchi;
                    mlp_in_range_f32(q.net_lo_f, q.net_hi_f, chi, lnchi);
                    if (km > 0.f && lnchi <= q.net_hi_f) {  // thinned up to the top of the network's range
                        const float genv = pair_envelope_f32(chi);
                        const float dtau = q.pref_f * genv / km;
                        if (!(dtau == 0.f && depth_positive(tau0))) {  // (else the depth stays, unstored)
                            tau = tau0 - (double)dtau;
                            cand = tau <= 0.0;
                            put_tau = !cand;
                            centry = make_float4(__int_as_float((int)p), lnchi, genv, chi);
                        }
                    } else {
                        qed_photon_f32<false>(q, nullptr, true, p, km, kx, ky, kz, eb, tau0, err, event, evd);
                    }
                } else {
                    qed_photon_f32<false>(q, nullptr, true, p, km, kx, ky, kz, eb, tau0, err, event, evd);
                }
            }
            bool dead = false;
            if (live) {
                drift_f32(c[0], o[0], d0);
                drift_f32(c[1], o[1], d1);
#pragma unroll
                for (int d = 0; d < 2; d++) {
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
                    cand = false;
                } else {
                    P.cell[p] = pack_cell(g, c[0], c[1], 0);
                }
                P.off[0][p] = o[0];
                P.off[1][p] = o[1];
            }
            if constexpr (SURR) {
                const unsigned cm = __ballot_sync(0xffffffffu, cand);
                if (cm) {
                    uint32_t at = 0;
                    if (lane == 0) at = atomicAdd(q.cq_n, (uint32_t)__popc(cm));
                    at = __shfl_sync(0xffffffffu, at, 0);
                    if (cand) q.cq[at + __popc(cm & ((1u << lane) - 1u))] = centry;
                }
            }
            if (li >= m.count) continue;
            if (!live) {
                q.ev[p] = 0;
                continue;
            }
            if (cand) continue;  // tau, flag and event data by k_photon_resolve
            if (SURR && put_tau) q.tau[p] = tau;  // (thinned, no candidate; qed_photon_f32 stores its own)
            q.ev[p] = event;
            if (event) reinterpret_cast<float4 *>(q.evk)[p] = evd;
        }
        __syncthreads();  // the next item's copies overwrite the box and the staging
    }
}

// ---------------------------------------------------------------------
// work items: chunks of at most `chunk` particles of one tile
// ---------------------------------------------------------------------
__global__ void k_item_counts(const uint32_t *__restrict__ starts, long long ntiles, uint32_t chunk, uint32_t *cnt)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t > ntiles) return;
    if (t == ntiles) {
        cnt[t] = 0;
        return;
    }
    uint32_t n = starts[t + 1] - starts[t];
    cnt[t] = (n + chunk - 1) / chunk;
}

__global__ void k_item_write(const uint32_t *__restrict__ starts, const uint32_t *__restrict__ off, long long ntiles,
                             uint32_t chunk, TileItem *items, uint32_t *nitems)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) {
        if (t == ntiles) *nitems = off[ntiles];
        return;
    }
    uint32_t s = starts[t], n = starts[t + 1] - s;
    uint32_t o = off[t];
    for (uint32_t q = 0; q * chunk < n; q++) {
        TileItem m;
        m.tile = (int)t;
        m.start = (int)(s + q * chunk);
        m.count = (int)min(chunk, n - q * chunk);
        m.pad = 0;
        items[o + q] = m;
    }
}

int tile_chunk(int dim) { return dim == 3 ? kChunk3 : kChunk; }

size_t tile_items_capacity(long long cap, long long ntiles, int dim)
{
    return (size_t)(ntiles + cap / tile_chunk(dim) + 2);
}

void build_tile_items(const uint32_t *starts, long long ntiles, int dim, uint32_t *cnt_scratch,
                      uint32_t *scan_scratch, TileItem *items, uint32_t *nitems, cudaStream_t st)
{
    const uint32_t chunk = (uint32_t)tile_chunk(dim);
    note_launch(2);
    k_item_counts<<<div_up(ntiles + 1, 256), 256, 0, st>>>(starts, ntiles, chunk, cnt_scratch);
    scan_exclusive(cnt_scratch, cnt_scratch, ntiles + 1, scan_scratch, st);
    k_item_write<<<div_up(ntiles + 1, 256), 256, 0, st>>>(starts, cnt_scratch, ntiles, chunk, items, nitems);
}

bool tile_push_supported(const Grid &g, int tile_edge)
{
    return g.dim == 2 && (1 << g.tile_log2[0]) == tile_edge && (1 << g.tile_log2[1]) == tile_edge;
}

template <int T, bool AGG, int QM>
static void launch_T(const PartF32 &P, const TileItem *items, const uint32_t *nitems, long long max_items, float *F,
                     const Grid &g, const PushConst &pc, int *err, double *e_abs, cudaStream_t st, const QedParams &q)
{
    // + alignment of the TMA destination (+ the network image)
    constexpr int smem = ((Box2<T>::SMEM + 15) & ~15) + 128 + (QM == 2 ? kMlpStageBytes : 0);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_push_tile2d<T, AGG, QM>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        attr = true;
    }
    static int nsm = 0;
    if (!nsm) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    }
    // the six field components as one 3D tensor (x, y, component); tiles of
    // the box shape.  Without a tensor map the kernel stages with loads.
    CUtensorMap tmap;
    const int box[3] = {Box2<T>::WX, Box2<T>::WY, 6};
    const bool tma = tma_encode_field_map(&tmap, F, g.ext[0], g.ext[1], g.sy, g.vol, 6, box);
    if (!tma) memset(&tmap, 0, sizeof tmap);
    static int per_sm = 0;  // resident CTAs per SM
    if (!per_sm) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_push_tile2d<T, AGG, QM>, kTileThreads, smem);
        if (per_sm < 1) per_sm = 1;
    }
    long long grid = std::min<long long>(max_items, (long long)nsm * per_sm);  // one resident wave
    if (grid < 1) grid = 1;
    note_launch();
    k_push_tile2d<T, AGG, QM><<<(int)grid, kTileThreads, smem, st>>>(P, items, nitems, F, g, pc, err, e_abs, tmap,
                                                                    tma ? 1 : 0, q);
}

template <int T>
static void launch_variant(const PartF32 &P, const TileItem *items, const uint32_t *nitems, long long max_items,
                           float *F, const Grid &g, const PushConst &pc, int *err, double *e_abs, cudaStream_t st,
                           bool agg, const QedParams *q)
{
    if (q && q->on) {
        if (q->net) launch_T<T, false, 2>(P, items, nitems, max_items, F, g, pc, err, e_abs, st, *q);
        else launch_T<T, false, 1>(P, items, nitems, max_items, F, g, pc, err, e_abs, st, *q);
        return;
    }
    const QedParams none{};
    if (agg) launch_T<T, true, 0>(P, items, nitems, max_items, F, g, pc, err, e_abs, st, none);
    else launch_T<T, false, 0>(P, items, nitems, max_items, F, g, pc, err, e_abs, st, none);
}

void launch_push_tile2d(const PartF32 &P, const TileItem *items, const uint32_t *nitems, long long max_items,
                        float *F, const Grid &g, const PushConst &pc, int *err, double *e_abs, cudaStream_t st,
                        bool agg, const QedParams *q)
{
    if (P.n == 0) return;
    if ((1 << g.tile_log2[0]) == 16) launch_variant<16>(P, items, nitems, max_items, F, g, pc, err, e_abs, st, agg, q);
    else launch_variant<8>(P, items, nitems, max_items, F, g, pc, err, e_abs, st, agg, q);
}

template <int T, bool SURR>
static void launch_photon_T(const PartF32 &P, const TileItem *items, const uint32_t *nitems, long long max_items,
                            const float *F, const Grid &g, const PushConst &pc, int *err, cudaStream_t st,
                            const QedParams &q)
{
    // field box + staging (tau 8 B, cell 4 B, 5 floats per photon), + TMA alignment
    constexpr int smem = ((6 * Box2<T>::N + 1) & ~1) * (int)sizeof(float) + kChunk * (8 + 4 + 20) + 128;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_push_photon_tile2d<T, SURR>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        attr = true;
    }
    static int nsm = 0, per_sm = 0;
    if (!nsm) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_push_photon_tile2d<T, SURR>, kTileThreads, smem);
        if (per_sm < 1) per_sm = 1;
    }
    CUtensorMap tmap;
    const int box[3] = {Box2<T>::WX, Box2<T>::WY, 6};
    const bool tma = tma_encode_field_map(&tmap, const_cast<float *>(F), g.ext[0], g.ext[1], g.sy, g.vol, 6, box);
    if (!tma) memset(&tmap, 0, sizeof tmap);
    long long grid = std::min<long long>(max_items, (long long)nsm * per_sm);
    if (grid < 1) grid = 1;
    note_launch();
    k_push_photon_tile2d<T, SURR><<<(int)grid, kTileThreads, smem, st>>>(P, items, nitems, F, g, pc, err, tmap,
                                                                         tma ? 1 : 0, q);
}

void launch_push_photon_tile2d(const PartF32 &P, const TileItem *items, const uint32_t *nitems, long long max_items,
                               const float *F, const Grid &g, const PushConst &pc, const QedParams &q, int *err,
                               cudaStream_t st)
{
    if (P.n == 0) return;
    const bool surr = q.on && q.net && q.cq;  // (the C ABI gives the QED photon species its queue)
    if ((1 << g.tile_log2[0]) == 16) {
        if (surr) launch_photon_T<16, true>(P, items, nitems, max_items, F, g, pc, err, st, q);
        else launch_photon_T<16, false>(P, items, nitems, max_items, F, g, pc, err, st, q);
    } else {
        if (surr) launch_photon_T<8, true>(P, items, nitems, max_items, F, g, pc, err, st, q);
        else launch_photon_T<8, false>(P, items, nitems, max_items, F, g, pc, err, st, q);
    }
}

// Work items over the photons appended since the last sort, [first, *dn):
// chunks of kChunk consecutive photons.  The spawn appends children in their
// parents' order, which is the parents' tile order, so a chunk's photons
// mostly share a tile: the item takes the tile of its middle photon (tile 0
// if that one is dead), and photons outside the item's field box take the
// kernel's global gather.  (The slots past the count need no event flag:
// the spawn reads flags up to the device count.)
__global__ void k_tail_items(const uint32_t *__restrict__ cell, const long long *__restrict__ dn,
                             const uint32_t *__restrict__ first, Grid g, TileItem *items, uint32_t *nitems)
{
    const long long f = *first, cnt = *dn;
    const long long ni = cnt > f ? (cnt - f + kChunk - 1) / kChunk : 0;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x, nt = (long long)gridDim.x * blockDim.x;
    if (t0 == 0) *nitems = (uint32_t)ni;
    for (long long k = t0; k < ni; k += nt) {
        TileItem m;
        m.start = (int)(f + k * kChunk);
        m.count = (int)min((long long)kChunk, cnt - m.start);
        m.pad = 0;
        const uint32_t c = cell[m.start + m.count / 2];
        m.tile = 0;
        if (c != kDead) {
            int a, b, d;
            unpack_cell(g, c, a, b, d);
            m.tile = (int)tile_of(g, a, b, d);
        }
        items[k] = m;
    }
}

size_t tail_items_capacity(long long cap) { return (size_t)((cap + kChunk - 1) / kChunk + 1); }

void launch_tail_items(const PartF32 &P, const uint32_t *first, const Grid &g, TileItem *items, uint32_t *nitems,
                       cudaStream_t st)
{
    static int nsm = 0;
    if (!nsm) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    }
    note_launch();
    k_tail_items<<<nsm * 4, 256, 0, st>>>(P.cell, P.dn, first, g, items, nitems);
}

void launch_photon_resolve(const QedParams &q, const PartF32 &P, int *err, cudaStream_t st)
{
    if (!q.on || !q.net || !q.cq) return;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_photon_resolve, cudaFuncAttributeMaxDynamicSharedMemorySize, kMlpStageBytes);
        attr = true;
    }
    static int nsm = 0;
    if (!nsm) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    }
    note_launch();
    k_photon_resolve<<<nsm, 256, kMlpStageBytes, st>>>(q, P, err);
}

}  // namespace pic
