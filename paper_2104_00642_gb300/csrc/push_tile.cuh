// push_tile.cuh -- tiled 2D push (push_tile.cu) and its work items.
#pragma once
#include "push.cuh"
#include "sort.cuh"

namespace pic {

struct QedParams;

constexpr int kChunk = 384;        // particles per work item at most
constexpr int kTileThreads = 128;  // threads per CTA of the tiled push
constexpr int kTileMinBlocks = 6;  // CTAs per SM: 80 registers, 35 KB shared memory each (measured best)

struct TileItem {
    int tile, start, count, pad;
};

// 3D items (the 3D push stages no particle state; 256 measured best among
// 256-1024 on the 8-ppc thermal workload: smaller items balance the CTAs)
constexpr int kChunk3 = 256;

size_t tile_items_capacity(long long cap, long long ntiles, int dim);
void build_tile_items(const uint32_t *starts, long long ntiles, int dim, uint32_t *cnt_scratch,
                      uint32_t *scan_scratch, TileItem *items, uint32_t *nitems, cudaStream_t st);
bool tile_push_supported(const Grid &g, int tile_edge);
// (agg: the warp-aggregated deposit, lanes on consecutive particles;
// q: a QED lepton species' Monte Carlo, fused in (lane-strided, agg
// ignored) -- nullptr or q->on == 0 for none; the particles appended since
// the sort, and their event flags, are left to launch_push_qed_f32)
void launch_push_tile2d(const PartF32 &P, const TileItem *items, const uint32_t *nitems, long long max_items,
                        float *F, const Grid &g, const PushConst &pc, int *err, double *e_abs, cudaStream_t st,
                        bool agg, const QedParams *q = nullptr);
// the tiled photon push (2D, FP32; tiles of 8 or 16 cells): the photons of
// the work items, their pair Monte Carlo with q; the photons appended since
// the sort are left to launch_push_photon_f32
void launch_push_photon_tile2d(const PartF32 &P, const TileItem *items, const uint32_t *nitems, long long max_items,
                               const float *F, const Grid &g, const PushConst &pc, const QedParams &q, int *err,
                               cudaStream_t st);
// 2D photons: work items over the photons appended since the sort ([*first,
// *P.dn), kChunk each)
size_t tail_items_capacity(long long cap);
void launch_tail_items(const PartF32 &P, const uint32_t *first, const Grid &g, TileItem *items, uint32_t *nitems,
                       cudaStream_t st);
// the surrogate's candidate conversions queued by the tiled photon push (q.cq)
void launch_photon_resolve(const QedParams &q, const PartF32 &P, int *err, cudaStream_t st);
// 3D: tiles of 4^3 cells, every n_d a multiple of 4
bool tile3d_push_supported(const Grid &g);
// (defer: a list of capacity >= the particle count, ndefer its device count;
// the particles the tiled kernel defers are pushed after it on the global
// path.  q: a QED lepton species' Monte Carlo, fused in -- nullptr or
// q->on == 0 for none; nothing is deferred then, and the particles appended
// since the sort are left to launch_push_qed_f32)
void launch_push_tile3d(const PartF32 &P, const TileItem *items, const uint32_t *nitems, long long max_items,
                        float *F, const Grid &g, const PushConst &pc, int *err, double *e_abs, uint32_t *defer,
                        uint32_t *ndefer, cudaStream_t st, const QedParams *q = nullptr);

}  // namespace pic
