// sort.cu -- stable counting sort of particles by tile (the tile holding a
// particle's cell) and, inside a tile, by cell (row-major within the tile),
// dead particles last, and the per-tile start offsets.  Cell order inside a
// tile puts the particles of one cell next to each other, so the lanes of a
// warp in the tiled push read the same field nodes and deposit into the
// same window.
//
// The sort is a least-significant-digit radix sort of (tile key, index)
// pairs with 8-bit digits.  Each pass is reduce-then-scan: per-block digit
// histograms (4096 keys per block), one device-wide exclusive scan of the
// (digit, block) counts, then a scatter in which every block walks its keys
// in order, 256 at a time, ranking equal digits with warp match masks and a
// per-warp prefix.  Every pass is stable, so the final permutation is the
// one a stable sort by key gives, independent of scheduling.
#include "scan_dev.cuh"
#include "sort.cuh"

namespace pic {

constexpr int kSortThreads = 256;
constexpr int kSortRounds = 16;
constexpr int kSortItems = kSortThreads * kSortRounds;  // keys per block

__global__ void k_make_keys(const uint32_t *__restrict__ cell, const long long *__restrict__ dn, long long n,
                            Grid g, uint32_t *key, uint32_t *val)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t c = i < *dn ? cell[i] : kDead;
    const int lb = g.tile_log2[0] + g.tile_log2[1] + g.tile_log2[2];  // bits of the cell within a tile
    uint32_t k;
    if (c == kDead) k = (uint32_t)g.ntiles << lb;
    else {
        int a, b, d;
        unpack_cell(g, c, a, b, d);
        const uint32_t local = (uint32_t)(a & ((1 << g.tile_log2[0]) - 1)) |
                               ((uint32_t)(b & ((1 << g.tile_log2[1]) - 1)) << g.tile_log2[0]) |
                               ((uint32_t)(d & ((1 << g.tile_log2[2]) - 1)) << (g.tile_log2[0] + g.tile_log2[1]));
        k = (tile_of(g, a, b, d) << lb) | local;
    }
    key[i] = k;
    val[i] = (uint32_t)i;
}

__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint32_t *__restrict__ kin, long long n,
                                                            int shift, uint32_t *counts, int nb)
{
    __shared__ uint32_t h[256];
    int tid = threadIdx.x;
    h[tid] = 0;
    __syncthreads();
    long long start = (long long)blockIdx.x * kSortItems;
    for (int r = 0; r < kSortRounds; r++) {
        long long i = start + r * kSortThreads + tid;
        if (i < n) atomicAdd(&h[(kin[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    counts[(long long)tid * nb + blockIdx.x] = h[tid];
}

__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(const uint32_t *__restrict__ kin,
                                                               const uint32_t *__restrict__ vin, uint32_t *kout,
                                                               uint32_t *vout, long long n, int shift,
                                                               const uint32_t *__restrict__ offs, int nb)
{
    __shared__ uint32_t base[256];
    __shared__ uint32_t wc[kSortThreads / 32][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    base[tid] = offs[(long long)tid * nb + blockIdx.x];
#pragma unroll
    for (int w = 0; w < kSortThreads / 32; w++) wc[w][tid] = 0;
    __syncthreads();
    const long long start = (long long)blockIdx.x * kSortItems;
    const unsigned lt = (1u << lane) - 1u;
    for (int r = 0; r < kSortRounds; r++) {
        long long i = start + r * kSortThreads + tid;
        bool valid = i < n;
        uint32_t k = valid ? kin[i] : 0u, v = valid ? vin[i] : 0u;
        uint32_t dg = valid ? ((k >> shift) & 255u) : 256u;
        unsigned peers = __match_any_sync(0xffffffffu, dg);
        uint32_t rank = __popc(peers & lt);
        if (valid && lane == __ffs(peers) - 1) wc[warp][dg] = __popc(peers);
        __syncthreads();
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kSortThreads / 32; w++) {
            uint32_t t = wc[w][tid];
            wc[w][tid] = run;
            run += t;
        }
        __syncthreads();
        if (valid) {
            uint32_t pos = base[dg] + wc[warp][dg] + rank;
            kout[pos] = k;
            vout[pos] = v;
        }
        __syncthreads();
        base[tid] += run;
#pragma unroll
        for (int w = 0; w < kSortThreads / 32; w++) wc[w][tid] = 0;
        __syncthreads();
    }
}

// ---------------------------------------------------------------------
// device-wide exclusive scan of u32 (reduce, scan of block sums, downsweep)
// ---------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_scan_reduce(const uint32_t *__restrict__ in, long long m, uint32_t *sums,
                                                     bool zero_end = false, const long long *__restrict__ dn = nullptr)
{
    if (zero_end && blockIdx.x == 0 && threadIdx.x == 0) sums[gridDim.x] = 0u;  // the slot that scans to the total
    if (dn && *dn < m) m = *dn < 0 ? 0 : *dn;  // words past the device count read as zero
    __shared__ uint32_t sh[32];
    long long b0 = (long long)blockIdx.x * kScanItems + threadIdx.x * 4;
    uint32_t s = 0;
#pragma unroll
    for (int q = 0; q < 4; q++)
        if (b0 + q < m) s += in[b0 + q];
    uint32_t tot;
    block_excl_scan_1024(s, sh, tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_down(const uint32_t *__restrict__ in, long long m, uint32_t *out,
                                                   const uint32_t *__restrict__ block_off)
{
    __shared__ uint32_t sh[32];
    long long b0 = (long long)blockIdx.x * kScanItems + threadIdx.x * 4;
    uint32_t v[4], s = 0;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        v[q] = b0 + q < m ? in[b0 + q] : 0u;
        s += v[q];
    }
    uint32_t tot;
    uint32_t run = block_excl_scan_1024(s, sh, tot) + (block_off ? block_off[blockIdx.x] : 0u);
#pragma unroll
    for (int q = 0; q < 4; q++) {
        if (b0 + q < m) out[b0 + q] = run;
        run += v[q];
    }
}

size_t scan_scratch_words(long long m)
{
    size_t w = 0;
    while (m > kScanItems) {
        m = (m + kScanItems - 1) / kScanItems;
        w += (size_t)m + 32;
    }
    return w + 32;
}

// the exclusive scan of the sums of in's blocks of kScanItems words:
// bsum[b] = sum of in[0, b kScanItems), bsum[nb] = the total (nb + 1 words,
// scratch past them as for scan_exclusive); dn (device, optional): the
// words from *dn on count as zero
void scan_block_sums(const uint32_t *in, long long m, uint32_t *bsum, uint32_t *scratch, cudaStream_t st,
                     const long long *dn)
{
    if (m <= 0) return;
    const long long nb = (m + kScanItems - 1) / kScanItems;
    note_launch();
    k_scan_reduce<<<(int)nb, 1024, 0, st>>>(in, m, bsum, true, dn);
    scan_exclusive(bsum, bsum, nb + 1, scratch, st);
}

long long scan_blocks(long long m) { return (m + kScanItems - 1) / kScanItems; }

// exclusive scan of m words, in may equal out
void scan_exclusive(const uint32_t *in, uint32_t *out, long long m, uint32_t *scratch, cudaStream_t st)
{
    if (m <= 0) return;
    if (m <= kScanItems) {
        note_launch();
        k_scan_down<<<1, 1024, 0, st>>>(in, m, out, nullptr);
        return;
    }
    long long nb = (m + kScanItems - 1) / kScanItems;
    uint32_t *sums = scratch;
    note_launch(2);
    k_scan_reduce<<<(int)nb, 1024, 0, st>>>(in, m, sums);
    scan_exclusive(sums, sums, nb, scratch + nb + 32, st);
    k_scan_down<<<(int)nb, 1024, 0, st>>>(in, m, out, sums);
}

__global__ void k_tile_starts(const uint32_t *__restrict__ skey, long long n, long long ntiles, int lb,
                              uint32_t *starts, long long *dcount)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    long long lo = i == 0 ? 0 : (long long)(skey[i - 1] >> lb) + 1;
    long long hi = i == n ? ntiles : (long long)(skey[i] >> lb);
    for (long long t = lo; t <= hi && t <= ntiles; t++) {
        starts[t] = (uint32_t)i;
        if (t == ntiles) *dcount = i;
    }
}

// ---------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------
size_t sort_scratch_bytes(long long cap)
{
    long long nb = (cap + kSortItems - 1) / kSortItems;
    size_t w = 4 * (size_t)cap + 256 * (size_t)nb + scan_scratch_words(256 * nb) + 256;
    return w * sizeof(uint32_t);
}

// 8-bit digits covering the largest key, (ntiles << lb) for the dead
int radix_passes(long long ntiles, int lb)
{
    int bits = 0;
    while ((1ll << bits) <= (ntiles << lb)) bits++;
    return (bits + 7) / 8;
}

// sorts the first n entries (entries at or past *dcount count as dead);
// returns the device pointer of the permutation (new -> old), the sorted
// keys, and updates starts[0..ntiles] and *dcount (live particles)
void sort_by_tile(const uint32_t *cell, long long n, const long long *dcount_in, const Grid &g, void *scratch,
                  uint32_t *starts, long long *dcount_out, const uint32_t **perm, const uint32_t **skeys,
                  cudaStream_t st)
{
    uint32_t *w = (uint32_t *)scratch;
    long long cap_n = n;
    uint32_t *kA = w, *kB = w + cap_n, *vA = w + 2 * cap_n, *vB = w + 3 * cap_n;
    long long nb = (n + kSortItems - 1) / kSortItems;
    uint32_t *counts = w + 4 * cap_n;
    uint32_t *sscr = counts + 256 * nb + 64;
    const int lb = g.tile_log2[0] + g.tile_log2[1] + g.tile_log2[2];
    if (n > 0) {
        note_launch(1 + 2 * radix_passes(g.ntiles, lb));
        k_make_keys<<<div_up(n, 256), 256, 0, st>>>(cell, dcount_in, n, g, kA, vA);
        int passes = radix_passes(g.ntiles, lb);
        for (int p = 0; p < passes; p++) {
            k_radix_hist<<<(int)nb, kSortThreads, 0, st>>>(kA, n, 8 * p, counts, (int)nb);
            scan_exclusive(counts, counts, 256 * nb, sscr, st);
            k_radix_scatter<<<(int)nb, kSortThreads, 0, st>>>(kA, vA, kB, vB, n, 8 * p, counts, (int)nb);
            uint32_t *t = kA; kA = kB; kB = t;
            t = vA; vA = vB; vB = t;
        }
    }
    note_launch();
    k_tile_starts<<<div_up(n + 1, 256), 256, 0, st>>>(kA, n, g.ntiles, lb, starts, dcount_out);
    *perm = vA;
    *skeys = kA;
}

// ---------------------------------------------------------------------
// apply the permutation to the particle arrays (new[i] = old[perm[i]])
// ---------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void mv(const T *s, T *d, uint32_t from, long long to)
{
    if (s) d[to] = s[from];
}

__global__ void k_permute_f32(PartF32 src, PartF32 dst, const uint32_t *__restrict__ perm,
                              const long long *__restrict__ dcount, int dim)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= *dcount) return;
    uint32_t a = perm[i];
    dst.cell[i] = src.cell[a];
    for (int d = 0; d < dim; d++) dst.off[d][i] = src.off[d][a];
    dst.u[0][i] = src.u[0][a];
    dst.u[1][i] = src.u[1][a];
    dst.u[2][i] = src.u[2][a];
    if (src.tau) {
        dst.tau[i] = src.tau[a];
        dst.id[i] = src.id[a];
    }
}

__global__ void k_permute_f64(PartF64 src, PartF64 dst, const uint32_t *__restrict__ perm,
                              const long long *__restrict__ dcount, int dim)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= *dcount) return;
    uint32_t a = perm[i];
    dst.cell[i] = src.cell[a];
    for (int d = 0; d < dim; d++) dst.x[d][i] = src.x[d][a];
    dst.u[0][i] = src.u[0][a];
    dst.u[1][i] = src.u[1][a];
    dst.u[2][i] = src.u[2][a];
    if (src.tau) {
        dst.tau[i] = src.tau[a];
        dst.id[i] = src.id[a];
    }
}

void launch_permute_f32(const PartF32 &src, const PartF32 &dst, const uint32_t *perm, const long long *dcount,
                        long long n, int dim, cudaStream_t st)
{
    if (n == 0) return;
    note_launch();
    k_permute_f32<<<div_up(n, 256), 256, 0, st>>>(src, dst, perm, dcount, dim);
}

void launch_permute_f64(const PartF64 &src, const PartF64 &dst, const uint32_t *perm, const long long *dcount,
                        long long n, int dim, cudaStream_t st)
{
    if (n == 0) return;
    note_launch();
    k_permute_f64<<<div_up(n, 256), 256, 0, st>>>(src, dst, perm, dcount, dim);
}

}  // namespace pic
