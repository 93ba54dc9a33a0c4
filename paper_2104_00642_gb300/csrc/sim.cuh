// sim.cuh -- the host-side state behind a pic_sim handle (capi.cu and
// checkpoint.cu): grid, species buffers, fields, QED and surrogate state,
// error flags and profiling marks; plus the error and allocation helpers
// every entry point uses.
#pragma once
#include <string>
#include <vector>

#include "../../include/pic.h"
#include "mlp_host.cuh"
#include "push.cuh"
#include "push_tile.cuh"
#include "qed_host.cuh"

namespace pic {

struct SpeciesState {
    double q = 0, m = 1, w = 0;
    long long cap = 0;
    long long n_hi = 0;        // host upper bound of the live count
    long long *d_count = nullptr;
    int cur = 0;
    uint32_t *cell[2] = {nullptr, nullptr};
    float *off[2][3] = {};
    float *uf[2][3] = {};
    double *x[2][3] = {};
    double *ud[2][3] = {};
    uint32_t *tile_start = nullptr;  // ntiles + 1
    // work items of the tiled push (rebuilt after every sort)
    TileItem *items = nullptr;
    uint32_t *nitems = nullptr;
    uint32_t *item_cnt = nullptr;   // ntiles + 1
    uint32_t *item_scan = nullptr;  // scan scratch
    uint32_t *defer = nullptr;      // 3D: particles the tiled push leaves to the global path ([0] = count)
    long long items_cap = 0;
    bool items_valid = false;
    // 2D photons: work items over the photons appended since the sort (rebuilt every step)
    TileItem *tail_items = nullptr;
    uint32_t *tail_nitems = nullptr;
    // QED: kind, optical depth and identity (double-buffered with the
    // particle arrays), event flags and data of the current step
    int kind = PIC_KIND_MASSIVE;
    int qed = 0;
    double *tau[2] = {nullptr, nullptr};
    uint64_t *id[2] = {nullptr, nullptr};
    uint32_t *ev = nullptr;
    float *evk = nullptr;
    bool has_qed_arrays() const { return tau[0] != nullptr; }
};

}  // namespace pic

struct pic_sim {
    pic::Grid g{};
    int precision = PIC_PREC_FP32_CELLOFF;
    int push_variant = PIC_PUSH_AUTO;
    int pusher = PIC_PUSHER_BORIS;
    // QED
    uint64_t seed = 0;
    pic_qed qed{};
    bool qed_on = false;
    void *qed_tables = nullptr;
    float4 *cand_q = nullptr;    // the photons' candidate conversions (surrogate form), one slot per photon
    long long cand_cap = 0;      // its slots
    uint32_t *cand_n = nullptr;
    pic::QedTables T{};
    double Es = 0.0;
    double *d_elost = nullptr;
    pic::MlpNet net[2];  // surrogate networks: emission, pairs
    pic::MlpScratch ms;  // their training scratch
    int sort_interval = 0;
    double rho_bg = 0.0;
    cudaStream_t st = nullptr;
    void *F = nullptr;       // 9 components
    double *rho = nullptr;   // padded, for diagnostics
    int nsp = 0;
    pic::SpeciesState sp[PIC_MAX_SPECIES];
    void *sort_scratch = nullptr;
    double *diag_scratch = nullptr;
    double *diag_out = nullptr;  // 16 doubles
    int *d_err = nullptr;
    double *d_eabs = nullptr;
    long long step = 0;
    pic::Laser laser{};
    pic_laser lp{};             // laser parameters (host)
    void *laser_prof = nullptr; // transverse profile arrays (device)
    std::vector<void *> allocs;
    // caller's device allocator (pic_options); NULL alloc = cudaMalloc/cudaFree
    pic_alloc_fn alloc_fn = nullptr;
    pic_free_fn free_fn = nullptr;
    void *alloc_ctx = nullptr;
    std::string err;
    // profiling
    bool prof = false;
    struct Mark {
        int phase;
        cudaEvent_t a, b;
    };
    std::vector<Mark> marks;
    long long prof_launch[PIC_NPHASE] = {0, 0, 0, 0};
    long long prof_push = 0;
    // per-species push (phase PIC_NPHASE + species in marks), accumulated
    // by pic_profile_read for pic_profile_read_species
    double prof_sp_ms[PIC_MAX_SPECIES] = {};
    long long prof_sp_n[PIC_MAX_SPECIES] = {};
    cudaEvent_t cur_a = nullptr;
    long long cur_l0 = 0;
};


namespace pic {

// record the message of a failed call (on sim, or for pic_last_error(NULL))
// and return code
int fail(pic_sim *s, int code, const char *fmt, ...);
// device memory owned by sim (released by pic_destroy), through the caller's
// allocator when one was given; PIC_ERR_NOMEM on failure
int dalloc(pic_sim *s, void **p, size_t bytes);
// temporary device memory of one call (released by tfree before it returns)
int talloc(pic_sim *s, void **p, size_t bytes);
void tfree(pic_sim *s, void *p);
inline size_t rsize(const pic_sim *s) { return s->precision == PIC_PREC_FP64_PLAIN ? 8 : 4; }

}  // namespace pic

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return pic::fail(s, PIC_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)
