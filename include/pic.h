/*
 * pic.h -- C ABI of the GB300 (sm_103a) relativistic electromagnetic
 * particle-in-cell hot path.
 *
 * The method is the PIC step of Song, Wang & Li, "YUNIC: A Multi-Dimensional
 * Particle-In-Cell Code for Laser-Plasma Interaction" (arXiv:2104.00642):
 * Yee FDTD field update (Sec. II.B, Eqs. (9)-(10)), Boris pusher (Sec. II.C,
 * Eqs. (11)-(16)), field interpolation with the W_2 weights (Sec. II.D,
 * Eqs. (17), (19)), Esirkepov charge-conserving current (Sec. II.E,
 * Eqs. (20)-(22)), in the split step that keeps fields and positions at both
 * integer and half steps (Sec. II.F).
 *
 * Units are the normalised units of Eq. (8): c = m_e = e = 1; time in
 * 1/omega_r, length in c/omega_r, E and B in m_e c omega_r/e, momentum per
 * mass u = gamma v, density in n_r, current in c e n_r.  In these units
 * div E = rho and dE/dt = curl B - J.
 *
 * Conventions shared by every call:
 *  - All compute runs in the library's CUDA kernels on the stream given at
 *    creation (NULL = the legacy default stream).  There is no CPU fallback:
 *    a call made without a usable GPU returns PIC_ERR_CUDA.
 *  - Calls return PIC_OK (0) or a negative PIC_ERR_* code; the message of the
 *    last failure is available from pic_last_error().
 *  - Host arrays passed in are caller-owned and only read during the call;
 *    host arrays passed out are caller-allocated and filled.
 *  - Field arrays exchanged with the host are FP64, x fastest, covering
 *    cells [0, N_d) along periodic axes and nodes [0, N_d] along absorbing
 *    axes (so every component has the same shape).  A component stored at
 *    node i or half node i+1/2 is exchanged at index i (standard Yee
 *    placement: Ex(i+1/2,j,k), Ey(i,j+1/2,k), Ez(i,j,k+1/2), Bx(i,j+1/2,k+1/2),
 *    By(i+1/2,j,k+1/2), Bz(i+1/2,j+1/2,k); J like E; RHO on nodes).
 *  - One pic_sim must not be used from two host threads at once.
 */
#ifndef PIC_H
#define PIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pic_sim pic_sim;

enum {
    PIC_OK = 0,
    PIC_ERR_ARG = -1,      /* invalid argument */
    PIC_ERR_CFL = -2,      /* dt above the Courant limit, or a particle moved more than one cell */
    PIC_ERR_CUDA = -3,     /* CUDA runtime/driver failure (message says which) */
    PIC_ERR_CAPACITY = -4, /* species capacity exceeded */
    PIC_ERR_NONFINITE = -5,/* NaN/Inf found in a particle or a diagnostic */
    PIC_ERR_NOMEM = -6,    /* device allocation failed */
    PIC_ERR_STATE = -7,    /* call not valid in the current state */
    PIC_ERR_TIMEOUT = -8   /* a bounded wait inside a kernel ran out (a bulk copy into shared memory or a
                              tensor-core commit did not complete); the kernel stopped, the context stays
                              usable, the step's results are not valid */
};

enum { PIC_BC_PERIODIC = 0, PIC_BC_ABSORB = 1 };
enum { PIC_PREC_FP32_CELLOFF = 0, PIC_PREC_FP64_PLAIN = 1 };
enum { PIC_EX = 0, PIC_EY, PIC_EZ, PIC_BX, PIC_BY, PIC_BZ, PIC_JX, PIC_JY, PIC_JZ, PIC_RHO };
enum { PIC_LASER_LINEAR_Y = 0, PIC_LASER_CIRCULAR = 1 };

#define PIC_MAX_SPECIES 8

/* Grid.  dim in {1,2,3}; n[d] cells and dx[d] spacing along active axes
 * (entries for inactive axes are ignored).  bc[d] applies to both faces of
 * axis d.  order is the shape order of Sec. II.D (Eqs. (17), (18)): 2 (the
 * three-node W_2 weights) or 4 (the five-node W_4, a 7-node Esirkepov
 * window; the push runs on the one-thread-per-particle kernels, and the QED
 * Monte Carlo needs order 2).  Periodic axes need n[d] >= 8. */
typedef struct {
    int dim;
    int64_t n[3];
    double dx[3];
    int bc[3];
    int order;
} pic_grid;

/* Species.  q in e, m in m_e, w = density carried by one macro-particle (in
 * n_r, the same for all particles of the species; a uniform density n with
 * ppc particles per cell has w = n/ppc).  capacity = maximum particle count
 * (created photons and pairs are appended up to it).  kind: PIC_KIND_MASSIVE
 * or PIC_KIND_PHOTON (q = 0, m = 0: moves at c along u, deposits no current).
 * qed: 1 if a massive species emits photons (nonlinear Compton, Sec. IV). */
typedef struct {
    double q, m, w;
    int64_t capacity;
    int kind;
    int qed;
} pic_species;

enum { PIC_KIND_MASSIVE = 0, PIC_KIND_PHOTON = 1 };

/* Device allocator a caller may hand the library (pic_options.alloc/free):
 * alloc returns a device block of `bytes` bytes aligned to 256 bytes (NULL
 * on failure), usable on `stream` (the simulation's cudaStream_t); free
 * releases a block alloc returned.  ctx is passed through unchanged. */
typedef void *(*pic_alloc_fn)(void *ctx, size_t bytes, void *stream);
typedef void (*pic_free_fn)(void *ctx, void *ptr, void *stream);

/* Options.  struct_size: sizeof(pic_options) as the caller compiled it
 * (pic_create rejects sizes it does not know, so a caller built against
 * another version of this header gets PIC_ERR_ARG instead of a misread
 * struct); zero-initialise the struct and set the fields you need.
 * precision: PIC_PREC_FP32_CELLOFF (int cell + FP32 in-cell offset, FP32
 * fields and push) or PIC_PREC_FP64_PLAIN (absolute FP64 positions and FP64
 * everything).  sort_interval: counting-sort particles by tile every K
 * steps (K >= 1; 0 = never after loading).  tile[d]: cells per tile along
 * active axes (powers of two, 0 = library default).  rho_bg: uniform
 * immobile background charge density used only by the Gauss diagnostic.
 * stream: a cudaStream_t (NULL = legacy default stream).  alloc/free: the
 * caller's device allocator (both or neither; NULL = cudaMalloc/cudaFree):
 * every device block the library uses for this simulation -- the state
 * pic_create allocates, and the temporary blocks of calls such as
 * pic_get_particles -- comes from it, and pic_destroy returns the state's
 * blocks to it. */
typedef struct {
    int struct_size;
    int precision;
    int sort_interval;
    int tile[3];
    double rho_bg;
    void *stream;
    int push_variant; /* PIC_PUSH_AUTO, PIC_PUSH_SIMPLE (one thread per particle, global atomics) or
                         PIC_PUSH_MLP_TC (as AUTO, but the surrogate of the photon push evaluated per
                         CTA on the tcgen05 tensor cores instead of per warp with mma.sync) */
    uint64_t seed;    /* key of the Philox4x32-10 stream of the QED Monte Carlo */
    int pusher;       /* momentum update: PIC_PUSHER_BORIS (Eqs. 13-16) or PIC_PUSHER_VAY (the
                         alternative Sec. II.C names after Eq. 16 for nearly cancelling E and v x B) */
    pic_alloc_fn alloc;
    pic_free_fn free;
    void *alloc_ctx;
} pic_options;

/* Push kernels: AUTO uses the tiled shared-memory kernel wherever it exists
 * (2D grids, FP32 form, 8x8 or 16x16 tiles, particles sorted at least once)
 * and the simple kernel elsewhere; SIMPLE always uses the simple kernel;
 * TILE_AGG is AUTO with the 2D tiled kernel's warp-aggregated deposit (the
 * lanes of a warp on consecutive, cell-sorted particles; lanes sharing a
 * deposit window summed by warp reductions before one atomic per value). */
enum { PIC_PUSH_AUTO = 0, PIC_PUSH_SIMPLE = 1, PIC_PUSH_MLP_TC = 2, PIC_PUSH_TILE_AGG = 3 };
enum { PIC_PUSHER_BORIS = 0, PIC_PUSHER_VAY = 1 };

/* Laser entering through the x-min face (requires bc[0] == PIC_BC_ABSORB):
 * paraxial Gaussian beam of peak amplitude a0 (normalised field), waist
 * radius `waist`, focus at x = x_focus, centred at (yc, zc), Gaussian
 * intensity envelope of full width at half maximum `fwhm` whose peak crosses
 * x = 0 at t_peak.  pol: linear along y or circular (both components of
 * amplitude a0).  It enters through the scattered-field Mur condition on the
 * x-min face (the paper uses absorbing faces and lasers from the left
 * boundary, Sec. III(a), without giving the method). */
typedef struct {
    double a0, waist, fwhm, t_peak, x_focus, yc, zc;
    int pol;
} pic_laser;

/* Diagnostics at the current integer step (FP64, Sec. II.B and Eq. (1)).
 * U_E = 1/2 sum E^2 dV and U_B = 1/2 sum B^2 dV over cells [0,N);
 * U_kin[s] = sum_p w m (gamma-1) dV; charge = sum_p q w dV + rho_bg * volume;
 * gauss_max = max over nodes [0,N) of |div E - rho - rho_bg| with rho the
 * particle density averaged over x -/+ (dt/2) v (conserved to round-off by
 * the charge-conserving deposit after the first step); E_absorbed = kinetic
 * energy removed at absorbing faces; n_alive[s] = live particles. */
typedef struct {
    int64_t step;
    double t;
    double U_E, U_B;
    double U_kin[PIC_MAX_SPECIES]; /* photons: sum_p w |k| dV */
    double charge;
    double gauss_max;
    double E_absorbed;
    int64_t n_alive[PIC_MAX_SPECIES];
    double E_photon_lost; /* energy of emitted photons below photon_emin */
} pic_diag;

/* QED Monte Carlo (Sec. IV) in the optical-depth form of Method I: every
 * emitting particle carries an optical depth tau (FP64) drawn as -ln r; each
 * step tau -= W dt with W the total rate of Eq. (23) (or (24) for photons) at
 * the particle's quantum parameter chi; when tau <= 0 the event happens, the
 * energy fraction comes from the inverse CDF of the spectrum at a Philox
 * draw, and tau restarts.  Draws: Philox4x32-10 with key = seed, counter =
 * (id_lo, id_hi, step, purpose).  Emitted photons go to photon_sp (collinear,
 * energy u gamma; the emitter recoils to gamma (1-u)); converting photons
 * create an electron in electron_sp and a positron in positron_sp (fractions
 * 1-v and v, collinear).  Particle identities: (species << 48) | load index.
 * lambda_r_m: wavelength of the reference frequency (2 pi c / omega_r, in
 * metres), which sets E_s = m c^2 / (hbar omega_r).  The FP32 form reads
 * the FP32 copy of the tables, the FP64 form the FP64 copy.
 * PIC_QED_SURROGATE (FP32 form; the FP64 form keeps its tables): as
 * PIC_QED_TABLE, but inside the chi range of a trained (or set) network the
 * rate and the energy fraction come from that network (pic_mlp_train); a
 * process without a network uses its tables. */
enum { PIC_QED_OFF = 0, PIC_QED_TABLE = 1, PIC_QED_SURROGATE = 2 };
enum { PIC_QED_EMISSION = 0, PIC_QED_PAIR = 1 };
/* Sampling method (Sec. IV): METHOD1 (0 also) is Method I in the optical-
 * depth form above.  METHOD2 is Method II: every step an emitter draws
 * r1, r2 and emits u0 = r1^3 when r2 < 3 r1^2 (dW_rad/du)(u0) dt; a photon
 * converts with v0 = r1 when r2 < (dW_pair/dv)(v0) dt (the pair spectrum is
 * bounded, so v0 is drawn uniform -- the paper applies the methods to pairs
 * "in the similar way"); no optical depth and no tables of the total rates
 * or inverse CDFs: the differential rates of Eqs. (23)/(24) are evaluated
 * from tables of K_{2/3} and Int K_{1/3}, so chi is not limited to the
 * tables' range.  An acceptance probability above one makes pic_step
 * return PIC_ERR_CFL (dt too long for the method).  Not with SURROGATE. */
enum { PIC_QED_METHOD1 = 1, PIC_QED_METHOD2 = 2 };
typedef struct {
    int mode;
    int photon_sp, electron_sp, positron_sp; /* -1 = none */
    double lambda_r_m;
    double photon_emin;
    int method; /* PIC_QED_METHOD1 (or 0) or PIC_QED_METHOD2 */
} pic_qed;

/* Configure the QED Monte Carlo (builds the rate and inverse-CDF tables on
 * the first call).  Call before loading particles of QED species, so their
 * identities and optical depths are initialised.  Errors: PIC_ERR_ARG. */
int pic_set_qed(pic_sim *sim, const pic_qed *qed);

/* Evaluate what the Monte Carlo uses, for inspection: with r == NULL,
 * rate[i] = G(chi[i]) = Int_0^1 F (the total rate is
 * alpha E_s G / (sqrt3 pi gamma)); otherwise rate[i] = the energy fraction
 * whose CDF is r[i].  The device tables, or in PIC_QED_SURROGATE mode the
 * ready network inside its chi range.  process: PIC_QED_EMISSION or
 * PIC_QED_PAIR.  Host arrays of n values.  Errors: PIC_ERR_ARG,
 * PIC_ERR_STATE (no tables). */
int pic_qed_eval(pic_sim *sim, int process, int64_t n, const double *chi, const double *r, double *out);

/* ---------------------------------------------------------------------
 * Surrogate network for the QED Monte Carlo (the paper has none: its
 * Method I and II use the spectra of Eqs. (23)/(24) directly).  One network
 * per process, 2 -> 64 -> 64 -> 64 -> 2 with SiLU, BF16 weights and FP32
 * accumulation.  Inputs x0 = 2 (ln chi - ln chi_min) / ln(chi_max/chi_min) - 1
 * and x1 = 2 t - 1, with t = 1 - sqrt(1 - r) for emission and
 * t = sqrt(2 min(r, 1 - r)) for pairs (r: the CDF value).  Outputs
 * y0 = s = fraction^(1/3) at r (pairs: the fraction of min(r, 1 - r)) and
 * y1 = (ln G (+ 8/(3 chi) for pairs) - mu) / sd.  Parameters (FP32, 8642):
 *   W0[64][2] b0[64] W1[64][64] b1[64] W2[64][64] b2[64] W3[2][64] b3[2]
 * with W[out][in]; the device holds them rounded to BF16 (biases FP32).
 * --------------------------------------------------------------------- */
#define PIC_MLP_NPARAMS 8642
typedef struct {
    int64_t iterations;      /* Adam steps (0: 40000) */
    int64_t batch;           /* samples per step, a multiple of 128 (0: 16384) */
    double lr, lr_final;     /* cosine schedule from lr to lr_final (0: 1e-2, 1e-4) */
    double chi_min, chi_max; /* trained range (0: 1e-3..1e2 emission, 1e-1..1e2 pairs) */
    double rate_weight;      /* loss weight of the rate output (0: 4) */
    uint64_t seed;           /* Philox key of samples and initial weights */
    int keep;                /* 1: continue from the present parameters */
} pic_mlp_train_opts;

typedef struct {
    double loss;               /* loss of the last batch */
    double max_err_lnG;        /* max |ln G_net - ln G_table| on the validation grid */
    double max_err_s, rms_err_s; /* |s_net - s_table| on the validation grid */
    double ms;                 /* device time of the training loop */
    int64_t iterations;
    int64_t table_bytes;       /* device bytes of one process's tables (FP32 + FP64) */
    int64_t net_bytes;         /* device bytes of the network the push reads */
    double max_err_mean;       /* max over the grid's chi rows of |<f>_net / <f>_table - 1|, <f> the
                                  mean energy fraction of an event (the energy an event carries) */
} pic_mlp_report;

typedef struct {
    double chi_min, chi_max; /* trained range */
    double mu, sd;           /* rate output normalisation */
} pic_mlp_info;

/* Train the network of `process` on the device with the library's own
 * kernels (forward, backward, Adam; one CUDA graph per iteration): each step
 * draws a fresh batch of (ln chi uniform in the range, r uniform; for
 * emission half the rows take r = 1 - (1 - t)^2 with t uniform instead, which
 * samples the hard end of the spectrum as densely as the soft end) and takes
 * the targets from the FP64 tables.  Then validates the network against the
 * tables on a 256 x 256 grid of cell midpoints in (ln chi, r) and marks it
 * ready.  Needs pic_set_qed first (the tables).  report may be NULL.
 * Errors: PIC_ERR_ARG, PIC_ERR_STATE, PIC_ERR_NOMEM, PIC_ERR_CUDA. */
int pic_mlp_train(pic_sim *sim, int process, const pic_mlp_train_opts *opt, pic_mlp_report *report);

/* Validation of the present network only (report->loss, ms, iterations 0). */
int pic_mlp_validate(pic_sim *sim, int process, pic_mlp_report *report);

/* Read (params: PIC_MLP_NPARAMS floats, FP32 master copy) or replace the
 * network of `process`; either pointer may be NULL on read.  pic_mlp_set
 * marks the network ready.  Errors: PIC_ERR_ARG, PIC_ERR_STATE (get: no
 * network), PIC_ERR_NOMEM, PIC_ERR_CUDA. */
int pic_mlp_get(pic_sim *sim, int process, float *params, pic_mlp_info *info);
int pic_mlp_set(pic_sim *sim, int process, const float *params, const pic_mlp_info *info);

/* The raw network on n normalised input rows x[n][2] -> y[n][2] (host
 * arrays), through the warp-level inference path the push uses. */
int pic_mlp_eval(pic_sim *sim, int process, int64_t n, const float *x, float *y);

/* The same evaluation batched on the fifth-generation tensor cores: CTAs of
 * 128 threads, one row per thread, the two 64 x 64 hidden layers as tcgen05
 * MMAs (M = 128, N = 64, K = 16 slices) with FP32 accumulators in tensor
 * memory.  The input layer, SiLU, BF16 activations and head are those of
 * pic_mlp_eval: the results differ only by the order of the FP32 sums.
 * x, y as for pic_mlp_eval; PIC_ERR_TIMEOUT if the tensor cores time out. */
int pic_mlp_eval_tc(pic_sim *sim, int process, int64_t n, const float *x, float *y);

/* Loss L = (1/n) sum_rows sum_o (y_o - t_o)^2 and its gradient with respect
 * to every parameter (grad: PIC_MLP_NPARAMS floats) at the present
 * parameters, by the training kernels (BF16 forward, backward on the tensor
 * cores, FP32 weight gradients).  n a multiple of 32, at most 1048576.
 * Errors: PIC_ERR_ARG, PIC_ERR_STATE, PIC_ERR_NOMEM, PIC_ERR_CUDA. */
int pic_mlp_grad(pic_sim *sim, int process, int64_t n, const float *x, const float *t, float *grad, double *loss);

/* Copy the identities and optical depths of a QED species (photon or
 * emitting species) in the current array order to caller-sized host arrays
 * (either may be NULL).  Errors: PIC_ERR_ARG, PIC_ERR_CAPACITY. */
int pic_get_qed_state(pic_sim *sim, int sp, int64_t cap, uint64_t *id, double *tau);

/* Create a simulation: validates the grid, the Courant condition
 * dt < 1/sqrt(sum_d 1/dx_d^2), species and options, allocates all device
 * memory (fields with ghost layers, double-buffered particle arrays, sort
 * and reduction scratch) and zeroes the fields.  *out is NULL on failure.
 * Errors: PIC_ERR_ARG, PIC_ERR_CFL, PIC_ERR_NOMEM, PIC_ERR_CUDA. */
int pic_create(const pic_grid *grid, double dt, const pic_species *species, int nsp,
               const pic_options *opt, pic_sim **out);

/* Release every device and host resource of sim (NULL is accepted). */
void pic_destroy(pic_sim *sim);

/* Message of the last failed call on sim (or of the last failed pic_create
 * when sim is NULL).  Valid until the next call on the same sim. */
const char *pic_last_error(const pic_sim *sim);

/* Append n particles to species sp.  x, y, z: absolute FP64 positions in
 * [0, n_d dx_d) (arrays of inactive axes may be NULL); ux, uy, uz: u = gamma v.
 * Host arrays (pageable or pinned) are copied; positions are converted to
 * the precision layout on the GPU and the species is sorted by tile.
 * Errors: PIC_ERR_ARG (bad species, position outside the domain, non-finite
 * input), PIC_ERR_CAPACITY. */
int pic_load_particles(pic_sim *sim, int sp, int64_t n, const double *x, const double *y,
                       const double *z, const double *ux, const double *uy, const double *uz);

/* Set the x-min laser (see pic_laser).  Errors: PIC_ERR_ARG. */
int pic_set_laser(pic_sim *sim, const pic_laser *laser);

/* Overwrite field component comp (PIC_EX..PIC_JZ) from a host FP64 array in
 * the exchange layout above; ghost layers are refreshed.  Errors: PIC_ERR_ARG. */
int pic_set_field(pic_sim *sim, int comp, const double *host_in);

/* Advance nsteps steps of the split PIC step (Sec. II.F): half E and B
 * updates, gather + Boris + drift + Esirkepov deposit for every live
 * particle, current fold, half B and E updates; counting sort by tile every
 * sort_interval steps.  Enqueued on the stream; returns after checking the
 * device error flags (one device->host read per call).
 * Errors: PIC_ERR_CFL (a particle crossed more than one cell),
 * PIC_ERR_NONFINITE (a particle momentum became NaN or infinite),
 * PIC_ERR_CAPACITY (QED children beyond a species' capacity; the excess is
 * not stored), PIC_ERR_TIMEOUT, PIC_ERR_CUDA. */
int pic_step(pic_sim *sim, int64_t nsteps);

/* Copy component comp (PIC_EX..PIC_JZ, or PIC_RHO = particle charge density
 * as in pic_diag) to host_out in the exchange layout.  Synchronises the
 * stream.  Errors: PIC_ERR_ARG. */
int pic_fields(pic_sim *sim, int comp, double *host_out);

/* Borrowed device view of a resident field component (PIC_EX..PIC_JZ, the
 * arrays of Sec. II.B's Yee grid; RHO is not resident): the value at stored
 * index (i, j, k) -- exchange-layout index, see above; ghost layers from
 * lo[d] to hi[d] inclusive -- is element origin + i*stride[0] + j*stride[1]
 * + k*stride[2] of `data`, elem_bytes wide (4: FP32 form, 8: FP64 form).
 * The library keeps ownership: the caller reads it and neither writes nor
 * frees it.  The address stays valid until pic_destroy; the contents are
 * those after the work enqueued on the simulation's stream, and change with
 * the next pic_step, pic_set_field or pic_restore (synchronise with pic_sync,
 * or order the reading stream after the simulation's).  Errors: PIC_ERR_ARG. */
typedef struct {
    void *data;
    int elem_bytes;
    int64_t origin;
    int64_t stride[3];
    int64_t lo[3], hi[3];
} pic_field_view;
int pic_field_device(pic_sim *sim, int comp, pic_field_view *view);

/* Checkpoint (the paper names no format; its code writes MPI-IO output,
 * Sec. II.F).  pic_save writes the whole simulation state to a file at path:
 * step, fields and currents with their ghost layers, every species' live
 * particles in array order (cell/offset or position, momentum, QED optical
 * depth and identity), the tile index of the last sort, the absorbed and
 * sub-threshold photon energy tallies, the laser, the QED set-up and the
 * surrogate networks.  pic_restore reads it into a simulation created with
 * the same grid, dt, species and options (else PIC_ERR_ARG): stepping on
 * from there takes the same decisions as the run that wrote it (identical
 * Philox counters and sort phase).  Both synchronise the stream.  The file
 * is host-endian raw binary with a version tag.  Errors: PIC_ERR_ARG (bad
 * path, unreadable or foreign file, other configuration), PIC_ERR_CUDA. */
int pic_save(pic_sim *sim, const char *path);
int pic_restore(pic_sim *sim, const char *path);

/* Number of live particles of species sp after the last sort (dead particles
 * are dropped at sorts; between sorts they are counted as not alive). */
int64_t pic_particle_count(pic_sim *sim, int sp);

/* Copy species sp to caller-sized host arrays (capacity cap >= count):
 * absolute FP64 positions and u, in the current array order; alive[i] = 0
 * for particles absorbed since the last sort.  Any pointer may be NULL.
 * *n receives the count.  Errors: PIC_ERR_ARG, PIC_ERR_CAPACITY. */
int pic_get_particles(pic_sim *sim, int sp, int64_t cap, int64_t *n, double *x, double *y,
                      double *z, double *ux, double *uy, double *uz, uint8_t *alive);

/* Device-resident particle state for inspection: packed cell index of each
 * particle (FP32 form: cell = i | j << bx | k << (bx+by), 0xFFFFFFFF = dead;
 * FP64 form: floor(x/dx) packed the same way), copied to host.  bits[3]
 * receives (bx, by, bz).  Errors: PIC_ERR_ARG, PIC_ERR_CAPACITY. */
int pic_get_cells(pic_sim *sim, int sp, int64_t cap, uint32_t *cells, int *bits);

/* Diagnostics of the current step (see pic_diag).  Runs FP64 reductions on
 * the GPU in a fixed order and synchronises the stream.
 * Errors: PIC_ERR_NONFINITE, PIC_ERR_CUDA. */
int pic_diagnostics(pic_sim *sim, pic_diag *d);

/* Gather E and B (Eq. (19)) at the current particle positions of species sp
 * without moving them; out6 receives 6*n FP64 values (Ex,Ey,Ez,Bx,By,Bz per
 * particle) in array order.  Errors: PIC_ERR_ARG, PIC_ERR_CAPACITY. */
int pic_gather(pic_sim *sim, int sp, int64_t cap, double *out6);

/* Synchronise the simulation's stream. */
int pic_sync(pic_sim *sim);

/* Phases of pic_step timed by pic_profile. */
enum { PIC_PHASE_SORT = 0, PIC_PHASE_FIELDS, PIC_PHASE_PUSH, PIC_PHASE_FOLD, PIC_NPHASE };

/* Enable (1) or disable (0) per-phase timing of pic_step: CUDA events are
 * recorded on the simulation's stream around each phase (no host
 * synchronisation inside the step).  Enabling clears the accumulators. */
int pic_profile(pic_sim *sim, int enable);

/* Read the accumulated device time of each phase in milliseconds
 * (ms[PIC_NPHASE], may be NULL), the kernel launches pic_step issued per
 * phase (launches[PIC_NPHASE], may be NULL) and the number of push-kernel
 * launches (push_launches, may be NULL) since profiling was enabled.
 * Synchronises the stream and clears the accumulators. */
int pic_profile_read(pic_sim *sim, double *ms, int64_t *launches, int64_t *push_launches);

/* The push phase split by species: device time in milliseconds of each
 * species' push (gather, push, deposit and its QED Monte Carlo; ms[nsp]) and
 * the number of such pushes (pushes[nsp]) timed up to the last
 * pic_profile_read (which gathers them); clears them.  Either pointer may be
 * NULL. */
int pic_profile_read_species(pic_sim *sim, double *ms, int64_t *pushes);

/* Field energy without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc (for example a plugin inside a host application that owns all
 * device memory through its own pool, or a real-time loop that must not
 * allocate), who therefore cannot create a pic_sim.
 *
 * dev_fields: host array of six device pointers (Ex, Ey, Ez, Bx, By, Bz),
 * each to n caller-owned FP64 values (any layout, e.g. the exchange layout
 * of pic_fields).  dev_out2: caller-owned device pointer to two doubles that
 * receive dV/2 * sum(Ex^2+Ey^2+Ez^2) and dV/2 * sum(Bx^2+By^2+Bz^2), summed
 * in FP64 in a fixed order.  stream: a cudaStream_t (NULL = legacy default);
 * the call only enqueues work on it.
 *
 * Scratch: the per-block partial sums live in a static device array of
 * 4096 x 2 doubles (64 KiB) that every GPU loading the library holds until
 * the process exits; n may be at most 67,108,864 (4096 blocks x 16384
 * elements), larger n returns PIC_ERR_ARG with a message.  The call makes no
 * cudaMalloc/cudaFree and calls no allocating library routine.  Its first
 * call on a device looks up the address of that array with
 * cudaGetSymbolAddress (with the device current); make that first call
 * before any stream capture.  The address is kept per device together with
 * the identifier of the CUDA context it was taken in; a call made in another
 * context of the device (after cudaDeviceReset, say) looks it up again, so
 * the first call after such a reset must also come before any capture.  Every call on a device shares the one array
 * and overwrites it completely (no state carries over between calls), so
 * calls that overlap on the GPU -- on two streams, or from two host threads
 * -- race and must be serialised by the caller.
 * Errors: PIC_ERR_ARG (null pointer, n out of range), PIC_ERR_CUDA; the
 * message is returned by pic_last_error(NULL). */
int pic_field_energy_noalloc(const double *const dev_fields[6], int64_t n, double dV, double *dev_out2,
                             void *stream);

/* Measurement, no counterpart in the paper: throughput ceilings of the
 * instruction mixes the push kernels are made of, on the current device
 * (each a timed kernel of independent chains over 8 CTAs of 256 threads per
 * SM): out[0] FP32 FMA flop/s, out[1] FP64 FMA flop/s, out[2] shared-memory
 * integer atomics per second with the 32 lanes of a warp on 32 words (the
 * lane-strided deposit), out[3] the same with the 32 lanes on one word,
 * out[4] lane values per second through a warp reduction over groups of 8
 * lanes plus one atomic per group (the warp-aggregated deposit).  out holds
 * 5 doubles (host).  Allocates 4 KiB of device memory for the duration of
 * the call; synchronises the device.  Errors: PIC_ERR_ARG, PIC_ERR_NOMEM,
 * PIC_ERR_CUDA. */
int pic_measure_ceilings(double *out);

#ifdef __cplusplus
}
#endif

#endif /* PIC_H */
