/*
 * pic_oracle.c -- plain, slow FP64 CPU oracle for the relativistic
 * electromagnetic particle-in-cell step of Song, Wang & Li, "YUNIC: A
 * Multi-Dimensional Particle-In-Cell Code for Laser-Plasma Interaction"
 * (arXiv:2104.00642).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the package smoke check and the
 * CPU-baseline leg of the benchmark load this library. It shares no code,
 * header, table or constant with the CUDA path and never calls it.
 *
 * Everything is FP64 with absolute particle positions and is compiled with
 * floating-point contraction off. Loops are written in the order of the
 * paper's equations; there is no blocking, fusion or reordering.
 *
 * Units: the normalised units of Eq. (8) (Sec. II.A): c = m_e = e = 1, time in
 * 1/omega_r, length in c/omega_r, fields in m_e c omega_r / e, densities in
 * n_r = m_e omega_r^2 / (4 pi e^2).  With these units the Gaussian 4*pi of
 * Eqs. (1) and (4) is absorbed: div E = rho, dE/dt = curl B - J.
 *
 * Step (Sec. II.E, the PSC/EPOCH split step that holds fields and positions at
 * both integer and half steps; the flow chart of Fig. 4 is not available, so
 * the order below is a reading of the text):
 *   1. E^{n+1/2} = E^n + (dt/2)(curl B^n - J^n)            [Eq. (9), half]
 *   2. B^{n+1/2} = B^n - (dt/2) curl E^{n+1/2}              [Eq. (10), half]
 *   3. per particle: x^{n+1/2} = x^n + (dt/2) u^n/gamma^n
 *      gather E, B at x^{n+1/2}                              [Eq. (19)]
 *      Boris u^n -> u^{n+1}                                  [Eqs. (13)-(16)]
 *      x^{n+1}   = x^{n+1/2} + (dt/2) u^{n+1}/gamma^{n+1}    [Eq. (12), half]
 *      x^{n+3/2} = x^{n+1}   + (dt/2) u^{n+1}/gamma^{n+1}
 *      Esirkepov J^{n+1} on the straight path x^{n+1/2} -> x^{n+3/2} [Eqs. (20)-(22)]
 *   4. B^{n+1} = B^{n+1/2} - (dt/2) curl E^{n+1/2}
 *   5. E^{n+1} = E^{n+1/2} + (dt/2)(curl B^{n+1} - J^{n+1})
 * Two consecutive steps give exactly the leapfrog of Eqs. (9)-(12).
 *
 * Yee placement (Fig. 1 is not available; standard Yee reading):
 *   Ex(i+1/2,j,k) Ey(i,j+1/2,k) Ez(i,j,k+1/2)   (J like E)
 *   Bx(i,j+1/2,k+1/2) By(i+1/2,j,k+1/2) Bz(i+1/2,j+1/2,k)
 * A value at node i or half node i+1/2 is addressed by the integer index i.
 *
 * Boundaries.  Periodic axes use modular indexing over [0, N).  On an
 * absorbing axis a node-centred component is physical on [0, N], a
 * half-node component on [0, N-1]; the tangential magnetic components also
 * keep one ghost at -1 and N, set by a first-order Mur condition applied to
 * the scattered field (the paper names absorbing boundaries without giving
 * the method, Sec. III(a)).  Reads outside the stored range are zero; current
 * deposited outside the physical range is discarded.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "pic_oracle.h"

enum { EX = 0, EY, EZ, BX, BY, BZ, JX, JY, JZ, NF };
/* BC_SLAB (test infrastructure for the domain decomposition of Sec. II.F):
 * the axis is one slab of a larger periodic grid; its SLAB_G ghost layers on
 * each side are stored and filled by the caller (neighbours' values), the
 * solver updates the slab's own nodes [0, N) only, deposits may land in the
 * ghosts (the caller sums them into the neighbours), and a particle whose
 * position leaves [0, L) is moved to its species' outbox (the caller hands
 * it to the neighbour) instead of being wrapped or absorbed.  Its QED event
 * of that step still happens; children born outside the slab go to their
 * species' outbox. */
enum { BC_PERIODIC = 0, BC_ABSORB = 1, BC_SLAB = 2 };
#define SLAB_G 4

/* ------------------------------------------------------------------ */
/* Sim state                                                           */
/* ------------------------------------------------------------------ */

typedef struct {
    double q, m, w;     /* charge (e), mass (m_e), density weight per macro-particle (n_r) */
    long n, cap;
    double *x;          /* 3*n absolute positions (L_r) */
    double *u;          /* 3*n momenta per mass, u = gamma v (photons: k in m c) */
    unsigned char *alive;
    uint64_t *id;
    int kind;           /* 0 massive, 1 photon (moves at c along k, no charge) */
    int qed;            /* massive species that emits photons */
    double *tau;        /* optical depth left (Sec. IV, Method I in optical-depth form) */
    /* BC_SLAB: particles that left the slab this step (x as computed, u, id, tau) */
    long nout, outcap;
    double *ox, *ou, *otau;
    uint64_t *oid;
} osp;

/* one QED event of the current step, kept for spawning in parent order */
typedef struct {
    long parent;
    double k[3];        /* photon momentum (emission) or converting photon's k */
    double frac;        /* pair: positron fraction v */
} oevent;

typedef struct {
    int on, pol;        /* pol 0: linear along y; 1: circular */
    double a0, waist, fwhm, t_peak, x_focus, yc, zc;
} olaser;

struct osim {
    int dim;
    long n[3];
    double dx[3];
    int bc[3];
    double dt;
    long lo[3], len[3];
    double *F[NF];
    double rho_bg;
    int nsp;
    osp sp[OR_MAX_SPECIES];
    long step;
    int sort_interval;
    int tile[3];
    int pusher; /* 0: Boris, 1: Vay */
    int order;  /* shape order of Sec. II.D: 2 (W_2, three nodes) or 4 (W_4, five nodes) */
    olaser L;
    double e_absorbed;
    /* QED */
    int qed_on, photon_sp, electron_sp, positron_sp;
    double Es, emin, e_lost;
    uint32_t key[2];
    int qed_method;     /* 1: Method I in the optical-depth form (default); 2: Method II */
    long m2_over;       /* Method II draws whose acceptance probability exceeded one */
    oevent *ev[OR_MAX_SPECIES];
    long nev[OR_MAX_SPECIES], evcap[OR_MAX_SPECIES];
};

static long imod(long a, long n) { long r = a % n; return r < 0 ? r + n : r; }

/* staggering of component c along axis d (1 = half node) */
static int stag(int c, int d)
{
    int base = c % 3;
    if (c >= BX && c <= BZ) return d != base;
    return d == base;
}

/* linear index of (i,j,k) in the storage of the grid, -1 if not stored */
static long lin(const osim *s, long i, long j, long k)
{
    long idx[3] = {i, j, k};
    long off = 0, stride = 1;
    for (int d = 0; d < 3; d++) {
        long v = idx[d];
        if (d >= s->dim) v = 0;
        else if (s->bc[d] == BC_PERIODIC) v = imod(v, s->n[d]);
        else if (v < s->lo[d] || v >= s->lo[d] + s->len[d]) return -1;
        off += (v - s->lo[d]) * stride;
        stride *= s->len[d];
    }
    return off;
}

static double getF(const osim *s, int c, long i, long j, long k)
{
    long l = lin(s, i, j, k);
    return l < 0 ? 0.0 : s->F[c][l];
}

/* physical (updated / deposit-receiving) position of component c */
static int phys(const osim *s, int c, long i, long j, long k)
{
    long idx[3] = {i, j, k};
    for (int d = 0; d < s->dim; d++) {
        if (s->bc[d] != BC_ABSORB) continue;
        long hi = stag(c, d) ? s->n[d] - 1 : s->n[d];
        if (idx[d] < 0 || idx[d] > hi) return 0;
    }
    return 1;
}

static void addF(osim *s, int c, long i, long j, long k, double v)
{
    if (!phys(s, c, i, j, k)) return;
    long l = lin(s, i, j, k);
    if (l >= 0) s->F[c][l] += v;
}

static long ncells_store(const osim *s) { return s->len[0] * s->len[1] * s->len[2]; }

osim *or_create(int dim, const long *n, const double *dx, const int *bc, double dt,
                double rho_bg, int sort_interval, const int *tile)
{
    if (dim < 1 || dim > 3) return NULL;
    osim *s = (osim *)calloc(1, sizeof(osim));
    s->dim = dim;
    s->dt = dt;
    s->rho_bg = rho_bg;
    s->sort_interval = sort_interval;
    s->order = 2;
    for (int d = 0; d < 3; d++) {
        int active = d < dim;
        s->n[d] = active ? n[d] : 1;
        s->dx[d] = active ? dx[d] : 1.0;
        s->bc[d] = active ? bc[d] : BC_PERIODIC;
        s->tile[d] = active ? (tile ? tile[d] : 8) : 1;
        if (!active) { s->lo[d] = 0; s->len[d] = 1; }
        else if (s->bc[d] == BC_PERIODIC) { s->lo[d] = 0; s->len[d] = s->n[d]; }
        else if (s->bc[d] == BC_SLAB) { s->lo[d] = -SLAB_G; s->len[d] = s->n[d] + 2 * SLAB_G; }
        else { s->lo[d] = -1; s->len[d] = s->n[d] + 2; }
    }
    for (int c = 0; c < NF; c++) s->F[c] = (double *)calloc((size_t)ncells_store(s), sizeof(double));
    return s;
}

void or_destroy(osim *s)
{
    if (!s) return;
    for (int c = 0; c < NF; c++) free(s->F[c]);
    for (int i = 0; i < s->nsp; i++) {
        free(s->sp[i].x); free(s->sp[i].u); free(s->sp[i].alive); free(s->sp[i].id); free(s->sp[i].tau);
        free(s->sp[i].ox); free(s->sp[i].ou); free(s->sp[i].otau); free(s->sp[i].oid);
        free(s->ev[i]);
    }
    free(s);
}

int or_add_species2(osim *s, double q, double m, double w, long cap, int kind, int qed)
{
    if (s->nsp >= OR_MAX_SPECIES) return -1;
    osp *p = &s->sp[s->nsp];
    p->q = q; p->m = m; p->w = w; p->cap = cap; p->n = 0;
    p->kind = kind; p->qed = qed;
    p->x = (double *)calloc((size_t)(3 * cap + 3), sizeof(double));
    p->u = (double *)calloc((size_t)(3 * cap + 3), sizeof(double));
    p->alive = (unsigned char *)calloc((size_t)cap + 1, 1);
    p->id = (uint64_t *)calloc((size_t)cap + 1, sizeof(uint64_t));
    p->tau = (double *)calloc((size_t)cap + 1, sizeof(double));
    s->ev[s->nsp] = (oevent *)calloc((size_t)cap + 1, sizeof(oevent));
    s->evcap[s->nsp] = cap + 1;
    return s->nsp++;
}

int or_add_species(osim *s, double q, double m, double w, long cap) { return or_add_species2(s, q, m, w, cap, 0, 0); }

/* -ln r of the Philox draw (id, step = 0xFFFFFFFF, purpose 2): the optical
 * depth a particle starts with */
static double initial_tau(const osim *s, uint64_t id)
{
    uint32_t c[4] = {(uint32_t)id, (uint32_t)(id >> 32), 0xFFFFFFFFu, 2u}, w[4];
    or_philox4x32_10(c, s->key, w);
    return -log(or_uniform24(w[0]));
}

void or_set_qed(osim *s, int photon_sp, int electron_sp, int positron_sp, double lambda_r_m, double emin,
                uint64_t seed)
{
    s->qed_on = 1;
    s->photon_sp = photon_sp;
    s->electron_sp = electron_sp;
    s->positron_sp = positron_sp;
    /* E_s = m c^2 / (hbar omega_r) = m c^2 lambda_r / (h c) */
    s->Es = 510998.95 * lambda_r_m / 1.239841984e-6;
    s->emin = emin;
    s->key[0] = (uint32_t)seed;
    s->key[1] = (uint32_t)(seed >> 32);
}

double or_Es(const osim *s) { return s->Es; }

/* QED sampling method: 1 (Method I, optical depth; default) or 2 (Method II) */
int or_set_qed_method(osim *s, int method)
{
    if (method != 1 && method != 2) return -1;
    s->qed_method = method;
    return 0;
}

long or_method2_over(const osim *s) { return s->m2_over; }

int or_load(osim *s, int isp, long n, const double *x, const double *y, const double *z,
            const double *ux, const double *uy, const double *uz)
{
    if (isp < 0 || isp >= s->nsp) return -1;
    osp *p = &s->sp[isp];
    if (p->n + n > p->cap) return -2;
    const double *xs[3] = {x, y, z};
    for (long a = 0; a < n; a++) {
        long b = p->n + a;
        for (int d = 0; d < 3; d++) p->x[3 * b + d] = (d < s->dim && xs[d]) ? xs[d][a] : 0.0;
        p->u[3 * b + 0] = ux[a];
        p->u[3 * b + 1] = uy[a];
        p->u[3 * b + 2] = uz[a];
        p->alive[b] = 1;
        p->id[b] = ((uint64_t)isp << 48) | (uint64_t)b;
        p->tau[b] = initial_tau(s, p->id[b]);
    }
    p->n += n;
    return 0;
}

/* identities given by the caller for particles [first, first + n) of a
   species (a sample of a larger load keeps the identities of that load);
   each optical depth restarts from its identity's initial draw */
int or_set_ids(osim *s, int isp, long first, long n, const uint64_t *id)
{
    if (isp < 0 || isp >= s->nsp) return -1;
    osp *p = &s->sp[isp];
    if (first < 0 || n < 0 || first + n > p->n) return -2;
    for (long a = 0; a < n; a++) {
        p->id[first + a] = id[a];
        p->tau[first + a] = initial_tau(s, id[a]);
    }
    return 0;
}

/* output box of a field: [0,N) on periodic axes, [0,N] on absorbing ones */
static void out_box(const osim *s, long *m)
{
    for (int d = 0; d < 3; d++)
        m[d] = d >= s->dim ? 1 : (s->bc[d] == BC_ABSORB ? s->n[d] + 1 : s->n[d]);
}

int or_get_field(const osim *s, int c, double *out)
{
    if (c < 0 || c >= NF) return -1;
    long m[3];
    out_box(s, m);
    for (long k = 0; k < m[2]; k++)
        for (long j = 0; j < m[1]; j++)
            for (long i = 0; i < m[0]; i++)
                out[(k * m[1] + j) * m[0] + i] = getF(s, c, i, j, k);
    return 0;
}

int or_set_field(osim *s, int c, const double *in)
{
    if (c < 0 || c >= NF) return -1;
    long m[3];
    out_box(s, m);
    for (long k = 0; k < m[2]; k++)
        for (long j = 0; j < m[1]; j++)
            for (long i = 0; i < m[0]; i++) {
                long l = lin(s, i, j, k);
                if (l >= 0) s->F[c][l] = in[(k * m[1] + j) * m[0] + i];
            }
    return 0;
}

/* ghost (Mur) values of the tangential B at -1 and N along an absorbing axis */
int or_get_ghost(const osim *s, int c, long i, long j, long k, double *v)
{
    long l = lin(s, i, j, k);
    if (l < 0) return -1;
    *v = s->F[c][l];
    return 0;
}

void or_set_laser(osim *s, int pol, double a0, double waist, double fwhm, double t_peak,
                  double x_focus, double yc, double zc)
{
    s->L.on = 1; s->L.pol = pol; s->L.a0 = a0; s->L.waist = waist; s->L.fwhm = fwhm;
    s->L.t_peak = t_peak; s->L.x_focus = x_focus; s->L.yc = yc; s->L.zc = zc;
}

/* ------------------------------------------------------------------ */
/* Field solver: Eqs. (9), (10) on the Yee grid                        */
/* ------------------------------------------------------------------ */

/* backward difference of component c along axis d at (i,j,k): (F[i]-F[i-1])/dx */
static double dback(const osim *s, int c, int d, long i, long j, long k)
{
    if (d >= s->dim) return 0.0;
    long a[3] = {i, j, k};
    a[d] -= 1;
    return (getF(s, c, i, j, k) - getF(s, c, a[0], a[1], a[2])) / s->dx[d];
}

/* forward difference: (F[i+1]-F[i])/dx */
static double dfwd(const osim *s, int c, int d, long i, long j, long k)
{
    if (d >= s->dim) return 0.0;
    long a[3] = {i, j, k};
    a[d] += 1;
    return (getF(s, c, a[0], a[1], a[2]) - getF(s, c, i, j, k)) / s->dx[d];
}

/* the index box the solver sweeps: [0,N) periodic, [0,N] absorbing */
static void sweep_box(const osim *s, long *m) { out_box(s, m); }

/* E += h (curl B - J)  (Eq. (9) over a time h) */
static void update_E(osim *s, double h)
{
    long m[3];
    sweep_box(s, m);
    for (long k = 0; k < m[2]; k++)
        for (long j = 0; j < m[1]; j++)
            for (long i = 0; i < m[0]; i++) {
                /* dEx/dt = dBz/dy - dBy/dz - Jx, etc.; B is half-staggered so
                 * its derivative at an E position is a backward difference */
                double cx = dback(s, BZ, 1, i, j, k) - dback(s, BY, 2, i, j, k);
                double cy = dback(s, BX, 2, i, j, k) - dback(s, BZ, 0, i, j, k);
                double cz = dback(s, BY, 0, i, j, k) - dback(s, BX, 1, i, j, k);
                long l = lin(s, i, j, k);
                if (phys(s, EX, i, j, k)) s->F[EX][l] += h * (cx - s->F[JX][l]);
                if (phys(s, EY, i, j, k)) s->F[EY][l] += h * (cy - s->F[JY][l]);
                if (phys(s, EZ, i, j, k)) s->F[EZ][l] += h * (cz - s->F[JZ][l]);
            }
}

/* laser field at the x-min face (x = 0) at time t and transverse (y, z):
 * paraxial Gaussian beam focused at x_focus, Gaussian intensity envelope
 * with full width at half maximum fwhm, peak crossing x = 0 at t_peak.
 * out[0] = E_y, out[1] = E_z. */
static void laser_field(const osim *s, double t, double y, double z, double *out)
{
    const olaser *L = &s->L;
    double r2 = 0.0, amp = 1.0, wxi = 1.0, rinv = 0.0, gouy = 0.0;
    if (s->dim >= 2) {
        double xr = 0.5 * L->waist * L->waist; /* Rayleigh length, k = 1 */
        double xi = -L->x_focus;
        wxi = L->waist * sqrt(1.0 + (xi / xr) * (xi / xr));
        rinv = xi / (xi * xi + xr * xr);
        gouy = atan(xi / xr);
        r2 = (y - L->yc) * (y - L->yc);
        if (s->dim == 3) r2 += (z - L->zc) * (z - L->zc);
        amp = (s->dim == 3) ? L->waist / wxi : sqrt(L->waist / wxi);
        if (s->dim == 2) gouy *= 0.5;
    }
    double tau = (t - L->t_peak) / L->fwhm;
    double env = exp(-2.0 * log(2.0) * tau * tau);
    double trans = (s->dim >= 2) ? exp(-r2 / (wxi * wxi)) : 1.0;
    double ph = (t - L->t_peak) - 0.5 * r2 * rinv + gouy;
    double a = L->a0 * amp * trans * env;
    out[0] = a * sin(ph);
    out[1] = L->pol == 1 ? a * cos(ph) : 0.0;
}

/* incident B of the laser at distance xoff from the x-min face at time t:
 * a wave travelling in +x has Bz = Ey and By = -Ez. */
static double incident_B(const osim *s, int c, double xoff, double t, long j, long k)
{
    if (!s->L.on) return 0.0;
    double y = 0.0, z = 0.0;
    if (s->dim >= 2) y = (j + (stag(c, 1) ? 0.5 : 0.0)) * s->dx[1];
    if (s->dim >= 3) z = (k + (stag(c, 2) ? 0.5 : 0.0)) * s->dx[2];
    double e[2];
    laser_field(s, t - xoff, y, z, e);
    if (c == BZ) return e[0];
    if (c == BY) return -e[1];
    return 0.0;
}

/* B -= h curl E (Eq. (10) over a time h), then the Mur ghosts at time t_new */
static void update_B(osim *s, double h, double t_new)
{
    long m[3];
    sweep_box(s, m);
    long nst = ncells_store(s);
    int any_abs = 0;
    for (int d = 0; d < s->dim; d++) any_abs |= s->bc[d] == BC_ABSORB;
    double *old[3] = {NULL, NULL, NULL};
    if (any_abs)
        for (int c = 0; c < 3; c++) {
            old[c] = (double *)malloc((size_t)nst * sizeof(double));
            memcpy(old[c], s->F[BX + c], (size_t)nst * sizeof(double));
        }
    for (long k = 0; k < m[2]; k++)
        for (long j = 0; j < m[1]; j++)
            for (long i = 0; i < m[0]; i++) {
                /* dBx/dt = -(dEz/dy - dEy/dz), etc.; forward differences */
                double cx = dfwd(s, EZ, 1, i, j, k) - dfwd(s, EY, 2, i, j, k);
                double cy = dfwd(s, EX, 2, i, j, k) - dfwd(s, EZ, 0, i, j, k);
                double cz = dfwd(s, EY, 0, i, j, k) - dfwd(s, EX, 1, i, j, k);
                long l = lin(s, i, j, k);
                if (phys(s, BX, i, j, k)) s->F[BX][l] -= h * cx;
                if (phys(s, BY, i, j, k)) s->F[BY][l] -= h * cy;
                if (phys(s, BZ, i, j, k)) s->F[BZ][l] -= h * cz;
            }
    if (!any_abs) return;
    /* Mur first-order absorbing condition on the scattered field s = B - B_inc:
     * an outgoing wave obeys (d/dt -+ d/dx) s = 0; centring that at the face
     * between ghost and first inner value gives
     *   s_g(new) = s_in(old) + (a-1)/(a+1) (s_in(new) - s_g(old)),  a = h/dx. */
    double t_old = t_new - h;
    for (int d = 0; d < s->dim; d++) {
        if (s->bc[d] != BC_ABSORB) continue;
        double a = h / s->dx[d];
        double c1 = (a - 1.0) / (a + 1.0);
        long N = s->n[d];
        long tm[3];
        for (int e = 0; e < 3; e++) tm[e] = (e == d) ? 1 : m[e];
        for (int c = BX; c <= BZ; c++) {
            if (!stag(c, d)) continue; /* tangential components only */
            for (long k = 0; k < tm[2]; k++)
                for (long j = 0; j < tm[1]; j++)
                    for (long i = 0; i < tm[0]; i++) {
                        long g[3] = {i, j, k}, in[3] = {i, j, k};
                        for (int face = 0; face < 2; face++) {
                            g[d] = face == 0 ? -1 : N;
                            in[d] = face == 0 ? 0 : N - 1;
                            long lg = lin(s, g[0], g[1], g[2]);
                            long li = lin(s, in[0], in[1], in[2]);
                            double ig_new = 0, ig_old = 0, ii_new = 0, ii_old = 0;
                            if (face == 0 && d == 0 && s->L.on) {
                                double hx = 0.5 * s->dx[0];
                                ig_new = incident_B(s, c, -hx, t_new, g[1], g[2]);
                                ig_old = incident_B(s, c, -hx, t_old, g[1], g[2]);
                                ii_new = incident_B(s, c, hx, t_new, g[1], g[2]);
                                ii_old = incident_B(s, c, hx, t_old, g[1], g[2]);
                            }
                            double sg_old = s->F[c][lg] - ig_old;
                            double si_old = old[c - BX][li] - ii_old;
                            double si_new = s->F[c][li] - ii_new;
                            s->F[c][lg] = ig_new + si_old + c1 * (si_new - sg_old);
                        }
                    }
        }
    }
    for (int c = 0; c < 3; c++) free(old[c]);
}

/* ------------------------------------------------------------------ */
/* Shape weights W_2 (Sec. II.D, Eq. (17) and the text after it)        */
/* ------------------------------------------------------------------ */

/* W_2 for the three nodes i_c-1, i_c, i_c+1 nearest to a particle at
 * distance delta = x/dx - i_c in [-1/2, 1/2) from its nearest node: the
 * integral of the hat S_2 over each cell. */
void or_weights2(double delta, double *w)
{
    w[0] = 0.5 * (0.5 - delta) * (0.5 - delta);
    w[1] = 0.75 - delta * delta;
    w[2] = 0.5 * (0.5 + delta) * (0.5 + delta);
}

/* Antiderivative of the order-4 shape S_4 of Eq. (18) (the cubic B-spline:
 * 2/3 - xi^2 + |xi|^3/2 for |xi| <= 1, (4/3)(1 - |xi|/2)^3 for 1 < |xi| <= 2),
 * P(x) = Int_{-2}^{x} S_4: piecewise quartic, 0 below -2, 1 above 2, and
 * P(x) = 1 - P(-x). */
static double prim_s4(double x)
{
    if (x <= -2.0) return 0.0;
    if (x >= 2.0) return 1.0;
    if (x > 0.0) return 1.0 - prim_s4(-x);
    if (x <= -1.0) {
        double t = 2.0 + x;
        return t * t * t * t / 24.0;
    }
    /* Int_{-2}^{-1} = 1/24, then Int_{-1}^{x} (2/3 - xi^2 - xi^3/2) */
    return 1.0 / 24.0 + (2.0 / 3.0) * (x + 1.0) - (x * x * x + 1.0) / 3.0 - (x * x * x * x - 1.0) / 8.0;
}

/* W_4 for the five nodes i_c-2 .. i_c+2 of a particle at delta = X - i_c in
 * [-1/2, 1/2): the integral of S_4(xi - delta) over each node's cell
 * [m - 1/2, m + 1/2] (Sec. II.D, the weight definition after Eq. (18)). */
void or_weights4(double delta, double *w)
{
    for (int m = -2; m <= 2; m++) w[m + 2] = prim_s4(m + 0.5 - delta) - prim_s4(m - 0.5 - delta);
}

/* the weights of the simulation's order: 3 (order 2) or 5 (order 4) values
 * for the nodes i_c - order/2 .. i_c + order/2 */
static void weights(const osim *s, double delta, double *w)
{
    if (s->order == 4) or_weights4(delta, w);
    else or_weights2(delta, w);
}

/* nearest (half-)node and weights of a coordinate X = x/dx for a component
 * that is node-centred (half = 0) or half-node-centred (half = 1) */
static long nearest(const osim *s, double X, int half, double *w)
{
    long ic;
    double delta;
    if (half) { ic = (long)floor(X); delta = X - ((double)ic + 0.5); }
    else { ic = (long)floor(X + 0.5); delta = X - (double)ic; }
    weights(s, delta, w);
    return ic;
}

/* Eq. (19): F_c(x_p) = sum_ijk W(i-ic) W(j-jc) W(k-kc) F_c(i,j,k), each
 * component with its own staggered nearest node */
static double gather1(const osim *s, int c, const double *x)
{
    const int P = s->order + 1, h = s->order / 2;
    double w[3][5];
    long ic[3];
    for (int d = 0; d < 3; d++) {
        if (d < s->dim) ic[d] = nearest(s, x[d] / s->dx[d], stag(c, d), w[d]);
        else { ic[d] = 0; for (int a = 0; a < P; a++) w[d][a] = a == h ? 1.0 : 0.0; }
    }
    double acc = 0.0;
    for (int c3 = 0; c3 < P; c3++) {
        if (2 >= s->dim && c3 != h) continue;
        for (int b = 0; b < P; b++) {
            if (1 >= s->dim && b != h) continue;
            for (int a = 0; a < P; a++)
                acc += w[0][a] * w[1][b] * w[2][c3] *
                       getF(s, c, ic[0] + a - h, ic[1] + b - h, ic[2] + c3 - h);
        }
    }
    return acc;
}

void or_gather(const osim *s, const double *x, double *eb)
{
    for (int c = 0; c < 6; c++) eb[c] = gather1(s, c, x);
}

/* ------------------------------------------------------------------ */
/* Boris pusher, Eqs. (13)-(16)                                        */
/* ------------------------------------------------------------------ */

void or_boris(double qm, double dt, const double *E, const double *B, double *u)
{
    double um[3], up[3], t[3], sv[3], ud[3];
    for (int d = 0; d < 3; d++) um[d] = u[d] + 0.5 * qm * dt * E[d];          /* Eq. (13) */
    double g = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
    for (int d = 0; d < 3; d++) t[d] = 0.5 * qm * dt * B[d] / g;
    double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    ud[0] = um[0] + (um[1] * t[2] - um[2] * t[1]);                           /* u' = u- + u- x t */
    ud[1] = um[1] + (um[2] * t[0] - um[0] * t[2]);
    ud[2] = um[2] + (um[0] * t[1] - um[1] * t[0]);
    for (int d = 0; d < 3; d++) sv[d] = 2.0 * t[d] / (1.0 + t2);
    up[0] = um[0] + (ud[1] * sv[2] - ud[2] * sv[1]);                         /* u+ = u- + u' x s */
    up[1] = um[1] + (ud[2] * sv[0] - ud[0] * sv[2]);
    up[2] = um[2] + (ud[0] * sv[1] - ud[1] * sv[0]);
    for (int d = 0; d < 3; d++) u[d] = up[d] + 0.5 * qm * dt * E[d];         /* Eq. (14) */
}

/* ------------------------------------------------------------------ */
/* Vay's pusher, the alternative Sec. II.C names for fields whose      */
/* electric and magnetic forces nearly cancel (J.-L. Vay, Phys.        */
/* Plasmas 15, 056701 (2008)): a first half kick with the full Lorentz */
/* force at the old velocity, then the second half kick solved for the */
/* new gamma in closed form, so that a particle moving at the E x B    */
/* drift velocity (E + v x B = 0) keeps its momentum exactly.          */
/* ------------------------------------------------------------------ */

void or_vay(double qm, double dt, const double *E, const double *B, double *u)
{
    const double h = 0.5 * qm * dt;
    double tau[3], up[3];
    const double g0 = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    for (int d = 0; d < 3; d++) tau[d] = h * B[d];
    /* u' = u + (q dt / m) (E + v x B / 2), v = u / gamma */
    up[0] = u[0] + 2.0 * h * E[0] + (u[1] * tau[2] - u[2] * tau[1]) / g0;
    up[1] = u[1] + 2.0 * h * E[1] + (u[2] * tau[0] - u[0] * tau[2]) / g0;
    up[2] = u[2] + 2.0 * h * E[2] + (u[0] * tau[1] - u[1] * tau[0]) / g0;
    const double tau2 = tau[0] * tau[0] + tau[1] * tau[1] + tau[2] * tau[2];
    const double ustar = up[0] * tau[0] + up[1] * tau[1] + up[2] * tau[2];
    const double sigma = 1.0 + up[0] * up[0] + up[1] * up[1] + up[2] * up[2] - tau2;
    const double g1 = sqrt(0.5 * (sigma + sqrt(sigma * sigma + 4.0 * (tau2 + ustar * ustar))));
    double t[3];
    for (int d = 0; d < 3; d++) t[d] = tau[d] / g1;
    const double sinv = 1.0 / (1.0 + t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    const double ut = up[0] * t[0] + up[1] * t[1] + up[2] * t[2];
    u[0] = sinv * (up[0] + ut * t[0] + (up[1] * t[2] - up[2] * t[1]));
    u[1] = sinv * (up[1] + ut * t[1] + (up[2] * t[0] - up[0] * t[2]));
    u[2] = sinv * (up[2] + ut * t[2] + (up[0] * t[1] - up[1] * t[0]));
}

void or_set_pusher(osim *s, int pusher) { s->pusher = pusher; }

/* shape order of gather, deposit and charge density: 2 or 4 (Sec. II.D) */
int or_set_order(osim *s, int order)
{
    if (order != 2 && order != 4) return -1;
    s->order = order;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Esirkepov charge-conserving current, Eqs. (20)-(22)                 */
/* ------------------------------------------------------------------ */

/* node-centred shapes (W_2 or W_4) of a particle at X0 and at X1 on the
 * window of order + 3 nodes that starts at node ic0 - order/2 - 1 (ic0 the
 * node nearest X0).  Returns the window base. */
static long window(const osim *s, double X0, double X1, double *S0, double *S1)
{
    const int P = s->order + 1, h = s->order / 2, Wn = P + 2;
    double w0[5], w1[5];
    long ic0 = nearest(s, X0, 0, w0);
    long ic1 = nearest(s, X1, 0, w1);
    long sh = ic1 - ic0; /* |sh| <= 1 under the Courant condition */
    for (int a = 0; a < Wn; a++) { S0[a] = 0.0; S1[a] = 0.0; }
    for (int a = 0; a < P; a++) {
        S0[a + 1] = w0[a];
        long b = a + 1 + sh;
        if (b >= 0 && b < Wn) S1[b] = w1[a];
    }
    return ic0 - h - 1;
}

/* deposit of one particle moving on a straight line from x0 to x1 with
 * velocity v (needed for the components along inactive axes), charge q and
 * weight w. Along an active axis d the paper's Eq. (20)-(22) difference
 * J_d(i+1/2) - J_d(i-1/2) = -q w (dx_d/dt) W_d(i) is summed from zero left of
 * the window; W_d is Esirkepov's decomposition (his Eq. 31) of the change of
 * the density shape. Along an inactive axis the current is q w v_d times the
 * shape product averaged along the path.  The same shape as the gather
 * (Sec. II.E after Eq. (22)): W_2 on a 5-node window, W_4 on 7 nodes. */
static void deposit(osim *s, const double *x0, const double *x1, const double *v, double qw)
{
    const int Wn = s->order + 3;
    double S0[3][7], S1[3][7], dS[3][7];
    long base[3] = {0, 0, 0};
    for (int d = 0; d < s->dim; d++) {
        base[d] = window(s, x0[d] / s->dx[d], x1[d] / s->dx[d], S0[d], S1[d]);
        for (int a = 0; a < Wn; a++) dS[d][a] = S1[d][a] - S0[d][a];
    }
    double dt = s->dt;
    if (s->dim == 1) {
        double cx = -qw * s->dx[0] / dt, acc = 0.0;
        /* the last partial sum is sum(dS) = 0 exactly: both shapes sum to one */
        for (int a = 0; a < Wn - 1; a++) {
            acc += cx * dS[0][a];
            addF(s, JX, base[0] + a, 0, 0, acc);
        }
        for (int a = 0; a < Wn; a++) {
            double f = 0.5 * (S0[0][a] + S1[0][a]);
            addF(s, JY, base[0] + a, 0, 0, qw * v[1] * f);
            addF(s, JZ, base[0] + a, 0, 0, qw * v[2] * f);
        }
        return;
    }
    if (s->dim == 2) {
        double cx = -qw * s->dx[0] / dt, cy = -qw * s->dx[1] / dt;
        for (int b = 0; b < Wn; b++) {
            double acc = 0.0;
            for (int a = 0; a < Wn - 1; a++) {
                double Wx = dS[0][a] * (S0[1][b] + 0.5 * dS[1][b]);
                acc += cx * Wx;
                addF(s, JX, base[0] + a, base[1] + b, 0, acc);
            }
        }
        for (int a = 0; a < Wn; a++) {
            double acc = 0.0;
            for (int b = 0; b < Wn - 1; b++) {
                double Wy = dS[1][b] * (S0[0][a] + 0.5 * dS[0][a]);
                acc += cy * Wy;
                addF(s, JY, base[0] + a, base[1] + b, 0, acc);
            }
        }
        for (int b = 0; b < Wn; b++)
            for (int a = 0; a < Wn; a++) {
                double Wz = S0[0][a] * S0[1][b] + 0.5 * dS[0][a] * S0[1][b] +
                            0.5 * S0[0][a] * dS[1][b] + (1.0 / 3.0) * dS[0][a] * dS[1][b];
                addF(s, JZ, base[0] + a, base[1] + b, 0, qw * v[2] * Wz);
            }
        return;
    }
    double cx = -qw * s->dx[0] / dt, cy = -qw * s->dx[1] / dt, cz = -qw * s->dx[2] / dt;
    for (int c = 0; c < Wn; c++)
        for (int b = 0; b < Wn; b++) {
            double acc = 0.0;
            for (int a = 0; a < Wn - 1; a++) {
                double Wx = dS[0][a] * (S0[1][b] * S0[2][c] + 0.5 * dS[1][b] * S0[2][c] +
                                        0.5 * S0[1][b] * dS[2][c] + (1.0 / 3.0) * dS[1][b] * dS[2][c]);
                acc += cx * Wx;
                addF(s, JX, base[0] + a, base[1] + b, base[2] + c, acc);
            }
        }
    for (int c = 0; c < Wn; c++)
        for (int a = 0; a < Wn; a++) {
            double acc = 0.0;
            for (int b = 0; b < Wn - 1; b++) {
                double Wy = dS[1][b] * (S0[0][a] * S0[2][c] + 0.5 * dS[0][a] * S0[2][c] +
                                        0.5 * S0[0][a] * dS[2][c] + (1.0 / 3.0) * dS[0][a] * dS[2][c]);
                acc += cy * Wy;
                addF(s, JY, base[0] + a, base[1] + b, base[2] + c, acc);
            }
        }
    for (int b = 0; b < Wn; b++)
        for (int a = 0; a < Wn; a++) {
            double acc = 0.0;
            for (int c = 0; c < Wn - 1; c++) {
                double Wz = dS[2][c] * (S0[0][a] * S0[1][b] + 0.5 * dS[0][a] * S0[1][b] +
                                        0.5 * S0[0][a] * dS[1][b] + (1.0 / 3.0) * dS[0][a] * dS[1][b]);
                acc += cz * Wz;
                addF(s, JZ, base[0] + a, base[1] + b, base[2] + c, acc);
            }
        }
}

/* single-particle deposit into a zeroed current, for unit tests */
void or_deposit_one(osim *s, const double *x0, const double *x1, const double *v, double qw)
{
    for (int c = JX; c <= JZ; c++) memset(s->F[c], 0, (size_t)ncells_store(s) * sizeof(double));
    deposit(s, x0, x1, v, qw);
}

/* ------------------------------------------------------------------ */
/* Particles                                                           */
/* ------------------------------------------------------------------ */

static double gamma_of(const double *u) { return sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]); }

static void half_drift(const osim *s, double *x, const double *u, double sign)
{
    double g = gamma_of(u);
    for (int d = 0; d < s->dim; d++) x[d] += sign * 0.5 * s->dt * u[d] / g;
}

/* sort key: the tile of the particle's cell, then the cell within the tile
 * (row-major, x fastest): key = tile * (cells per tile) + local cell */
static long tile_key(const osim *s, const double *x)
{
    long tile = 0, stride = 1, local = 0, lstride = 1;
    for (int d = 0; d < 3; d++) {
        long c = 0;
        if (d < s->dim) {
            c = (long)floor(x[d] / s->dx[d]);
            if (c < 0) c = 0;
            if (c > s->n[d] - 1) c = s->n[d] - 1;
        }
        long nt = (s->n[d] + s->tile[d] - 1) / s->tile[d];
        tile += (c / s->tile[d]) * stride;
        stride *= nt;
        local += (c % s->tile[d]) * lstride;
        lstride *= s->tile[d];
    }
    return tile * lstride + local;
}

static long cells_per_tile(const osim *s) { return (long)s->tile[0] * s->tile[1] * s->tile[2]; }

static long ntiles(const osim *s)
{
    long t = 1;
    for (int d = 0; d < 3; d++) t *= (s->n[d] + s->tile[d] - 1) / s->tile[d];
    return t;
}

/* stable counting sort of one species by tile key (tile, then cell within
 * the tile); dead particles get the key past the last one, sort last and are
 * dropped */
static void sort_species(osim *s, osp *p, long *perm_out)
{
    long nt = ntiles(s) * cells_per_tile(s);
    long *cnt = (long *)calloc((size_t)nt + 2, sizeof(long));
    long *key = (long *)malloc((size_t)p->n * sizeof(long) + 8);
    for (long a = 0; a < p->n; a++) {
        key[a] = p->alive[a] ? tile_key(s, &p->x[3 * a]) : nt;
        cnt[key[a] + 1]++;
    }
    for (long t = 0; t <= nt; t++) cnt[t + 1] += cnt[t]; /* exclusive starts in cnt[t] */
    long *perm = (long *)malloc((size_t)p->n * sizeof(long) + 8);
    for (long a = 0; a < p->n; a++) perm[cnt[key[a]]++] = a;
    long nalive = 0;
    for (long a = 0; a < p->n; a++) nalive += p->alive[a];
    double *x = (double *)malloc((size_t)(3 * p->n + 3) * sizeof(double));
    double *u = (double *)malloc((size_t)(3 * p->n + 3) * sizeof(double));
    uint64_t *id = (uint64_t *)malloc((size_t)p->n * sizeof(uint64_t) + 8);
    double *tau = (double *)malloc((size_t)p->n * sizeof(double) + 8);
    for (long b = 0; b < nalive; b++) {
        long a = perm[b];
        for (int d = 0; d < 3; d++) { x[3 * b + d] = p->x[3 * a + d]; u[3 * b + d] = p->u[3 * a + d]; }
        id[b] = p->id[a];
        tau[b] = p->tau[a];
        if (perm_out) perm_out[b] = a;
    }
    memcpy(p->x, x, (size_t)(3 * nalive) * sizeof(double));
    memcpy(p->u, u, (size_t)(3 * nalive) * sizeof(double));
    memcpy(p->id, id, (size_t)nalive * sizeof(uint64_t));
    memcpy(p->tau, tau, (size_t)nalive * sizeof(double));
    for (long b = 0; b < nalive; b++) p->alive[b] = 1;
    p->n = nalive;
    free(x); free(u); free(id); free(tau); free(perm); free(key); free(cnt);
}

long or_sort_species(osim *s, int isp, long *perm_out)
{
    if (isp < 0 || isp >= s->nsp) return -1;
    sort_species(s, &s->sp[isp], perm_out);
    return s->sp[isp].n;
}

/* quantum parameter chi = sqrt((g E + u x B)^2 - (u.E)^2) / E_s (Sec. IV:
 * |F_{mu nu} p^nu| over the Schwinger field in the units of Eq. (8)) */
static double chi_of(const osim *s, double g, const double *u, const double *eb)
{
    double fx = g * eb[0] + (u[1] * eb[5] - u[2] * eb[4]);
    double fy = g * eb[1] + (u[2] * eb[3] - u[0] * eb[5]);
    double fz = g * eb[2] + (u[0] * eb[4] - u[1] * eb[3]);
    double ue = u[0] * eb[0] + u[1] * eb[1] + u[2] * eb[2];
    double q = fx * fx + fy * fy + fz * fz - ue * ue;
    return q > 0.0 ? sqrt(q) / s->Es : 0.0;
}

/* chi as the Monte Carlo evaluates it, for inspection: gamma (or |k|), u (or
 * k) and the six fields E, B */
double or_chi(const osim *s, double g, const double *u, const double *eb) { return chi_of(s, g, u, eb); }

/* the prefactor alpha E_s dt / (sqrt 3 pi) of W dt (alpha = 1/137.035999084) */
static double qed_pref(const osim *s)
{
    return (1.0 / 137.035999084) * s->Es * s->dt / (sqrt(3.0) * 3.14159265358979323846);
}

static void record(osim *s, int isp, long parent, const double *k, double frac)
{
    oevent *e = &s->ev[isp][s->nev[isp]++];
    e->parent = parent;
    e->k[0] = k[0]; e->k[1] = k[1]; e->k[2] = k[2];
    e->frac = frac;
}

/* BC_SLAB: move particle a to its species' outbox (it leaves the slab) */
static void to_outbox(osp *p, long a)
{
    if (p->nout == p->outcap) {
        p->outcap = p->outcap ? 2 * p->outcap : 64;
        p->ox = (double *)realloc(p->ox, (size_t)p->outcap * 3 * sizeof(double));
        p->ou = (double *)realloc(p->ou, (size_t)p->outcap * 3 * sizeof(double));
        p->otau = (double *)realloc(p->otau, (size_t)p->outcap * sizeof(double));
        p->oid = (uint64_t *)realloc(p->oid, (size_t)p->outcap * sizeof(uint64_t));
    }
    long b = p->nout++;
    for (int d = 0; d < 3; d++) {
        p->ox[3 * b + d] = p->x[3 * a + d];
        p->ou[3 * b + d] = p->u[3 * a + d];
    }
    p->otau[b] = p->tau[a];
    p->oid[b] = p->id[a];
    p->alive[a] = 0;
}

static void push_species(osim *s, osp *p)
{
    double qm = p->q / p->m, qw = p->q * p->w;
    double dV = 1.0;
    for (int d = 0; d < s->dim; d++) dV *= s->dx[d];
    int isp = (int)(p - s->sp);
    int mc = s->qed_on && p->qed && s->photon_sp >= 0;
    for (long a = 0; a < p->n; a++) {
        if (!p->alive[a]) continue;
        double *x = &p->x[3 * a], *u = &p->u[3 * a];
        double xh[3] = {x[0], x[1], x[2]};
        half_drift(s, xh, u, 1.0);                 /* x^{n+1/2} */
        double eb[6];
        or_gather(s, xh, eb);                      /* E, B at x^{n+1/2} */
        if (s->pusher) or_vay(qm, s->dt, eb, eb + 3, u);  /* u^{n+1} */
        else or_boris(qm, s->dt, eb, eb + 3, u);
        int emitted = 0;
        double kph[3] = {0, 0, 0};
        if (mc) {
            /* optical depth form of Method I: tau -= W_rad dt; at tau <= 0
             * emit u gamma along u (u from the inverse CDF of Eq. (23)),
             * recoil to gamma (1-u), restart tau from -ln r.
             * Method II: every step u0 = r1^3 is emitted when
             * r2 < 3 r1^2 dW_rad/du(u0) dt (no optical depth) */
            double gam = gamma_of(u);
            double chi = chi_of(s, gam, u, eb);
            int event = 0;
            double frac = 0.0;
            uint32_t c[4] = {(uint32_t)p->id[a], (uint32_t)(p->id[a] >> 32), (uint32_t)s->step, 0u}, w[4];
            if (s->qed_method == 2) {
                or_philox4x32_10(c, s->key, w);
                double r1 = or_uniform24(w[0]), r2 = or_uniform24(w[1]);
                double u0 = r1 * r1 * r1;
                double pacc = 3.0 * r1 * r1 * qed_pref(s) * or_qed_Frad(u0, chi) / gam;
                if (pacc > 1.0) s->m2_over++;
                if (r2 < pacc) { event = 1; frac = u0; }
            } else {
                p->tau[a] -= qed_pref(s) * or_qed_Grad(chi) / gam;
                if (p->tau[a] <= 0.0) {
                    or_philox4x32_10(c, s->key, w);
                    frac = or_qed_sample_rad(chi, or_uniform24(w[0]));
                    p->tau[a] = -log(or_uniform24(w[1]));
                    event = 1;
                }
            }
            if (event) {
                double eg = frac * gam, um = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
                double g1 = gam * (1.0 - frac);
                if (g1 < 1.0) g1 = 1.0;
                double sc = um > 0.0 ? sqrt(g1 * g1 - 1.0) / um : 0.0;
                for (int d = 0; d < 3; d++) {
                    kph[d] = um > 0.0 ? eg * u[d] / um : 0.0;
                    u[d] *= sc;
                }
                if (eg >= s->emin) emitted = 1;
                else s->e_lost += eg * p->w * dV;
            }
        }
        double x1[3] = {xh[0], xh[1], xh[2]};
        half_drift(s, x1, u, 1.0);                 /* x^{n+1} */
        double x32[3] = {x1[0], x1[1], x1[2]};
        half_drift(s, x32, u, 1.0);                /* x^{n+3/2} */
        double g = gamma_of(u);
        double v[3] = {u[0] / g, u[1] / g, u[2] / g};
        deposit(s, xh, x32, v, qw);                /* J^{n+1} */
        int dead = 0, leaves = 0;
        for (int d = 0; d < s->dim; d++) {
            double L = (double)s->n[d] * s->dx[d];
            if (s->bc[d] == BC_PERIODIC) {
                if (x1[d] < 0.0) x1[d] += L;
                if (x1[d] >= L) x1[d] -= L;
            } else if (x1[d] < 0.0 || x1[d] >= L) {
                if (s->bc[d] == BC_SLAB) leaves = 1;
                else dead = 1;
            }
        }
        for (int d = 0; d < s->dim; d++) x[d] = x1[d];
        if (dead) {
            double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
            s->e_absorbed += p->w * p->m * (uu / (g + 1.0)) * dV;
            p->alive[a] = 0;
        } else if (leaves) {
            /* (its photon is born at x^{n+1} outside the slab: spawn sends it
             * to the outbox too) */
            if (emitted) record(s, isp, a, kph, 0.0);
            to_outbox(p, a);
        } else if (emitted) {
            record(s, isp, a, kph, 0.0);  /* an emitter absorbed in the same step leaves no photon */
        }
    }
}

/* photons move at c along k; W_pair dt of Eq. (24) at chi_gamma of the
 * fields at x^{n+1/2} drains tau; at tau <= 0 the photon converts (the
 * positron fraction v from the inverse CDF) */
static void push_photons(osim *s, osp *p)
{
    int isp = (int)(p - s->sp);
    int mc = s->qed_on && s->electron_sp >= 0 && s->positron_sp >= 0;
    for (long a = 0; a < p->n; a++) {
        if (!p->alive[a]) continue;
        double *x = &p->x[3 * a], *k = &p->u[3 * a];
        double km = sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
        double v[3] = {km > 0 ? k[0] / km : 0, km > 0 ? k[1] / km : 0, km > 0 ? k[2] / km : 0};
        double xh[3] = {x[0], x[1], x[2]};
        for (int d = 0; d < s->dim; d++) xh[d] += 0.5 * s->dt * v[d];
        int conv = 0;
        double frac = 0.0;
        if (mc && km > 0.0) {
            double eb[6];
            or_gather(s, xh, eb);
            double chi = chi_of(s, km, k, eb);
            uint32_t c[4] = {(uint32_t)p->id[a], (uint32_t)(p->id[a] >> 32), (uint32_t)s->step, 1u}, w[4];
            if (s->qed_method == 2) {
                /* Method II for pairs (the paper: "in the similar way"): the
                 * pair spectrum of Eq. (24) is bounded, so v0 = r1 is taken
                 * uniform and accepted when r2 < dW_pair/dv(v0) dt */
                or_philox4x32_10(c, s->key, w);
                double r1 = or_uniform24(w[0]), r2 = or_uniform24(w[1]);
                double pacc = qed_pref(s) * or_qed_Fpair(r1, chi) / km;
                if (pacc > 1.0) s->m2_over++;
                if (r2 < pacc) { frac = r1; conv = 1; }
            } else {
                p->tau[a] -= qed_pref(s) * or_qed_Gpair(chi) / km;
                if (p->tau[a] <= 0.0) {
                    or_philox4x32_10(c, s->key, w);
                    frac = or_qed_sample_pair(chi, or_uniform24(w[0]));
                    p->tau[a] = -log(or_uniform24(w[1]));
                    conv = 1;
                }
            }
        }
        double x1[3] = {xh[0], xh[1], xh[2]};
        for (int d = 0; d < s->dim; d++) x1[d] += 0.5 * s->dt * v[d];
        int dead = 0, leaves = 0;
        for (int d = 0; d < s->dim; d++) {
            double L = (double)s->n[d] * s->dx[d];
            if (s->bc[d] == BC_PERIODIC) {
                if (x1[d] < 0.0) x1[d] += L;
                if (x1[d] >= L) x1[d] -= L;
            } else if (x1[d] < 0.0 || x1[d] >= L) {
                if (s->bc[d] == BC_SLAB) leaves = 1;
                else dead = 1;
            }
        }
        for (int d = 0; d < s->dim; d++) x[d] = x1[d];
        if (dead) p->alive[a] = 0;
        else if (conv) record(s, isp, a, k, frac);  /* (leaving the slab or not: its pair goes where it is) */
        else if (leaves) to_outbox(p, a);
    }
}

static void append(osim *s, int isp, const double *x, const double *u, uint64_t id)
{
    osp *p = &s->sp[isp];
    if (p->n >= p->cap) return;
    long b = p->n++;
    for (int d = 0; d < 3; d++) { p->x[3 * b + d] = x[d]; p->u[3 * b + d] = u[d]; }
    p->alive[b] = 1;
    p->id[b] = id;
    p->tau[b] = initial_tau(s, id);
    /* BC_SLAB: a child born outside the slab (its parent left in the step of
     * its event) goes to the outbox with it */
    for (int d = 0; d < s->dim; d++)
        if (s->bc[d] == BC_SLAB && (x[d] < 0.0 || x[d] >= (double)s->n[d] * s->dx[d])) {
            to_outbox(p, b);
            break;
        }
}

/* children of this step's events: first the pairs of converted photons
 * (electron, then positron, in photon order), then the photons of each
 * emitting species in species and parent order */
static void spawn(osim *s)
{
    int ph = s->photon_sp;
    if (ph >= 0 && s->electron_sp >= 0 && s->positron_sp >= 0) {
        osp *P = &s->sp[ph];
        for (long e = 0; e < s->nev[ph]; e++) {
            oevent *ev = &s->ev[ph][e];
            long a = ev->parent;
            uint32_t c[4] = {(uint32_t)P->id[a], (uint32_t)(P->id[a] >> 32), (uint32_t)s->step, 1u}, w[4];
            or_philox4x32_10(c, s->key, w);
            uint64_t eid = ((uint64_t)w[3] << 32) | w[2];
            double km = sqrt(ev->k[0] * ev->k[0] + ev->k[1] * ev->k[1] + ev->k[2] * ev->k[2]);
            double ep = ev->frac * km, em = (1.0 - ev->frac) * km;
            double pm = em > 1.0 ? sqrt(em * em - 1.0) : 0.0, pp = ep > 1.0 ? sqrt(ep * ep - 1.0) : 0.0;
            double ue[3], uq[3];
            for (int d = 0; d < 3; d++) {
                ue[d] = km > 0 ? pm * ev->k[d] / km : 0.0;
                uq[d] = km > 0 ? pp * ev->k[d] / km : 0.0;
            }
            append(s, s->electron_sp, &P->x[3 * a], ue, eid);
            append(s, s->positron_sp, &P->x[3 * a], uq, eid + 1);
            P->alive[a] = 0;
        }
    }
    if (ph >= 0)
        for (int i = 0; i < s->nsp; i++) {
            osp *p = &s->sp[i];
            if (p->kind != 0 || !p->qed) continue;
            for (long e = 0; e < s->nev[i]; e++) {
                oevent *ev = &s->ev[i][e];
                long a = ev->parent;
                uint32_t c[4] = {(uint32_t)p->id[a], (uint32_t)(p->id[a] >> 32), (uint32_t)s->step, 0u}, w[4];
                or_philox4x32_10(c, s->key, w);
                append(s, ph, &p->x[3 * a], ev->k, ((uint64_t)w[3] << 32) | w[2]);
            }
        }
    for (int i = 0; i < s->nsp; i++) s->nev[i] = 0;
}

/* The split step of Sec. II.F in five phases (a slab's caller exchanges
 * ghost layers, currents and particles between them):
 *   0: (sort) E^{n+1/2} with J^n;   1: B^{n+1/2};
 *   2: push every species (J^{n+1}), QED spawn;
 *   3: B^{n+1};                     4: E^{n+1} with J^{n+1}, n -> n+1. */
int or_step_phase(osim *s, int phase)
{
    double h = 0.5 * s->dt;
    double t0 = (double)s->step * s->dt;
    switch (phase) {
    case 0:
        if (s->sort_interval > 0 && s->step % s->sort_interval == 0)
            for (int i = 0; i < s->nsp; i++) sort_species(s, &s->sp[i], NULL);
        update_E(s, h);                       /* E^{n+1/2} with J^n */
        return 0;
    case 1:
        update_B(s, h, t0 + h);               /* B^{n+1/2} */
        return 0;
    case 2:
        for (int c = JX; c <= JZ; c++) memset(s->F[c], 0, (size_t)ncells_store(s) * sizeof(double));
        for (int i = 0; i < s->nsp; i++) {
            if (s->sp[i].kind == 1) push_photons(s, &s->sp[i]);
            else push_species(s, &s->sp[i]);
        }
        if (s->qed_on) spawn(s);
        return 0;
    case 3:
        update_B(s, h, t0 + s->dt);           /* B^{n+1} */
        return 0;
    case 4:
        update_E(s, h);                       /* E^{n+1} with J^{n+1} */
        s->step++;
        return 0;
    }
    return -1;
}

int or_step(osim *s, long nsteps)
{
    for (long it = 0; it < nsteps; it++)
        for (int ph = 0; ph < 5; ph++) or_step_phase(s, ph);
    return 0;
}

/* BC_SLAB: the whole stored array of component c (ghost layers included),
 * x fastest, len[0] x len[1] x len[2] */
long or_field_raw_size(const osim *s, long *len)
{
    for (int d = 0; d < 3; d++) len[d] = s->len[d];
    return ncells_store(s);
}

int or_get_field_raw(const osim *s, int c, double *out)
{
    if (c < 0 || c >= NF) return -1;
    memcpy(out, s->F[c], (size_t)ncells_store(s) * sizeof(double));
    return 0;
}

int or_set_field_raw(osim *s, int c, const double *in)
{
    if (c < 0 || c >= NF) return -1;
    memcpy(s->F[c], in, (size_t)ncells_store(s) * sizeof(double));
    return 0;
}

/* BC_SLAB: the particles of species isp that left the slab since the last
 * call (positions as computed, momenta, identities, optical depths); with
 * x == NULL only the count; a call with arrays empties the outbox */
long or_take_outbox(osim *s, int isp, double *x, double *u, uint64_t *id, double *tau)
{
    if (isp < 0 || isp >= s->nsp) return -1;
    osp *p = &s->sp[isp];
    long n = p->nout;
    if (!x) return n;
    memcpy(x, p->ox, (size_t)n * 3 * sizeof(double));
    memcpy(u, p->ou, (size_t)n * 3 * sizeof(double));
    memcpy(id, p->oid, (size_t)n * sizeof(uint64_t));
    memcpy(tau, p->otau, (size_t)n * sizeof(double));
    p->nout = 0;
    return n;
}

/* append particles with their identities and optical depths (migration) */
int or_load_state(osim *s, int isp, long n, const double *x, const double *u, const uint64_t *id,
                  const double *tau)
{
    if (isp < 0 || isp >= s->nsp) return -1;
    osp *p = &s->sp[isp];
    if (p->n + n > p->cap) return -2;
    for (long a = 0; a < n; a++) {
        long b = p->n + a;
        for (int d = 0; d < 3; d++) {
            p->x[3 * b + d] = d < s->dim ? x[3 * a + d] : 0.0;
            p->u[3 * b + d] = u[3 * a + d];
        }
        p->alive[b] = 1;
        p->id[b] = id[a];
        p->tau[b] = tau[a];
    }
    p->n += n;
    return 0;
}

long or_get_particles(const osim *s, int isp, double *x, double *y, double *z, double *ux,
                      double *uy, double *uz, unsigned char *alive)
{
    if (isp < 0 || isp >= s->nsp) return -1;
    const osp *p = &s->sp[isp];
    for (long a = 0; a < p->n; a++) {
        if (x) x[a] = p->x[3 * a + 0];
        if (y) y[a] = p->x[3 * a + 1];
        if (z) z[a] = p->x[3 * a + 2];
        if (ux) ux[a] = p->u[3 * a + 0];
        if (uy) uy[a] = p->u[3 * a + 1];
        if (uz) uz[a] = p->u[3 * a + 2];
        if (alive) alive[a] = p->alive[a];
    }
    return p->n;
}

/* ------------------------------------------------------------------ */
/* Diagnostics                                                         */
/* ------------------------------------------------------------------ */

/* charge density on nodes: rho = sum_p q w W(node - x_p), averaged over the
 * two half-step positions x -/+ (dt/2) v that bracket the integer step;
 * Gauss's law holds to round-off for this average under the split step. */
static void deposit_rho(const osim *s, double *rho)
{
    long m[3];
    out_box(s, m);
    long nb = m[0] * m[1] * m[2];
    memset(rho, 0, (size_t)nb * sizeof(double));
    for (int isp = 0; isp < s->nsp; isp++) {
        const osp *p = &s->sp[isp];
        for (long a = 0; a < p->n; a++) {
            if (!p->alive[a]) continue;
            for (int side = 0; side < 2; side++) {
                double xs[3] = {p->x[3 * a], p->x[3 * a + 1], p->x[3 * a + 2]};
                half_drift(s, xs, &p->u[3 * a], side == 0 ? -1.0 : 1.0);
                const int P = s->order + 1, h = s->order / 2;
                double w[3][5];
                long ic[3];
                for (int d = 0; d < 3; d++) {
                    if (d < s->dim) ic[d] = nearest(s, xs[d] / s->dx[d], 0, w[d]);
                    else { ic[d] = 0; for (int a = 0; a < P; a++) w[d][a] = a == h ? 1.0 : 0.0; }
                }
                for (int c = 0; c < P; c++)
                    for (int b = 0; b < P; b++)
                        for (int aa = 0; aa < P; aa++) {
                            double wt = w[0][aa] * w[1][b] * w[2][c];
                            if (wt == 0.0) continue;
                            long idx[3] = {ic[0] + aa - h, ic[1] + b - h, ic[2] + c - h};
                            int ok = 1;
                            for (int d = 0; d < 3; d++) {
                                if (d >= s->dim) { idx[d] = 0; continue; }
                                if (s->bc[d] == BC_PERIODIC) idx[d] = imod(idx[d], s->n[d]);
                                else if (idx[d] < 0 || idx[d] >= m[d]) ok = 0;
                            }
                            if (!ok) continue;
                            rho[(idx[2] * m[1] + idx[1]) * m[0] + idx[0]] += 0.5 * p->q * p->w * wt;
                        }
            }
        }
    }
}

int or_get_rho(const osim *s, double *rho)
{
    deposit_rho(s, rho);
    return 0;
}

/* out: [0] step, [1] t, [2] U_E, [3] U_B, [4] charge, [5] max |div E - rho - rho_bg|,
 *      [6] absorbed kinetic energy, [7 .. 7+nsp) U_kin per species */
int or_diagnostics(const osim *s, double *out)
{
    double dV = 1.0;
    for (int d = 0; d < s->dim; d++) dV *= s->dx[d];
    long m[3];
    out_box(s, m);
    double ue = 0.0, ub = 0.0;
    for (long k = 0; k < (s->dim > 2 ? s->n[2] : 1); k++)
        for (long j = 0; j < (s->dim > 1 ? s->n[1] : 1); j++)
            for (long i = 0; i < s->n[0]; i++) {
                long l = lin(s, i, j, k);
                for (int c = 0; c < 3; c++) {
                    ue += 0.5 * s->F[EX + c][l] * s->F[EX + c][l];
                    ub += 0.5 * s->F[BX + c][l] * s->F[BX + c][l];
                }
            }
    out[0] = (double)s->step;
    out[1] = (double)s->step * s->dt;
    out[2] = ue * dV;
    out[3] = ub * dV;
    double charge = 0.0;
    for (int isp = 0; isp < s->nsp; isp++) {
        const osp *p = &s->sp[isp];
        double uk = 0.0;
        long na = 0;
        for (long a = 0; a < p->n; a++) {
            if (!p->alive[a]) continue;
            const double *u = &p->u[3 * a];
            double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
            if (p->kind == 1) uk += p->w * sqrt(uu); /* photon energy |k| */
            else uk += p->w * p->m * uu / (gamma_of(u) + 1.0);
            na++;
        }
        out[7 + isp] = uk * dV;
        charge += p->q * p->w * (double)na * dV;
    }
    double vol = dV;
    for (int d = 0; d < s->dim; d++) vol *= (double)s->n[d];
    out[4] = charge + s->rho_bg * vol;
    long nb = m[0] * m[1] * m[2];
    double *rho = (double *)malloc((size_t)nb * sizeof(double));
    deposit_rho(s, rho);
    double gmax = 0.0;
    for (long k = 0; k < (s->dim > 2 ? s->n[2] : 1); k++)
        for (long j = 0; j < (s->dim > 1 ? s->n[1] : 1); j++)
            for (long i = 0; i < s->n[0]; i++) {
                double div = dback(s, EX, 0, i, j, k) + dback(s, EY, 1, i, j, k) +
                             dback(s, EZ, 2, i, j, k);
                double r = div - rho[(k * m[1] + j) * m[0] + i] - s->rho_bg;
                if (fabs(r) > gmax) gmax = fabs(r);
            }
    free(rho);
    out[5] = gmax;
    out[6] = s->e_absorbed;
    return 7 + s->nsp;
}

long or_step_count(const osim *s) { return s->step; }

double or_photon_lost(const osim *s) { return s->e_lost; }

long or_get_qed_state(const osim *s, int isp, uint64_t *id, double *tau)
{
    if (isp < 0 || isp >= s->nsp) return -1;
    const osp *p = &s->sp[isp];
    for (long a = 0; a < p->n; a++) {
        if (id) id[a] = p->id[a];
        if (tau) tau[a] = p->tau[a];
    }
    return p->n;
}
