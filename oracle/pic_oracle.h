/*
 * pic_oracle.h -- API of the FP64 CPU oracle (test infrastructure only).
 * Private to oracle/: the CUDA path neither includes nor links it.
 */
#ifndef PIC_ORACLE_H
#define PIC_ORACLE_H

#include <stdint.h>

#define OR_MAX_SPECIES 8

typedef struct osim osim;

osim *or_create(int dim, const long *n, const double *dx, const int *bc, double dt,
                double rho_bg, int sort_interval, const int *tile);
void or_destroy(osim *s);
int or_add_species(osim *s, double q, double m, double w, long cap);
int or_add_species2(osim *s, double q, double m, double w, long cap, int kind, int qed);
void or_set_qed(osim *s, int photon_sp, int electron_sp, int positron_sp, double lambda_r_m, double emin,
                uint64_t seed);
double or_Es(const osim *s);
int or_set_qed_method(osim *s, int method);
long or_method2_over(const osim *s);
double or_chi(const osim *s, double g, const double *u, const double *eb);
double or_photon_lost(const osim *s);
long or_get_qed_state(const osim *s, int isp, uint64_t *id, double *tau);
int or_load(osim *s, int isp, long n, const double *x, const double *y, const double *z,
            const double *ux, const double *uy, const double *uz);
/* caller-given identities (and their initial optical depths) for particles [first, first + n) */
int or_set_ids(osim *s, int isp, long first, long n, const uint64_t *id);
int or_get_field(const osim *s, int c, double *out);
int or_set_field(osim *s, int c, const double *in);
int or_get_ghost(const osim *s, int c, long i, long j, long k, double *v);
void or_set_laser(osim *s, int pol, double a0, double waist, double fwhm, double t_peak,
                  double x_focus, double yc, double zc);
void or_weights2(double delta, double *w);
void or_gather(const osim *s, const double *x, double *eb);
void or_boris(double qm, double dt, const double *E, const double *B, double *u);
/* Vay's pusher (Sec. II.C's alternative to Boris), same arguments */
void or_vay(double qm, double dt, const double *E, const double *B, double *u);
/* 0: Boris (default), 1: Vay, for every massive species of the step */
void or_set_pusher(osim *s, int pusher);
/* shape order 2 (default) or 4; returns -1 for others */
int or_set_order(osim *s, int order);
void or_weights4(double delta, double *w);
void or_deposit_one(osim *s, const double *x0, const double *x1, const double *v, double qw);
long or_sort_species(osim *s, int isp, long *perm_out);
int or_step(osim *s, long nsteps);
/* the split step in its five phases (BC_SLAB callers exchange between them) */
int or_step_phase(osim *s, int phase);
/* BC_SLAB = 2: a slab of a larger periodic grid (ghost layers set by the caller) */
long or_field_raw_size(const osim *s, long *len);
int or_get_field_raw(const osim *s, int c, double *out);
int or_set_field_raw(osim *s, int c, const double *in);
long or_take_outbox(osim *s, int isp, double *x, double *u, uint64_t *id, double *tau);
int or_load_state(osim *s, int isp, long n, const double *x, const double *u, const uint64_t *id,
                  const double *tau);
long or_get_particles(const osim *s, int isp, double *x, double *y, double *z, double *ux,
                      double *uy, double *uz, unsigned char *alive);
int or_get_rho(const osim *s, double *rho);
int or_diagnostics(const osim *s, double *out);
long or_step_count(const osim *s);

void or_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out);
double or_uniform24(uint32_t x);

double or_bessel_k(double nu, double x);
double or_int_k13(double y);
double or_qed_Frad(double u, double chi);
double or_qed_Fpair(double v, double chi);
double or_qed_Grad(double chi);
double or_qed_Gpair(double chi);
double or_qed_Prad(double chi);
double or_qed_cdf_rad(double u, double chi);
double or_qed_cdf_pair(double v, double chi);
double or_qed_sample_rad(double chi, double r);
double or_qed_sample_pair(double chi, double r);
double or_qed_method2_rad(double chi, double dwdt, double r1, double r2);

long or_mlp_nparams(void);
void or_mlp_forward(const double *P, long n, const double *in, double *out);
double or_mlp_loss_grad(const double *P, long n, const double *in, const double *tgt, double *G);

#endif
