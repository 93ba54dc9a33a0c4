// qed_host.cuh -- host entry points of the QED module (qed.cu).
#pragma once
#include "push.cuh"
#include "qed.cuh"

namespace pic {

size_t qed_table_bytes();
int qed_upload_tables(void *dev, QedTables *T, cudaStream_t st);
void qed_spectra(int p, double frac, double chi, double *F);
void launch_qed_eval(const QedTables &T, bool f64, int p, long long n, const double *chi, const double *r,
                     double *out, cudaStream_t st);
void launch_init_qed(long long first, long long n, uint64_t id0, uint64_t *id, double *tau, const uint32_t *key,
                     cudaStream_t st);
void launch_spawn_photons(const PartF32 &parent, const uint32_t *bsum, const uint32_t *total, long long m,
                          const QedParams &q,
                          const PartF32 &ph, double *ph_tau, uint64_t *ph_id, uint32_t *ph_ev, long long *ph_count,
                          long long ph_cap, int dim, int *err, cudaStream_t st);
void launch_spawn_pairs(const PartF32 &phot, const uint32_t *bsum, const uint32_t *total, long long m,
                        const QedParams &q,
                        const PartF32 &el, double *el_tau, uint64_t *el_id, uint32_t *el_ev, long long *el_count,
                        long long el_cap, const PartF32 &po, double *po_tau, uint64_t *po_id, uint32_t *po_ev,
                        long long *po_count, long long po_cap, int dim, int *err, cudaStream_t st);
void launch_spawn_photons(const PartF64 &parent, const uint32_t *bsum, const uint32_t *total, long long m,
                          const QedParams &q,
                          const PartF64 &ph, double *ph_tau, uint64_t *ph_id, uint32_t *ph_ev, long long *ph_count,
                          long long ph_cap, int dim, int *err, cudaStream_t st);
void launch_spawn_pairs(const PartF64 &phot, const uint32_t *bsum, const uint32_t *total, long long m,
                        const QedParams &q,
                        const PartF64 &el, double *el_tau, uint64_t *el_id, uint32_t *el_ev, long long *el_count,
                        long long el_cap, const PartF64 &po, double *po_tau, uint64_t *po_id, uint32_t *po_ev,
                        long long *po_count, long long po_cap, int dim, int *err, cudaStream_t st);
void launch_push_qed_f64(const PartF64 &P, double *F, const Grid &g, const PushConst &pc, const QedParams &q,
                         int *err, double *e_abs, cudaStream_t st);
void launch_push_photon_f64(const PartF64 &P, const double *F, const Grid &g, const PushConst &pc,
                            const QedParams &q, int *err, cudaStream_t st);
// (first: see k_push_qed_f32 -- nullptr pushes every particle)
void launch_push_qed_f32(const PartF32 &P, float *F, const Grid &g, const PushConst &pc, const QedParams &q,
                         int *err, double *e_abs, cudaStream_t st, const uint32_t *first = nullptr);
// (tc: with the surrogate, evaluate the pair network per CTA on the tcgen05
// tensor cores instead of per warp with mma.sync)
// (first: see k_push_photon_f32 -- nullptr pushes every photon; tc is not
// taken with first)
void launch_push_photon_f32(const PartF32 &P, const float *F, const Grid &g, const PushConst &pc,
                            const QedParams &q, int *err, cudaStream_t st, bool tc, const uint32_t *first = nullptr);

}  // namespace pic
