// diag.cuh -- FP64 diagnostics (diag.cu).
#pragma once
#include "pic_internal.cuh"
#include "push.cuh"

namespace pic {

size_t diag_scratch_doubles();
template <typename R>
void diag_field_energy(const R *F, const Grid &g, double *scratch, double *out2, cudaStream_t st);
void diag_kinetic_f32(const PartF32 &P, bool photon, double *scratch, double *out2, cudaStream_t st);
void diag_kinetic_f64(const PartF64 &P, bool photon, double *scratch, double *out2, cudaStream_t st);
void diag_rho_f32(const PartF32 &P, const Grid &g, double qw, double *rho, cudaStream_t st);
void diag_rho_f64(const PartF64 &P, const Grid &g, double qw, double *rho, cudaStream_t st);
template <typename R>
void diag_gauss(const R *F, const double *rho, const Grid &g, double rho_bg, double *scratch, double *out1,
                cudaStream_t st);

}  // namespace pic
