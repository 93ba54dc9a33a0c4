// fdtd.cuh -- launchers of the field kernels (fdtd.cu).
#pragma once
#include "pic_internal.cuh"

namespace pic {

template <typename R>
void launch_update_E(R *F, const Grid &g, double h, bool twice, bool zeroJ, cudaStream_t st);
template <typename R>
void launch_update_B(R *F, const Grid &g, double h, double t_new, const Laser &L, cudaStream_t st);
template <typename R>
void launch_fold(R *F, const Grid &g, cudaStream_t st);
void launch_fold_rho(double *rho, const Grid &g, cudaStream_t st);

}  // namespace pic
