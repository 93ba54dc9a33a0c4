// push.cuh -- particle arrays and launchers of the particle kernels (push.cu).
#pragma once
#include "pic_internal.cuh"

namespace pic {

// FP32 cell+offset species view (one buffer of the double-buffered pair)
struct PartF32 {
    uint32_t *cell;
    float *off[3];
    float *u[3];
    long long n;           // host-side upper bound of the count (grid sizing)
    const long long *dn;   // live count on the device (updated by sorts)
    double *tau;           // QED optical depth (NULL when the species has none)
    uint64_t *id;          // QED identity (NULL when the species has none)
};

// FP64 plain species view
struct PartF64 {
    uint32_t *cell;  // packed floor(x/dx), the sort key source; kDead when absorbed
    double *x[3];
    double *u[3];
    long long n;           // host-side upper bound of the count (grid sizing)
    const long long *dn;   // live count on the device (updated by sorts)
    double *tau;           // QED optical depth (NULL when the species has none)
    uint64_t *id;          // QED identity (NULL when the species has none)
};

struct PushConst {
    double qmdt2;  // q/m * dt/2
    double qw;     // q * w
    double hdx[3]; // dt / (2 dx_d)  (FP32 offset drift)
    double hdt;    // dt / 2         (FP64 absolute drift)
    double cJ[3];  // -q w dx_d / dt (Esirkepov prefix coefficient)
    double wmdV;   // w * m * dV     (absorbed kinetic energy)
    // FP32 copies for the FP32 form (converted once on the host)
    float qmdt2_f, qw_f, hdx_f[3], cJ_f[3];
    int pusher;    // 0: Boris, 1: Vay
};

void launch_push_f32(const PartF32 &P, float *F, const Grid &g, const PushConst &pc, int *err, double *e_abs,
                     cudaStream_t st);
// the particles listed in list[0 .. *count) (count on the device, at most max_n)
void launch_push_list_f32(const PartF32 &P, const uint32_t *list, const uint32_t *count, long long max_n, float *F,
                          const Grid &g, const PushConst &pc, int *err, double *e_abs, cudaStream_t st);
void launch_push_f64(const PartF64 &P, double *F, const Grid &g, const PushConst &pc, int *err, double *e_abs,
                     cudaStream_t st);
void launch_gather_f32(const PartF32 &P, const float *F, const Grid &g, double *out, cudaStream_t st);
void launch_gather_f64(const PartF64 &P, const double *F, const Grid &g, double *out, cudaStream_t st);
// (bad: the lowest index of a particle outside the domain or with a
// non-finite momentum; such particles are not stored; preset to all ones)
void launch_load_f32(const PartF32 &P, long long first, long long n, const double *const *xs,
                     const double *const *us, const Grid &g, unsigned long long *bad, cudaStream_t st);
void launch_load_f64(const PartF64 &P, long long first, long long n, const double *const *xs,
                     const double *const *us, const Grid &g, unsigned long long *bad, cudaStream_t st);
void launch_unload_f32(const PartF32 &P, const Grid &g, double *const *xs, double *const *us, uint8_t *alive,
                       cudaStream_t st);
void launch_unload_f64(const PartF64 &P, const Grid &g, double *const *xs, double *const *us, uint8_t *alive,
                       cudaStream_t st);

}  // namespace pic
