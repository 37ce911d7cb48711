// aba_warp_f32x.cu -- float instantiations of the warp-per-instance
// forward-dynamics kernel (aba_warp.cuh) with the bias sweeps in double-float.
#include "aba_warp.cuh"

int rd_aba_warp_f32x(const rd_model *m, int B, const void *q, const void *qd, const void *tau,
                     void *qdd, int *status, const double *base18, bool fp64_update,
                     cudaStream_t s)
{
    using rdyn::DF;
    return fp64_update
               ? rdyn::launch_aba_warp<float, double, DF>(m, B, q, qd, tau, qdd, status, base18, s)
               : rdyn::launch_aba_warp<float, DF, DF>(m, B, q, qd, tau, qdd, status, base18, s);
}
