// aba_warp_f32.cu -- float instantiations of the warp-per-instance
// forward-dynamics kernel (aba_warp.cuh), bias sweeps in FP32; the
// double-float ones are in aba_warp_f32x.cu (two units build in parallel).
#include "aba_warp.cuh"

int rd_aba_warp_f32x(const rd_model *m, int B, const void *q, const void *qd, const void *tau,
                     void *qdd, int *status, const double *base18, bool fp64_update,
                     cudaStream_t s);

int rd_aba_warp_f32(const rd_model *m, int B, const void *q, const void *qd, const void *tau,
                    void *qdd, int *status, const double *base18, bool fp64_update,
                    bool extended_bias, cudaStream_t s)
{
    using rdyn::DF;
    if (extended_bias)
        return rd_aba_warp_f32x(m, B, q, qd, tau, qdd, status, base18, fp64_update, s);
    return fp64_update
               ? rdyn::launch_aba_warp<float, double, float>(m, B, q, qd, tau, qdd, status, base18, s)
               : rdyn::launch_aba_warp<float, DF, float>(m, B, q, qd, tau, qdd, status, base18, s);
}
