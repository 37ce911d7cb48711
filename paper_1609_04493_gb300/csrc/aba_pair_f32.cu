// aba_pair_f32.cu -- instantiations of the two-warp forward-dynamics kernel
// (aba_pair.cuh).
#include "aba_pair_launch.cuh"

int rd_aba_pair_f32(const rd_model *m, int B, const void *q, const void *qd, const void *tau,
                    void *qdd, int *status, void *ws, const double *base18, bool fp64_update,
                    bool extended_bias, bool withhold, cudaStream_t s)
{
    using rdyn::DF;
    using rdyn::launch_aba_multi;
    if (extended_bias)
        return fp64_update
                   ? launch_aba_multi<float, double, DF, 2>(m, B, q, qd, tau, qdd, status, ws, base18, s, withhold)
                   : launch_aba_multi<float, DF, DF, 2>(m, B, q, qd, tau, qdd, status, ws, base18, s, withhold);
    return fp64_update
               ? launch_aba_multi<float, double, float, 2>(m, B, q, qd, tau, qdd, status, ws, base18, s, withhold)
               : launch_aba_multi<float, DF, float, 2>(m, B, q, qd, tau, qdd, status, ws, base18, s, withhold);
}

int rd_aba_pair_f64(const rd_model *m, int B, const void *q, const void *qd, const void *tau,
                    void *qdd, int *status, void *ws, const double *base18, bool withhold,
                    cudaStream_t s)
{
    return rdyn::launch_aba_multi<double, double, double, 2>(m, B, q, qd, tau, qdd, status, ws,
                                                             base18, s, withhold);
}
