// aba_warp_f64.cu -- double instantiation of the warp-per-instance
// forward-dynamics kernel (aba_warp.cuh).
#include "aba_warp.cuh"

int rd_aba_warp_f64(const rd_model *m, int B, const void *q, const void *qd, const void *tau,
                    void *qdd, int *status, const double *base18, cudaStream_t s)
{
    return rdyn::launch_aba_warp<double, double, double>(m, B, q, qd, tau, qdd, status, base18, s);
}
