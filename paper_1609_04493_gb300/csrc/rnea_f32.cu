// rnea_f32.cu -- float instantiations of the inverse-dynamics kernels.
#include "rnea_launch.cuh"

int rd_rnea_dispatch_f32(const rd_model *m, int B, const void *q, const void *qd,
                          const void *qdd, void *tau, const double *base18, int variant,
                          cudaStream_t s)
{
    return rdyn::dispatch<float>(m, B, q, qd, qdd, tau, base18, variant, s);
}
