// vjp_f32.cu -- float instantiations of the adjoint kernel.
#include "rnea_vjp_launch.cuh"

int rd_vjp_dispatch_f32(const rd_model *m, int B, const void *q, const void *qd,
                         const void *qdd, const void *w, void *gq, void *gqd, void *gqdd,
                         const double *base18, int mode, void *ws, size_t ws_bytes,
                         cudaStream_t s)
{
    return rdyn::vjp_dispatch<float>(m, B, q, qd, qdd, w, gq, gqd, gqdd, base18, mode, ws,
                                   ws_bytes, s);
}
