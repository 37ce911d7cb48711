// aba_f32.cu -- float instantiations of the forward-dynamics kernel.
#include "aba_launch.cuh"

int rd_aba_dispatch_f32(const rd_model *m, int B, const void *q, const void *qd,
                         const void *tau, void *qdd, int *status, void *ws, size_t ws_bytes,
                         const double *base18, int flags, cudaStream_t s)
{
    return rdyn::aba_dispatch<float>(m, B, q, qd, tau, qdd, status, ws, ws_bytes, base18, flags, s);
}

size_t rd_aba_ws_bytes_f32(int n, int B, int flags)
{
    return rdyn::aba_ws_bytes<float>(n, B, flags);
}
