// rdyn_aba.cu -- aba_batch and its workspace query.
#include <cuda_runtime.h>

#include "rdyn_internal.h"

extern "C" int aba_workspace_size(const rd_model *m, int B, int dtype, int flags, size_t *bytes)
{
    g_rd_error.clear();
    if (!m || !bytes) return rd_fail(RD_ERR_ARG, "aba_workspace_size: null argument");
    if (B < 0) return rd_fail(RD_ERR_RANGE, "aba_workspace_size: B = %d < 0", B);
    if (dtype != RD_F32 && dtype != RD_F64)
        return rd_fail(RD_ERR_DTYPE, "aba_workspace_size: dtype %d", dtype);
    *bytes = dtype == RD_F32 ? rd_aba_ws_bytes_f32(m->n, B, flags) : rd_aba_ws_bytes_f64(m->n, B, flags);
    return RD_OK;
}

extern "C" int aba_batch(const rd_model *m, int B, int dtype, const void *q, const void *qd,
                         const void *tau, void *qdd, const double *base, int *status, int flags,
                         void *workspace, size_t workspace_bytes, void *stream)
{
    g_rd_error.clear();
    if (!m) return rd_fail(RD_ERR_ARG, "aba_batch: null model");
    if (B < 0) return rd_fail(RD_ERR_RANGE, "aba_batch: B = %d < 0", B);
    if (dtype != RD_F32 && dtype != RD_F64)
        return rd_fail(RD_ERR_DTYPE, "aba_batch: dtype %d is not RD_F32 or RD_F64", dtype);
    if (B == 0) return RD_OK;
    if (!q || !qd || !tau || !qdd) return rd_fail(RD_ERR_ARG, "aba_batch: null batch pointer");
    if (qdd == q || qdd == qd || qdd == tau)
        return rd_fail(RD_ERR_ARG, "aba_batch: qdd aliases an input");
    double b18[18];
    rd_convert_base(m, base, b18);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (dtype == RD_F32)
        return rd_aba_dispatch_f32(m, B, q, qd, tau, qdd, status, workspace, workspace_bytes, b18,
                                   flags, s);
    return rd_aba_dispatch_f64(m, B, q, qd, tau, qdd, status, workspace, workspace_bytes, b18,
                               flags, s);
}
