// rdyn_vjp.cu -- rnea_vjp and its workspace query: argument checks and
// dispatch of the adjoint kernels.
#include <cuda_runtime.h>

#include "rdyn_internal.h"

extern "C" int rnea_vjp_workspace_size(const rd_model *m, int B, int dtype, size_t *bytes)
{
    g_rd_error.clear();
    if (!m || !bytes) return rd_fail(RD_ERR_ARG, "rnea_vjp_workspace_size: null argument");
    if (B < 0) return rd_fail(RD_ERR_RANGE, "rnea_vjp_workspace_size: B = %d < 0", B);
    if (dtype != RD_F32 && dtype != RD_F64)
        return rd_fail(RD_ERR_DTYPE, "rnea_vjp_workspace_size: dtype %d", dtype);
    *bytes = (size_t)m->n * 20 * (size_t)B * (dtype == RD_F32 ? 4 : 8);
    return RD_OK;
}

extern "C" int rnea_vjp(const rd_model *m, int B, int dtype, const void *q, const void *qd,
                        const void *qdd, const void *w, void *gq, void *gqd, void *gqdd,
                        const double *base, int mode, void *workspace, size_t workspace_bytes,
                        void *stream)
{
    g_rd_error.clear();
    if (!m) return rd_fail(RD_ERR_ARG, "rnea_vjp: null model");
    if (B < 0) return rd_fail(RD_ERR_RANGE, "rnea_vjp: B = %d < 0", B);
    if (dtype != RD_F32 && dtype != RD_F64)
        return rd_fail(RD_ERR_DTYPE, "rnea_vjp: dtype %d is not RD_F32 or RD_F64", dtype);
    if (B == 0) return RD_OK;
    if (!q || !qd || !qdd || !w || !gq || !gqd || !gqdd)
        return rd_fail(RD_ERR_ARG, "rnea_vjp: null batch pointer");
    const void *outs[3] = {gq, gqd, gqdd};
    const void *ins[4] = {q, qd, qdd, w};
    for (const void *o : outs)
        for (const void *in : ins)
            if (o == in) return rd_fail(RD_ERR_ARG, "rnea_vjp: a gradient aliases an input");
    if (gq == gqd || gq == gqdd || gqd == gqdd)
        return rd_fail(RD_ERR_ARG, "rnea_vjp: gradient outputs alias each other");
    double b18[18];
    rd_convert_base(m, base, b18);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (dtype == RD_F32)
        return rd_vjp_dispatch_f32(m, B, q, qd, qdd, w, gq, gqd, gqdd, b18, mode, workspace,
                                   workspace_bytes, s);
    return rd_vjp_dispatch_f64(m, B, q, qd, qdd, w, gq, gqd, gqdd, b18, mode, workspace,
                               workspace_bytes, s);
}
