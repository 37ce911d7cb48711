// rdyn_trig.cu -- the joint sine/cosine of the FP32 inverse-dynamics kernels,
// exposed on its own so its accuracy can be checked (diagnostic, not on the
// dynamics path).
#include <cuda_runtime.h>

#include "rdyn_internal.h"
#include "rnea_serial.cuh"
#include "trig_poly.cuh"

namespace {

template <bool FAST>
__global__ void __launch_bounds__(256) trig_kernel(const float *x, float *s, float *c, int count)
{
    const int i = blockIdx.x * 256 + threadIdx.x;
    if (i >= count) return;
    float sv, cv;
    if constexpr (FAST) rdyn::sincos_fast(x[i], &sv, &cv);
    else rdyn::sincos_poly(x[i], &sv, &cv);
    s[i] = sv;
    c[i] = cv;
}

}  // namespace

extern "C" int rd_joint_trig(int flags, const float *x, float *s, float *c, int count,
                             void *stream)
{
    g_rd_error.clear();
    if (count < 0) return rd_fail(RD_ERR_RANGE, "rd_joint_trig: count %d < 0", count);
    if (count == 0) return RD_OK;
    if (!x || !s || !c) return rd_fail(RD_ERR_ARG, "rd_joint_trig: null pointer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const unsigned grid = (unsigned)((count + 255) / 256);
    if (flags & RD_FLAG_FAST_TRIG) trig_kernel<true><<<grid, 256, 0, st>>>(x, s, c, count);
    else trig_kernel<false><<<grid, 256, 0, st>>>(x, s, c, count);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return rd_cuda_fail(e, "rd_joint_trig launch");
    return RD_OK;
}

extern "C" int rd_joint_trig_df(const double *x, double *s, double *c, int count, void *stream)
{
    g_rd_error.clear();
    if (count < 0) return rd_fail(RD_ERR_RANGE, "rd_joint_trig_df: count %d < 0", count);
    if (count == 0) return RD_OK;
    if (!x || !s || !c) return rd_fail(RD_ERR_ARG, "rd_joint_trig_df: null pointer");
    return rd_df_trig_launch(x, s, c, count, static_cast<cudaStream_t>(stream));
}
