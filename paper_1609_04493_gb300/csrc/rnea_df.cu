// rnea_df.cu -- launches of the double-float inverse-dynamics kernel for FP64
// data (rnea_df.cuh), and of its sine / cosine for rd_joint_trig_df.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "rdyn_internal.h"
#include "rnea_df.cuh"

namespace rdyn {
namespace {

template <int NMAX, int BLOCK>
int launch_df_k(const rd_model *m, int B, const void *q, const void *qd, const void *qdd,
                void *tau, const double *base18, cudaStream_t stream)
{
    static std::atomic<uint64_t> configured{0};
    const int n = m->n;
    auto kern = rnea_df_kernel<NMAX, BLOCK>;
    const size_t smem = (size_t)n * BLOCK * sizeof(float4);
    const uint64_t bit = 1ull << (m->device & 63);
    if (!(configured.load() & bit)) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)((size_t)NMAX * BLOCK * sizeof(float4)));
        if (e != cudaSuccess) return rd_cuda_fail(e, "cudaFuncSetAttribute");
        configured.fetch_or(bit);
    }
    DfParamConsts<NMAX> pc;
    for (int k = 0; k < NMAX * kDhConsts; ++k)
        pc.c[k] = df_split_host(k < n * kDhConsts ? m->host_dh64[k] : 0.0);
    for (int i = 0; i < NMAX; ++i) pc.th0[i] = i < n ? m->host_dh64[(size_t)i * kDhConsts + 5] : 0.0;
    double bb[18];
    rd_convert_base_dh(m, base18, bb);
    BaseParams<DF> bp;
    for (int k = 0; k < 6; ++k) {
        bp.V0[k] = df_split_host(bb[k]);
        bp.dV0[k] = df_split_host(bb[6 + k]);
        bp.Fn[k] = df_split_host(bb[12 + k]);
    }
    const unsigned grid = (unsigned)((B + BLOCK - 1) / BLOCK);
    rd_note_rnea(RD_VARIANT_SERIAL_DF, BLOCK, 0);
    kern<<<grid, BLOCK, smem, stream>>>(pc, n, B, static_cast<const double *>(q),
                                        static_cast<const double *>(qd),
                                        static_cast<const double *>(qdd),
                                        static_cast<double *>(tau), bp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return rd_cuda_fail(e, "rnea double-float kernel launch");
    return RD_OK;
}

__global__ void df_trig_kernel(const double *__restrict__ x, double *__restrict__ s,
                               double *__restrict__ c, int count)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    DF sv, cv;
    df_sincos(x[i], &sv, &cv);
    s[i] = df_to_double(sv);
    c[i] = df_to_double(cv);
}

}  // namespace
}  // namespace rdyn

int rd_rnea_df_f64(const rd_model *m, int B, const void *q, const void *qd, const void *qdd,
                   void *tau, const double *base18, int block, cudaStream_t s)
{
    if (m->n > 64)
        return rd_fail(RD_ERR_ARG, "rnea_batch: the double-float kernel is built for n <= 64 (n = %d)",
                       m->n);
    if (!block) block = 64;  // n = 32, B = 65536: 263.7 us against 273.0 with 32 threads
    if (block != 32 && block != 64)
        return rd_fail(RD_ERR_ARG, "rnea_batch: double-float kernel built for 32 or 64 threads (%d)",
                       block);
    if (m->n <= 32)
        return block == 32 ? rdyn::launch_df_k<32, 32>(m, B, q, qd, qdd, tau, base18, s)
                           : rdyn::launch_df_k<32, 64>(m, B, q, qd, qdd, tau, base18, s);
    return block == 32 ? rdyn::launch_df_k<64, 32>(m, B, q, qd, qdd, tau, base18, s)
                       : rdyn::launch_df_k<64, 64>(m, B, q, qd, qdd, tau, base18, s);
}

int rd_df_trig_launch(const double *x, double *s, double *c, int count, cudaStream_t stream)
{
    if (count <= 0) return RD_OK;
    rdyn::df_trig_kernel<<<(count + 255) / 256, 256, 0, stream>>>(x, s, c, count);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return rd_cuda_fail(e, "double-float trig kernel launch");
    return RD_OK;
}
