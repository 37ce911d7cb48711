// rnea_dhz.cu -- launches of the inverse-dynamics kernel that reads and
// writes mapped pinned host arrays itself (rnea_dhz.cuh).
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "rdyn_internal.h"
#include "rnea_dhz.cuh"

namespace rdyn {
namespace {

template <int NMAX, int BLOCK>
int launch_dhz_k(const rd_model *m, int B, const float *q, const float *qd, const float *qdd,
                 float *tau, const double *base18, cudaStream_t stream)
{
    static std::atomic<uint64_t> configured{0};
    const int n = m->n;
    auto kern = rnea_dhz_kernel<NMAX, BLOCK>;
    const size_t smem = (size_t)4 * BLOCK * (n + 1) * sizeof(float);
    const uint64_t bit = 1ull << (m->device & 63);
    if (!(configured.load() & bit)) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)((size_t)4 * BLOCK * (NMAX + 1) * sizeof(float)));
        if (e != cudaSuccess) return rd_cuda_fail(e, "cudaFuncSetAttribute");
        configured.fetch_or(bit);
    }
    DhParamConsts<float, NMAX> pc;
    for (int k = 0; k < NMAX * kDhConsts; ++k)
        pc.c[k] = k < n * kDhConsts ? (float)m->host_dh64[k] : 0.0f;
    double bb[18];
    rd_convert_base_dh(m, base18, bb);
    BaseParams<float> bp;
    for (int k = 0; k < 6; ++k) {
        bp.V0[k] = (float)bb[k];
        bp.dV0[k] = (float)bb[6 + k];
        bp.Fn[k] = (float)bb[12 + k];
    }
    // blocks per SM (n = 32, B = 65536, 32 threads): 1: 246 us, 2: 171, 3 or 4:
    // 160, 6: 164, 8: 158, 13 (all slabs resident at once): 179; the staged
    // copies take 209
    constexpr int per_sm = 8;
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device);
    const long long slabs = (B + BLOCK - 1) / BLOCK;
    const unsigned grid = (unsigned)(slabs < (long long)sms * per_sm ? slabs : (long long)sms * per_sm);
    rd_note_rnea(RD_RNEA_KERNEL_DH_HOST, BLOCK, 0);
    kern<<<grid, BLOCK, smem, stream>>>(pc, n, B, q, qd, qdd, tau, bp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return rd_cuda_fail(e, "rnea host-memory kernel launch");
    return RD_OK;
}

}  // namespace
}  // namespace rdyn

int rd_rnea_dhz_f32(const rd_model *m, int B, const void *q, const void *qd, const void *qdd,
                    void *tau, const double *base18, cudaStream_t s)
{
    const float *a = static_cast<const float *>(q), *b = static_cast<const float *>(qd);
    const float *c = static_cast<const float *>(qdd);
    float *t = static_cast<float *>(tau);
    if (m->n <= 32) return rdyn::launch_dhz_k<32, 32>(m, B, a, b, c, t, base18, s);
    return rdyn::launch_dhz_k<64, 32>(m, B, a, b, c, t, base18, s);
}
