// vjp_lane_f32.cu -- launches of the lane-parallel adjoint (rnea_vjp_lane.cuh),
// FP32 data, common-normal frames, no workspace.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "rdyn_internal.h"
#include "rnea_vjp_lane.cuh"

namespace rdyn {
namespace {

template <int NMAX, int L, int K, int TRIG>
int launch_vjp_lane_k(const rd_model *m, int B, const void *q, const void *qd, const void *qdd,
                      const void *w, void *gq, void *gqd, void *gqdd, const double *base18,
                      cudaStream_t stream)
{
    constexpr int BLOCK = 128;
    static std::atomic<uint64_t> configured{0};
    const size_t smem = ((size_t)NMAX * kVjpLaneConstStride + (size_t)K * kVjpLaneScalars * BLOCK) *
                        sizeof(float);
    auto kern = rnea_vjp_lane_kernel<float, NMAX, L, K, BLOCK, TRIG>;
    const uint64_t bit = 1ull << (m->device & 63);
    if (smem > 48 * 1024 && !(configured.load() & bit)) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return rd_cuda_fail(e, "cudaFuncSetAttribute");
        configured.fetch_or(bit);
    }
    double b[18];
    rd_convert_base_dh(m, base18, b);
    BaseParams<float> bp;
    for (int k = 0; k < 6; ++k) {
        bp.V0[k] = (float)b[k];
        bp.dV0[k] = (float)b[6 + k];
        bp.Fn[k] = (float)b[12 + k];
    }
    DhParamConsts<float, NMAX> pc;
    for (int k = 0; k < m->n * kDhConsts; ++k) pc.c[k] = (float)m->host_dh64[k];
    for (int k = m->n * kDhConsts; k < NMAX * kDhConsts; ++k) pc.c[k] = 0.0f;
    const long long threads = (long long)B * L;
    const unsigned grid = (unsigned)((threads + BLOCK - 1) / BLOCK);
    kern<<<grid, BLOCK, smem, stream>>>(pc, m->n, B, static_cast<const float *>(q),
                                        static_cast<const float *>(qd),
                                        static_cast<const float *>(qdd),
                                        static_cast<const float *>(w), static_cast<float *>(gq),
                                        static_cast<float *>(gqd), static_cast<float *>(gqdd), bp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return rd_cuda_fail(e, "rnea_vjp lane-parallel kernel launch");
    return RD_OK;
}

template <int TRIG>
int launch_vjp_lane(const rd_model *m, int B, const void *q, const void *qd, const void *qdd,
                    const void *w, void *gq, void *gqd, void *gqdd, const double *base18,
                    int lanes, cudaStream_t s)
{
    const int n = m->n;
    if (lanes == 4) {
        if (n <= 16)
            return launch_vjp_lane_k<32, 4, 4, TRIG>(m, B, q, qd, qdd, w, gq, gqd, gqdd, base18, s);
        if (n <= 32)
            return launch_vjp_lane_k<32, 4, 8, TRIG>(m, B, q, qd, qdd, w, gq, gqd, gqdd, base18, s);
    }
    if (n <= 32)
        return launch_vjp_lane_k<32, 8, 4, TRIG>(m, B, q, qd, qdd, w, gq, gqd, gqdd, base18, s);
    if (n <= 64)
        return launch_vjp_lane_k<64, 8, 8, TRIG>(m, B, q, qd, qdd, w, gq, gqd, gqdd, base18, s);
    return launch_vjp_lane_k<128, 8, 16, TRIG>(m, B, q, qd, qdd, w, gq, gqd, gqdd, base18, s);
}

}  // namespace
}  // namespace rdyn

int rd_vjp_lane_f32(const rd_model *m, int B, const void *q, const void *qd, const void *qdd,
                    const void *w, void *gq, void *gqd, void *gqdd, const double *base18,
                    bool fast_trig, int lanes, cudaStream_t s)
{
    if (fast_trig)
        return rdyn::launch_vjp_lane<rdyn::kTrigSfu>(m, B, q, qd, qdd, w, gq, gqd, gqdd, base18,
                                                     lanes, s);
    return rdyn::launch_vjp_lane<rdyn::kTrigPoly>(m, B, q, qd, qdd, w, gq, gqd, gqdd, base18,
                                                  lanes, s);
}
