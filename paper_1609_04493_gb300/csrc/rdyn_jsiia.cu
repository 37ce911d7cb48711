// rdyn_jsiia.cu -- jsiia_batch: forward dynamics by joint-space-inertia
// inversion for chains of at most 32 links.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "jsiia.cuh"
#include "rdyn_internal.h"

namespace {

constexpr int kWarps = 4;

template <typename T>
int run_jsiia(const rd_model *m, int B, const void *q, const void *qd, const void *tau, void *qdd,
              int *status, const double *b18, cudaStream_t s)
{
    static std::atomic<uint64_t> configured{0};
    auto kern = rdyn::jsiia_kernel<T, kWarps>;
    const size_t smem = rdyn::jsiia_smem_bytes<T, kWarps>(m->n);
    const uint64_t bit = 1ull << (m->device & 63);
    if (!(configured.load() & bit)) {
        int lim = 48 * 1024;
        cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, m->device);
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        if (e != cudaSuccess) return rd_cuda_fail(e, "cudaFuncSetAttribute");
        configured.fetch_or(bit);
    }
    const T *consts = nullptr;
    if constexpr (sizeof(T) == 4) consts = reinterpret_cast<const T *>(m->d_c32);
    else consts = reinterpret_cast<const T *>(m->d_c64);
    rdyn::BaseParams<T> bp;
    for (int k = 0; k < 6; ++k) {
        bp.V0[k] = (T)b18[k];
        bp.dV0[k] = (T)b18[6 + k];
        bp.Fn[k] = (T)b18[12 + k];
    }
    const unsigned grid = (unsigned)((B + kWarps - 1) / kWarps);
    kern<<<grid, 32 * kWarps, smem, s>>>(consts, m->n, B, static_cast<const T *>(q),
                                         static_cast<const T *>(qd), static_cast<const T *>(tau),
                                         static_cast<T *>(qdd), status, bp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return rd_cuda_fail(e, "jsiia kernel launch");
    return RD_OK;
}

}  // namespace

extern "C" int jsiia_batch(const rd_model *m, int B, int dtype, const void *q, const void *qd,
                           const void *tau, void *qdd, const double *base, int *status,
                           void *stream)
{
    g_rd_error.clear();
    if (!m) return rd_fail(RD_ERR_ARG, "jsiia_batch: null model");
    if (m->n > 32)
        return rd_fail(RD_ERR_RANGE, "jsiia_batch: n = %d; the joint-space solve takes n <= 32 "
                                     "(use aba_batch)", m->n);
    if (B < 0) return rd_fail(RD_ERR_RANGE, "jsiia_batch: B = %d < 0", B);
    if (dtype != RD_F32 && dtype != RD_F64)
        return rd_fail(RD_ERR_DTYPE, "jsiia_batch: dtype %d is not RD_F32 or RD_F64", dtype);
    if (B == 0) return RD_OK;
    if (!q || !qd || !tau || !qdd) return rd_fail(RD_ERR_ARG, "jsiia_batch: null batch pointer");
    if (qdd == q || qdd == qd || qdd == tau)
        return rd_fail(RD_ERR_ARG, "jsiia_batch: qdd aliases an input");
    double b18[18];
    rd_convert_base(m, base, b18);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (dtype == RD_F32) return run_jsiia<float>(m, B, q, qd, tau, qdd, status, b18, s);
    return run_jsiia<double>(m, B, q, qd, tau, qdd, status, b18, s);
}
