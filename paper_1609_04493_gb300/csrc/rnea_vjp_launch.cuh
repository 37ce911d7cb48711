// rnea_vjp_launch.cuh -- launches of the adjoint kernel; included once per
// element type (vjp_f32.cu, vjp_f64.cu).
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "rdyn_internal.h"
#include "rnea_vjp.cuh"

namespace rdyn {
namespace {

int vjp_max_smem(int device)
{
    int v = 48 * 1024;
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    return v;
}

template <typename T, int BLOCK, int MODE, bool VEC, bool FAST>
int launch_vjp_k(const rd_model *m, int B, const void *q, const void *qd, const void *qdd,
                 const void *w, void *gq, void *gqd, void *gqdd, void *ws,
                 const double *base18, cudaStream_t stream)
{
    static std::atomic<uint64_t> configured{0};
    const int n = m->n;
    const size_t smem = (size_t)n * kLinkConsts * sizeof(T);
    auto kern = rnea_vjp_kernel<T, BLOCK, MODE, VEC, FAST>;
    const uint64_t bit = 1ull << (m->device & 63);
    if (!(configured.load() & bit)) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             vjp_max_smem(m->device));
        if (e != cudaSuccess) return rd_cuda_fail(e, "cudaFuncSetAttribute");
        configured.fetch_or(bit);
    }
    const T *consts = nullptr;
    if constexpr (sizeof(T) == 4) consts = reinterpret_cast<const T *>(m->d_c32);
    else consts = reinterpret_cast<const T *>(m->d_c64);
    BaseParams<T> bp;
    for (int k = 0; k < 6; ++k) {
        bp.V0[k] = (T)base18[k];
        bp.dV0[k] = (T)base18[6 + k];
        bp.Fn[k] = (T)base18[12 + k];
    }
    const unsigned grid = (unsigned)((B + BLOCK - 1) / BLOCK);
    kern<<<grid, BLOCK, smem, stream>>>(consts, n, B, static_cast<const T *>(q),
                                        static_cast<const T *>(qd), static_cast<const T *>(qdd),
                                        static_cast<const T *>(w), static_cast<T *>(gq),
                                        static_cast<T *>(gqd), static_cast<T *>(gqdd),
                                        static_cast<T *>(ws), bp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return rd_cuda_fail(e, "rnea_vjp kernel launch");
    return RD_OK;
}

inline bool vjp_aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

template <typename T, int MODE>
int launch_vjp_mode(const rd_model *m, int B, const void *q, const void *qd, const void *qdd,
                    const void *w, void *gq, void *gqd, void *gqdd, void *ws,
                    const double *base18, bool fast, cudaStream_t s)
{
    const bool vec = m->n % 4 == 0 && vjp_aligned16(q) && vjp_aligned16(qd) &&
                     vjp_aligned16(qdd) && vjp_aligned16(w) && vjp_aligned16(gq) &&
                     vjp_aligned16(gqd) && vjp_aligned16(gqdd);
    if constexpr (sizeof(T) == 4) {
        if (fast)
            return vec ? launch_vjp_k<T, 64, MODE, true, true>(m, B, q, qd, qdd, w, gq, gqd, gqdd, ws, base18, s)
                       : launch_vjp_k<T, 64, MODE, false, true>(m, B, q, qd, qdd, w, gq, gqd, gqdd, ws, base18, s);
    }
    return vec ? launch_vjp_k<T, 64, MODE, true, false>(m, B, q, qd, qdd, w, gq, gqd, gqdd, ws, base18, s)
               : launch_vjp_k<T, 64, MODE, false, false>(m, B, q, qd, qdd, w, gq, gqd, gqdd, ws, base18, s);
}

template <typename T>
int vjp_dispatch(const rd_model *m, int B, const void *q, const void *qd, const void *qdd,
                 const void *w, void *gq, void *gqd, void *gqdd, const double *base18, int mode,
                 void *ws, size_t ws_bytes, cudaStream_t s)
{
    const bool fast = (mode & RD_FLAG_FAST_TRIG) != 0;
    mode &= 0xff;
    const size_t need = (size_t)m->n * kVjpStateScalars * (size_t)B * sizeof(T);
    if (mode == RD_VJP_AUTO) {
        // Measured at n = 32: in FP32 re-deriving the state beats the extra
        // workspace traffic (B = 65536: 51 us vs 78 us); in FP64 the FP64 pipe is
        // the bound and storing saves work (B = 8192: 421 us vs 512 us).
        mode = (sizeof(T) == 8 && ws && ws_bytes >= need) ? RD_VJP_STORE : RD_VJP_RECOMPUTE;
    }
    if (mode == RD_VJP_STORE) {
        if (!ws || ws_bytes < need)
            return rd_fail(RD_ERR_ARG, "rnea_vjp: store mode needs a %zu-byte workspace (%zu given)",
                           need, ws_bytes);
        if (!vjp_aligned16(ws)) return rd_fail(RD_ERR_ARG, "rnea_vjp: workspace not 16-byte aligned");
        return launch_vjp_mode<T, kVjpStore>(m, B, q, qd, qdd, w, gq, gqd, gqdd, ws, base18, fast, s);
    }
    if (mode == RD_VJP_RECOMPUTE)
        return launch_vjp_mode<T, kVjpRecompute>(m, B, q, qd, qdd, w, gq, gqd, gqdd, nullptr, base18,
                                                 fast, s);
    return rd_fail(RD_ERR_ARG, "rnea_vjp: unknown mode %d", mode);
}

}  // namespace
}  // namespace rdyn
