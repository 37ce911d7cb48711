// aba_pair_launch.cuh -- host launcher of the forward-dynamics kernels with two
// (aba_pair.cuh) or three (aba_tri.cuh) warps per 32 instances.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "aba_tri.cuh"
#include "rdyn_internal.h"

namespace rdyn {

// One block per 32 instances, WARPS warps per block. Workspace: the sweep-1
// state in the bias precision TB, then (256-byte aligned) the solve state in D.
// withhold: the two-warp kernel's test hook (aba_pair_kernel).
template <typename T, typename D, typename TB, int WARPS>
int launch_aba_multi(const rd_model *m, int B, const void *q, const void *qd, const void *tau,
                     void *qdd, int *status, void *ws, const double *base18, cudaStream_t stream,
                     bool withhold = false)
{
    static_assert(WARPS == 2 || WARPS == 3, "two or three warps per 32 instances");
    const int n = m->n;
    double bb[18];
    rd_convert_base_dh(m, base18, bb);
    BaseParams<T> bp;
    for (int k = 0; k < 6; ++k) {
        bp.V0[k] = (T)bb[k];
        bp.dV0[k] = (T)bb[6 + k];
        bp.Fn[k] = (T)bb[12 + k];
    }
    const T *sc = nullptr;
    if constexpr (sizeof(T) == 4) sc = reinterpret_cast<const T *>(m->d_dh32);
    else sc = reinterpret_cast<const T *>(m->d_dh64);
    const D *sd = nullptr;
    if constexpr (std::is_same<D, double>::value) sd = m->d_aba64;
    else sd = reinterpret_cast<const D *>(m->d_abadf);
    const DF *sdf = reinterpret_cast<const DF *>(m->d_abadf);
    const size_t a = (size_t)n * aba_bias_ws_scalars<T, TB>() * (size_t)B * sizeof(T);
    D *wsz = reinterpret_cast<D *>(static_cast<char *>(ws) + ((a + 255) & ~(size_t)255));
    const unsigned grid = (unsigned)((B + 31) / 32);
    if constexpr (WARPS == 2)
        aba_pair_kernel<T, D, TB, kTrigPoly><<<grid, 64, 0, stream>>>(
            sc, sd, sdf, n, B, static_cast<const T *>(q), static_cast<const T *>(qd),
            static_cast<const T *>(tau), static_cast<T *>(qdd), status, static_cast<T *>(ws), wsz,
            bp, withhold ? 1 : 0);
    else
        aba_tri_kernel<T, D, TB, kTrigPoly><<<grid, 96, 0, stream>>>(
            sc, sd, sdf, n, B, static_cast<const T *>(q), static_cast<const T *>(qd),
            static_cast<const T *>(tau), static_cast<T *>(qdd), status, static_cast<T *>(ws), wsz,
            bp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return rd_cuda_fail(e, WARPS == 2 ? "aba two-warp kernel launch" : "aba three-warp kernel launch");
    return RD_OK;
}

}  // namespace rdyn
