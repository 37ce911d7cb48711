// aba_pair_f32.cu -- float instantiations of the two-warp forward-dynamics
// kernel (aba_pair.cuh).
#include <cuda_runtime.h>

#include <type_traits>

#include "aba_pair.cuh"
#include "rdyn_internal.h"

namespace rdyn {
namespace {

template <typename T, typename D, typename TB>
int launch_aba_pair(const rd_model *m, int B, const void *q, const void *qd, const void *tau,
                    void *qdd, int *status, void *ws, const double *base18, cudaStream_t stream)
{
    constexpr bool kExt = !std::is_same<TB, T>::value;
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
    (void)kExt;
    const unsigned grid = (unsigned)((B + 31) / 32);
    aba_pair_kernel<T, D, TB, kTrigPoly><<<grid, 64, 0, stream>>>(
        sc, sd, sdf, n, B, static_cast<const T *>(q), static_cast<const T *>(qd),
        static_cast<const T *>(tau), static_cast<T *>(qdd), status, static_cast<T *>(ws), wsz, bp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return rd_cuda_fail(e, "aba two-warp kernel launch");
    return RD_OK;
}

}  // namespace
}  // namespace rdyn

int rd_aba_pair_f32(const rd_model *m, int B, const void *q, const void *qd, const void *tau,
                    void *qdd, int *status, void *ws, const double *base18, bool fp64_update,
                    bool extended_bias, cudaStream_t s)
{
    using rdyn::DF;
    if (extended_bias)
        return fp64_update
                   ? rdyn::launch_aba_pair<float, double, DF>(m, B, q, qd, tau, qdd, status, ws, base18, s)
                   : rdyn::launch_aba_pair<float, DF, DF>(m, B, q, qd, tau, qdd, status, ws, base18, s);
    return fp64_update
               ? rdyn::launch_aba_pair<float, double, float>(m, B, q, qd, tau, qdd, status, ws, base18, s)
               : rdyn::launch_aba_pair<float, DF, float>(m, B, q, qd, tau, qdd, status, ws, base18, s);
}

int rd_aba_pair_f64(const rd_model *m, int B, const void *q, const void *qd, const void *tau,
                    void *qdd, int *status, void *ws, const double *base18, cudaStream_t s)
{
    return rdyn::launch_aba_pair<double, double, double>(m, B, q, qd, tau, qdd, status, ws, base18, s);
}
