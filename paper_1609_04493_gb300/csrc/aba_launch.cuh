// aba_launch.cuh -- launches of the forward-dynamics kernel; included once
// per element type (aba_f32.cu, aba_f64.cu).
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <type_traits>

#include "aba.cuh"
#include "aba_dh.cuh"
#include "rdyn_internal.h"

namespace rdyn {
namespace {

inline bool aba_aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Bias sweeps in double-float (FP32 data): by flag, or for chains longer than
// RD_ABA_EXTENDED_BIAS_LINKS unless RD_ABA_FP32_BIAS asks for FP32.
template <typename T>
bool aba_extended_bias(int n, int flags)
{
    if (sizeof(T) != 4 || (flags & RD_ABA_JOINT_FRAMES)) return false;
    if (flags & RD_ABA_EXTENDED_BIAS) return true;
    return n > RD_ABA_EXTENDED_BIAS_LINKS && !(flags & RD_ABA_FP32_BIAS);
}

// bytes of the sweep-1 state (F_hat, cos, sin per link)
template <typename T>
size_t aba_bias_bytes(int n, int B, bool extended)
{
    const int per = extended ? aba_bias_ws_scalars<T, DF>() : aba_bias_ws_scalars<T, T>();
    return (size_t)n * per * (size_t)B * sizeof(T);
}

template <typename T>
size_t aba_ws_bytes(int n, int B, int flags)
{
    const bool fp32_scans = sizeof(T) == 4 && (flags & RD_ABA_SCANS_IN_DTYPE);
    const size_t a = aba_bias_bytes<T>(n, B, aba_extended_bias<T>(n, flags));
    const size_t a16 = (a + 255) & ~(size_t)255;
    return a16 + (size_t)n * kAbaSolveScalars * (size_t)B * (fp32_scans ? sizeof(T) : sizeof(double));
}

template <typename T, typename Z, int BLOCK, bool VEC>
int launch_aba_k(const rd_model *m, int B, const void *q, const void *qd, const void *tau,
                 void *qdd, int *status, void *ws, const double *base18, cudaStream_t stream)
{
    static std::atomic<uint64_t> configured{0};
    const int n = m->n;
    const size_t smem = (((size_t)n * kLinkConsts * sizeof(T) + 15) & ~(size_t)15) +
                        (size_t)n * kLinkConsts * sizeof(double);
    auto kern = aba_kernel<T, Z, BLOCK, VEC>;
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
    BaseParams<T> bp;
    for (int k = 0; k < 6; ++k) {
        bp.V0[k] = (T)base18[k];
        bp.dV0[k] = (T)base18[6 + k];
        bp.Fn[k] = (T)base18[12 + k];
    }
    const unsigned grid = (unsigned)((B + BLOCK - 1) / BLOCK);
    const size_t a = (size_t)n * kAbaStateScalars * (size_t)B * sizeof(T);
    Z *wsz = reinterpret_cast<Z *>(static_cast<char *>(ws) + ((a + 255) & ~(size_t)255));
    kern<<<grid, BLOCK, smem, stream>>>(consts, m->d_c64, n, B, static_cast<const T *>(q),
                                        static_cast<const T *>(qd), static_cast<const T *>(tau),
                                        static_cast<T *>(qdd), status, static_cast<T *>(ws), wsz,
                                        bp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return rd_cuda_fail(e, "aba kernel launch");
    return RD_OK;
}

template <typename T, typename D, typename Z, int NMAX, int TRIG>
int launch_aba_dh_k(const rd_model *m, int B, const void *q, const void *qd, const void *tau,
                    void *qdd, int *status, void *ws, const double *base18, cudaStream_t stream)
{
    constexpr int BLOCK = 64;
    const int n = m->n;
    double bb[18];
    rd_convert_base_dh(m, base18, bb);
    BaseParams<T> bp;
    for (int k = 0; k < 6; ++k) {
        bp.V0[k] = (T)bb[k];
        bp.dV0[k] = (T)bb[6 + k];
        bp.Fn[k] = (T)bb[12 + k];
    }
    AbaDhConsts<T, D, NMAX> pc;
    for (int k = 0; k < NMAX * kDhConsts; ++k)
        pc.c[k] = k < n * kDhConsts ? (T)m->host_dh64[k] : T(0);
    for (int k = 0; k < NMAX * kAbaDh64; ++k) {
        const double v = k < n * kAbaDh64 ? m->host_aba64[k] : 0.0;
        if constexpr (std::is_same<D, double>::value) pc.d[k] = v;
        else pc.d[k] = df_split_host(v);
    }
    const size_t a = (size_t)n * kAbaStateScalars * (size_t)B * sizeof(T);
    Z *wsz = reinterpret_cast<Z *>(static_cast<char *>(ws) + ((a + 255) & ~(size_t)255));
    const unsigned grid = (unsigned)((B + BLOCK - 1) / BLOCK);
    aba_dh_kernel<T, D, Z, NMAX, BLOCK, TRIG><<<grid, BLOCK, 0, stream>>>(
        pc, n, B, static_cast<const T *>(q), static_cast<const T *>(qd),
        static_cast<const T *>(tau), static_cast<T *>(qdd), status, static_cast<T *>(ws), wsz, bp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return rd_cuda_fail(e, "aba common-normal kernel launch");
    return RD_OK;
}

template <typename T, typename D, typename Z>
int launch_aba_dh(const rd_model *m, int B, const void *q, const void *qd, const void *tau,
                  void *qdd, int *status, void *ws, const double *base18, cudaStream_t s)
{
    if (m->n <= 32)
        return launch_aba_dh_k<T, D, Z, 32, kTrigPoly>(m, B, q, qd, tau, qdd, status, ws, base18, s);
    return launch_aba_dh_k<T, D, Z, 64, kTrigPoly>(m, B, q, qd, tau, qdd, status, ws, base18, s);
}

template <typename T, typename D, typename Z, bool VEC, typename TB = T>
int launch_aba_dhg(const rd_model *m, int B, const void *q, const void *qd, const void *tau,
                   void *qdd, int *status, void *ws, const double *base18, cudaStream_t stream)
{
    constexpr bool kExt = !std::is_same<TB, T>::value;
    constexpr int BLOCK = 64;
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
    const size_t a = aba_bias_bytes<T>(n, B, kExt);
    Z *wsz = reinterpret_cast<Z *>(static_cast<char *>(ws) + ((a + 255) & ~(size_t)255));
    const DF *sdf = kExt ? reinterpret_cast<const DF *>(m->d_abadf) : nullptr;
    if (kExt && !sdf) return rd_fail(RD_ERR_ARG, "aba_batch: model has no double-float records");
    const unsigned grid = (unsigned)((B + BLOCK - 1) / BLOCK);
    aba_dhg_kernel<T, D, Z, BLOCK, VEC, TB><<<grid, BLOCK, 0, stream>>>(
        sc, sd, n, B, static_cast<const T *>(q), static_cast<const T *>(qd),
        static_cast<const T *>(tau), static_cast<T *>(qdd), status, static_cast<T *>(ws), wsz, bp,
        sdf);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return rd_cuda_fail(e, "aba global-constant kernel launch");
    return RD_OK;
}

template <typename T, typename D, typename Z>
int launch_aba_dhg_v(bool vec, bool ext, const rd_model *m, int B, const void *q, const void *qd,
                     const void *tau, void *qdd, int *status, void *ws, const double *base18,
                     cudaStream_t s)
{
    if constexpr (sizeof(T) == 4) {
        if (ext)
            return vec ? launch_aba_dhg<T, D, Z, true, DF>(m, B, q, qd, tau, qdd, status, ws, base18, s)
                       : launch_aba_dhg<T, D, Z, false, DF>(m, B, q, qd, tau, qdd, status, ws, base18, s);
    }
    return vec ? launch_aba_dhg<T, D, Z, true>(m, B, q, qd, tau, qdd, status, ws, base18, s)
               : launch_aba_dhg<T, D, Z, false>(m, B, q, qd, tau, qdd, status, ws, base18, s);
}

// Warp per instance or thread per instance: by flag, else by the crossover
// measured on GB300 (FP32 data, double-float updates, warp / thread time:
// n = 64: 0.67 at B = 256, 0.85 at 1024, 3.2 at 4096; n = 100: 0.45 / 0.54 /
// 2.0; n = 32: 0.94 / 1.12; n = 16: 1.7 at B = 256, never faster. With FP64
// updates the warp's FP64 work saturates sooner: n = 64: 0.59 at 256, 1.08 at
// 1024). The scans' fixed cost keeps short chains on threads.
template <typename T>
bool aba_use_warp(int n, int B, int flags)
{
    if (flags & RD_ABA_WARP_PER_INSTANCE) return true;
    if (flags & (RD_ABA_THREAD_PER_INSTANCE | RD_ABA_JOINT_FRAMES | RD_ABA_SCANS_IN_DTYPE))
        return false;
    if (n < 48) return false;
    const bool fp64 = sizeof(T) == 8 || (flags & RD_ABA_FP64_UPDATE);
    // against two warps per 32 instances (aba_use_pair), n = 64: warp 180 vs
    // 201 us at B = 256, 226 vs 205 at 1024; n = 100 and 128: the warp wins up
    // to B = 1024 (388 vs 434, 430 vs 563)
    return B <= (fp64 || n < 96 ? 512 : 1024);
}

// Two warps per 32 instances: by flag, else for FP32 data where the measured
// times favour it over one thread per instance (double-float updates, thread /
// pair: n = 16: 1.25 at B = 1024, 1.04 at 16384, 0.80 at 65536; n = 64: 1.31 /
// 1.17 / 0.76; n = 100: 1.90 / 1.20; FP64 updates: n = 64: 1.15 at 1024, 1.03 at
// 16384, 1.05 at 65536; n = 100: 1.46 / 1.19) and the warp-per-instance mapping
// does not apply.
template <typename T>
bool aba_use_pair(int n, int B, int flags)
{
    if (flags & RD_ABA_TWO_WARPS) return true;
    if (sizeof(T) != 4 || (flags & (RD_ABA_THREAD_PER_INSTANCE | RD_ABA_WARP_PER_INSTANCE |
                                    RD_ABA_THREE_WARPS | RD_ABA_JOINT_FRAMES |
                                    RD_ABA_SCANS_IN_DTYPE)))
        return false;
    if (aba_use_warp<T>(n, B, flags)) return false;
    return (flags & RD_ABA_FP64_UPDATE) ? true : B <= 16384;
}

// Three warps per 32 instances (aba_tri.cuh): by flag, else for FP32 data where
// the measured times favour it (GB300, CUDA events, two-warp /
// three-warp time): double-float updates, n = 16: 1.27 at B = 1024, 1.01 at
// 4096, 0.99 at 16384; n = 32: 1.23 / 0.99 / 0.99; n = 64: 1.22 at B = 256 and
// 1024, 0.98 / 0.96 (and 161 us against 180 for one warp per instance at n = 64,
// B = 256); with the double-float bias sweeps beyond 64 links the split does not
// pay (n = 100: 0.99 at 1024, 0.82 at 4096). FP64 updates: 1.21 to 1.31 up to B =
// 4096 for n = 16 to 100, 0.92 to 0.97 at 16384; below B = 512 one warp per
// instance stays ahead for n >= 48. Beyond the crossover every instance is
// resident at once and the kernels stall on instruction fetch; the third warp
// then adds work without shortening the chain.
template <typename T>
bool aba_use_tri(int n, int B, int flags, bool ext)
{
    if (flags & RD_ABA_THREE_WARPS) return true;
    if (sizeof(T) != 4 ||
        (flags & (RD_ABA_THREAD_PER_INSTANCE | RD_ABA_WARP_PER_INSTANCE | RD_ABA_TWO_WARPS |
                  RD_ABA_JOINT_FRAMES | RD_ABA_SCANS_IN_DTYPE)))
        return false;
    if (flags & RD_ABA_FP64_UPDATE) return B <= 4096 && !aba_use_warp<T>(n, B, flags);
    return !ext && B <= 2048;
}

template <typename T>
int aba_dispatch(const rd_model *m, int B, const void *q, const void *qd, const void *tau,
                 void *qdd, int *status, void *ws, size_t ws_bytes, const double *base18,
                 int flags, cudaStream_t s)
{
    const bool fp32_scans = sizeof(T) == 4 && (flags & RD_ABA_SCANS_IN_DTYPE);
    const bool ext = aba_extended_bias<T>(m->n, flags);
    const size_t need = aba_ws_bytes<T>(m->n, B, flags);
    if (!ws || ws_bytes < need)
        return rd_fail(RD_ERR_ARG, "aba_batch: needs a %zu-byte workspace (%zu given)", need,
                       ws_bytes);
    if (!aba_aligned16(ws)) return rd_fail(RD_ERR_ARG, "aba_batch: workspace not 16-byte aligned");
    {
        const int maps = !!(flags & RD_ABA_WARP_PER_INSTANCE) + !!(flags & RD_ABA_TWO_WARPS) +
                         !!(flags & RD_ABA_THREE_WARPS) + !!(flags & RD_ABA_THREAD_PER_INSTANCE);
        if (maps > 1 ||
            ((flags & (RD_ABA_WARP_PER_INSTANCE | RD_ABA_TWO_WARPS | RD_ABA_THREE_WARPS)) &&
             (flags & (RD_ABA_JOINT_FRAMES | RD_ABA_SCANS_IN_DTYPE))))
            return rd_fail(RD_ERR_ARG, "aba_batch: RD_ABA_WARP_PER_INSTANCE, RD_ABA_TWO_WARPS, "
                                       "RD_ABA_THREE_WARPS and RD_ABA_THREAD_PER_INSTANCE exclude "
                                       "one another, and the first three RD_ABA_JOINT_FRAMES and "
                                       "RD_ABA_SCANS_IN_DTYPE");
    }
    const bool withhold = (flags & RD_ABA_TEST_WITHHOLD) != 0;
    if (withhold && !(flags & RD_ABA_TWO_WARPS))
        return rd_fail(RD_ERR_ARG, "aba_batch: RD_ABA_TEST_WITHHOLD needs RD_ABA_TWO_WARPS");
    if (aba_use_tri<T>(m->n, B, flags, ext)) {
        if constexpr (sizeof(T) == 4)
            return rd_aba_tri_f32(m, B, q, qd, tau, qdd, status, ws, base18,
                                  (flags & RD_ABA_FP64_UPDATE) != 0, ext, s);
        else
            return rd_aba_tri_f64(m, B, q, qd, tau, qdd, status, ws, base18, s);
    }
    if (aba_use_pair<T>(m->n, B, flags)) {
        if constexpr (sizeof(T) == 4)
            return rd_aba_pair_f32(m, B, q, qd, tau, qdd, status, ws, base18,
                                   (flags & RD_ABA_FP64_UPDATE) != 0, ext, withhold, s);
        else
            return rd_aba_pair_f64(m, B, q, qd, tau, qdd, status, ws, base18, withhold, s);
    }
    if (aba_use_warp<T>(m->n, B, flags)) {
        if constexpr (sizeof(T) == 4)
            return rd_aba_warp_f32(m, B, q, qd, tau, qdd, status, base18,
                                   (flags & RD_ABA_FP64_UPDATE) != 0, ext, s);
        else
            return rd_aba_warp_f64(m, B, q, qd, tau, qdd, status, base18, s);
    }
    const bool vec = m->n % 4 == 0 && aba_aligned16(q) && aba_aligned16(qd) &&
                     aba_aligned16(tau) && aba_aligned16(qdd);
    if (vec && m->n <= 64 && !ext && !(flags & RD_ABA_JOINT_FRAMES)) {
        // common-normal frames, constants as a kernel parameter (aba_dh.cuh)
        if constexpr (sizeof(T) == 4) {
            if (!(flags & RD_ABA_FP64_UPDATE))
                return fp32_scans
                           ? launch_aba_dh<T, DF, T>(m, B, q, qd, tau, qdd, status, ws, base18, s)
                           : launch_aba_dh<T, DF, DF>(m, B, q, qd, tau, qdd, status, ws, base18, s);
            if (fp32_scans)
                return launch_aba_dh<T, double, T>(m, B, q, qd, tau, qdd, status, ws, base18, s);
        }
        return launch_aba_dh<T, double, double>(m, B, q, qd, tau, qdd, status, ws, base18, s);
    }
    if (!(flags & RD_ABA_JOINT_FRAMES)) {
        // common-normal frames, constants and records in global memory
        if constexpr (sizeof(T) == 4) {
            if (!(flags & RD_ABA_FP64_UPDATE)) {
                if (fp32_scans)
                    return launch_aba_dhg_v<T, DF, T>(vec, ext, m, B, q, qd, tau, qdd, status, ws, base18, s);
                return launch_aba_dhg_v<T, DF, DF>(vec, ext, m, B, q, qd, tau, qdd, status, ws, base18, s);
            }
            if (fp32_scans)
                return launch_aba_dhg_v<T, double, T>(vec, ext, m, B, q, qd, tau, qdd, status, ws, base18, s);
        }
        return launch_aba_dhg_v<T, double, double>(vec, ext, m, B, q, qd, tau, qdd, status, ws, base18, s);
    }
    // joint frames (RD_ABA_JOINT_FRAMES), full 6x6 congruence (aba.cuh); its
    // bias sweeps stay in FP32 for FP32 data, which meets the 1e-3 bar on qdd
    // only up to RD_ABA_EXTENDED_BIAS_LINKS links
    if constexpr (sizeof(T) == 4) {
        if (m->n > RD_ABA_EXTENDED_BIAS_LINKS)
            return rd_fail(RD_ERR_RANGE,
                           "aba_batch: RD_ABA_JOINT_FRAMES takes at most %d links for RD_F32 "
                           "data (n = %d)", RD_ABA_EXTENDED_BIAS_LINKS, m->n);
        if (fp32_scans)
            return vec ? launch_aba_k<T, T, 64, true>(m, B, q, qd, tau, qdd, status, ws, base18, s)
                       : launch_aba_k<T, T, 64, false>(m, B, q, qd, tau, qdd, status, ws, base18, s);
    }
    return vec ? launch_aba_k<T, double, 64, true>(m, B, q, qd, tau, qdd, status, ws, base18, s)
               : launch_aba_k<T, double, 64, false>(m, B, q, qd, tau, qdd, status, ws, base18, s);
}

}  // namespace
}  // namespace rdyn
