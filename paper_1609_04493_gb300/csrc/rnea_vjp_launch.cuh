// rnea_vjp_launch.cuh -- launches of the adjoint kernel; included once per
// element type (vjp_f32.cu, vjp_f64.cu).
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "rdyn_internal.h"
#include "rnea_vjp.cuh"
#include "rnea_vjp_dh.cuh"
#include "rnea_vjp_duo.cuh"
#include "rnea_vjp_pair.cuh"

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

template <typename T, int NMAX, int BLOCK, int MODE, int TRIG>
int launch_vjp_dh_k(const rd_model *m, int B, const void *q, const void *qd, const void *qdd,
                    const void *w, void *gq, void *gqd, void *gqdd, void *ws,
                    const double *base18, cudaStream_t stream)
{
    double b[18];
    rd_convert_base_dh(m, base18, b);
    BaseParams<T> bp;
    for (int k = 0; k < 6; ++k) {
        bp.V0[k] = (T)b[k];
        bp.dV0[k] = (T)b[6 + k];
        bp.Fn[k] = (T)b[12 + k];
    }
    DhParamConsts<T, NMAX> pc;
    for (int k = 0; k < m->n * kDhConsts; ++k) pc.c[k] = (T)m->host_dh64[k];
    for (int k = m->n * kDhConsts; k < NMAX * kDhConsts; ++k) pc.c[k] = T(0);
    const unsigned grid = (unsigned)((B + BLOCK - 1) / BLOCK);
    size_t smem = 0;
    if constexpr (MODE == kVjpStoreShared) {
        static std::atomic<uint64_t> configured{0};
        smem = (size_t)m->n * kVjpStateScalars * BLOCK * sizeof(T);
        const uint64_t bit = 1ull << (m->device & 63);
        if (smem > 48 * 1024 && !(configured.load() & bit)) {
            cudaError_t e = cudaFuncSetAttribute(rnea_vjp_dh_kernel<T, NMAX, BLOCK, MODE, TRIG>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 vjp_max_smem(m->device));
            if (e != cudaSuccess) return rd_cuda_fail(e, "cudaFuncSetAttribute");
            configured.fetch_or(bit);
        }
    }
    rnea_vjp_dh_kernel<T, NMAX, BLOCK, MODE, TRIG><<<grid, BLOCK, smem, stream>>>(
        pc, m->n, B, static_cast<const T *>(q), static_cast<const T *>(qd),
        static_cast<const T *>(qdd), static_cast<const T *>(w), static_cast<T *>(gq),
        static_cast<T *>(gqd), static_cast<T *>(gqdd), static_cast<T *>(ws), bp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return rd_cuda_fail(e, "rnea_vjp common-normal kernel launch");
    return RD_OK;
}

template <int NMAX, int TRIG>
int launch_vjp_pair_k(const rd_model *m, int B, const void *q, const void *qd, const void *qdd,
                      const void *w, void *gq, void *gqd, void *gqdd, const double *base18,
                      cudaStream_t stream)
{
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
    const unsigned grid = (unsigned)((B + 31) / 32);
    rnea_vjp_pair_kernel<NMAX, TRIG><<<grid, 64, 0, stream>>>(
        pc, m->n, B, static_cast<const float *>(q), static_cast<const float *>(qd),
        static_cast<const float *>(qdd), static_cast<const float *>(w), static_cast<float *>(gq),
        static_cast<float *>(gqd), static_cast<float *>(gqdd), bp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return rd_cuda_fail(e, "rnea_vjp two-warp kernel launch");
    return RD_OK;
}

// Two warps per 32 instances with the state in shared memory (rnea_vjp_duo.cuh).
template <int NMAX, int TRIG>
int launch_vjp_duo_k(const rd_model *m, int B, const void *q, const void *qd, const void *qdd,
                     const void *w, void *gq, void *gqd, void *gqdd, const double *base18,
                     cudaStream_t stream)
{
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
    const size_t smem = vjp_duo_smem(m->n);
    if (smem > (size_t)vjp_max_smem(m->device))
        return rd_fail(RD_ERR_ARG, "rnea_vjp: the two-warp shared-state kernel needs %zu bytes of "
                                   "shared memory per block at n = %d", smem, m->n);
    static std::atomic<uint64_t> configured{0};
    const uint64_t bit = 1ull << (m->device & 63);
    if (smem > 48 * 1024 && !(configured.load() & bit)) {
        cudaError_t e = cudaFuncSetAttribute(rnea_vjp_duo_kernel<NMAX, TRIG>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             vjp_max_smem(m->device));
        if (e != cudaSuccess) return rd_cuda_fail(e, "cudaFuncSetAttribute");
        configured.fetch_or(bit);
    }
    const unsigned grid = (unsigned)((B + 31) / 32);
    rnea_vjp_duo_kernel<NMAX, TRIG><<<grid, 64, smem, stream>>>(
        pc, m->n, B, static_cast<const float *>(q), static_cast<const float *>(qd),
        static_cast<const float *>(qdd), static_cast<const float *>(w), static_cast<float *>(gq),
        static_cast<float *>(gqd), static_cast<float *>(gqdd), bp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return rd_cuda_fail(e, "rnea_vjp two-warp shared-state kernel launch");
    return RD_OK;
}

// split: 1 two warps per instance, 2 one thread with the state in shared
// memory, -1 one thread re-deriving it, 0 the library's choice; lanes: lanes
// per instance for the lane-parallel kernel (0: not asked for)
template <typename T, int MODE, int TRIG>
int launch_vjp_dh(const rd_model *m, int B, const void *q, const void *qd, const void *qdd,
                  const void *w, void *gq, void *gqd, void *gqdd, void *ws,
                  const double *base18, int split, int lanes, cudaStream_t s)
{
    if constexpr (sizeof(T) == 4 && MODE == kVjpRecompute) {
        // The library's choice for small batches, from CUDA-graph timings on
        // GB300 (8 rotating input sets; microseconds one thread / shared state /
        // 8 lanes / two warps): n = 16, B = 8192: 7.97 / 7.53 / 17.0 / 8.96;
        // n = 32, B = 1024: 13.6 / 12.7 / 10.4 / 12.5, B = 4096: 13.6 / 12.7 /
        // 11.3 / 13.5, B = 8192: 13.9 / 13.5 / 19.1 / 14.2; n = 64, B = 8192:
        // 26.8 / 45.0 / 57.7 / 25.8; n = 100, B = 8192: 45.8 / - / 201 / 41.9.
        // Two warps with the state in shared memory (rnea_vjp_duo.cuh; B = 1024 /
        // 4096 / 8192): n = 32: 11.6 / 12.1 / 13.4 against 12.6 / 12.7 / 13.5 for
        // the shared state and 10.3 / 11.4 / 18.8 for 8 lanes; n = 64: 20.7 /
        // 21.1 / 40.2 (one block per SM) against 22.3 / 23.1 / 24.6 for two warps.
        if (split == 0 && lanes == 0) {
            const int n = m->n;
            if (n > 16 && n <= 32 && B <= 4096) lanes = 8;
            else if (n <= 32 && B <= 8192) split = 2;
            else if (n > 32 && n <= 64 && B <= 4096) split = 3;
            else if (n > 32 && B <= 8192) split = 1;
        }
        if (lanes > 0)
            return rd_vjp_lane_f32(m, B, q, qd, qdd, w, gq, gqd, gqdd, base18, TRIG == kTrigSfu,
                                   lanes, s);
        if (split == 2) {  // state of every link in shared memory, 32-thread blocks
            if (m->n <= 32)
                return launch_vjp_dh_k<T, 32, 32, kVjpStoreShared, TRIG>(m, B, q, qd, qdd, w, gq, gqd,
                                                                         gqdd, ws, base18, s);
            return launch_vjp_dh_k<T, 64, 32, kVjpStoreShared, TRIG>(m, B, q, qd, qdd, w, gq, gqd,
                                                                     gqdd, ws, base18, s);
        }
        if (split == 1) {
            if (m->n <= 32)
                return launch_vjp_pair_k<32, TRIG>(m, B, q, qd, qdd, w, gq, gqd, gqdd, base18, s);
            return launch_vjp_pair_k<128, TRIG>(m, B, q, qd, qdd, w, gq, gqd, gqdd, base18, s);
        }
        if (split == 3) {
            if (m->n <= 32)
                return launch_vjp_duo_k<32, TRIG>(m, B, q, qd, qdd, w, gq, gqd, gqdd, base18, s);
            return launch_vjp_duo_k<64, TRIG>(m, B, q, qd, qdd, w, gq, gqd, gqdd, base18, s);
        }
    }
    // small batches: 32-thread blocks spread the few warps over more SMs
    const bool small = B <= 152 * 128;
    if (m->n <= 32)
        return small ? launch_vjp_dh_k<T, 32, 32, MODE, TRIG>(m, B, q, qd, qdd, w, gq, gqd, gqdd, ws, base18, s)
                     : launch_vjp_dh_k<T, 32, 64, MODE, TRIG>(m, B, q, qd, qdd, w, gq, gqd, gqdd, ws, base18, s);
    return small ? launch_vjp_dh_k<T, 128, 32, MODE, TRIG>(m, B, q, qd, qdd, w, gq, gqd, gqdd, ws, base18, s)
                 : launch_vjp_dh_k<T, 128, 64, MODE, TRIG>(m, B, q, qd, qdd, w, gq, gqd, gqdd, ws, base18, s);
}

// Common-normal kernel for whole 16-byte chunks (n % 4 == 0, n <= 128, aligned
// rows), unless the joint-frame kernel is asked for; else the joint-frame kernel.
template <typename T, int MODE>
int launch_vjp_any(const rd_model *m, int B, const void *q, const void *qd, const void *qdd,
                   const void *w, void *gq, void *gqd, void *gqdd, void *ws,
                   const double *base18, bool fast, bool joint_frames, int split, int lanes,
                   cudaStream_t s)
{
    const bool dh = !joint_frames && m->n % 4 == 0 && m->n <= 128 && vjp_aligned16(q) &&
                    vjp_aligned16(qd) && vjp_aligned16(qdd) && vjp_aligned16(w) &&
                    vjp_aligned16(gq) && vjp_aligned16(gqd) && vjp_aligned16(gqdd);
    if ((split == 2 || split == 3) && (!dh || MODE != kVjpRecompute))
        return rd_fail(RD_ERR_ARG, "rnea_vjp: RD_VJP_FLAG_SHARED_STATE and "
                                   "RD_VJP_FLAG_TWO_WARPS_SHARED need recompute (or AUTO) mode and "
                                   "16-byte aligned rows");
    if (lanes && (!dh || sizeof(T) != 4 || MODE != kVjpRecompute))
        return rd_fail(RD_ERR_ARG, "rnea_vjp: RD_VJP_FLAG_LANES needs FP32 data in recompute mode, "
                                   "n %% 4 == 0, n <= 128 and 16-byte aligned rows");
    if (dh) {
        if (sizeof(T) == 4 && fast)
            return launch_vjp_dh<T, MODE, kTrigSfu>(m, B, q, qd, qdd, w, gq, gqd, gqdd, ws, base18,
                                                    split, lanes, s);
        return launch_vjp_dh<T, MODE, kTrigPoly>(m, B, q, qd, qdd, w, gq, gqd, gqdd, ws, base18,
                                                 split, lanes, s);
    }
    return launch_vjp_mode<T, MODE>(m, B, q, qd, qdd, w, gq, gqd, gqdd, ws, base18, fast, s);
}

template <typename T>
int vjp_dispatch(const rd_model *m, int B, const void *q, const void *qd, const void *qdd,
                 const void *w, void *gq, void *gqd, void *gqdd, const double *base18, int mode,
                 void *ws, size_t ws_bytes, cudaStream_t s)
{
    const bool fast = (mode & RD_FLAG_FAST_TRIG) != 0;
    const bool joint_frames = (mode & RD_VJP_FLAG_JOINT_FRAMES) != 0;
    if ((mode & RD_VJP_FLAG_TWO_WARPS) && (mode & RD_VJP_FLAG_ONE_THREAD))
        return rd_fail(RD_ERR_ARG, "rnea_vjp: RD_VJP_FLAG_TWO_WARPS and RD_VJP_FLAG_ONE_THREAD both set");
    int split = (mode & RD_VJP_FLAG_TWO_WARPS) ? 1 : (mode & RD_VJP_FLAG_ONE_THREAD) ? -1 : 0;
    if (mode & RD_VJP_FLAG_SHARED_STATE) {
        if (split != 0 || sizeof(T) != 4 || m->n > 64 || m->n % 4 != 0 ||
            (mode & (RD_VJP_FLAG_LANES | RD_VJP_FLAG_LANES4 | RD_VJP_FLAG_JOINT_FRAMES |
                     RD_VJP_FLAG_TWO_WARPS_SHARED)))
            return rd_fail(RD_ERR_ARG, "rnea_vjp: RD_VJP_FLAG_SHARED_STATE needs FP32, n %% 4 == 0, "
                                       "n <= 64 and no other mapping flag");
        split = 2;
    }
    if (mode & RD_VJP_FLAG_TWO_WARPS_SHARED) {
        if (split != 0 || sizeof(T) != 4 || m->n > 64 || m->n % 4 != 0 ||
            (mode & (RD_VJP_FLAG_LANES | RD_VJP_FLAG_LANES4 | RD_VJP_FLAG_JOINT_FRAMES)) ||
            (mode & 0xff) == RD_VJP_STORE)
            return rd_fail(RD_ERR_ARG, "rnea_vjp: RD_VJP_FLAG_TWO_WARPS_SHARED needs FP32, "
                                       "n %% 4 == 0, n <= 64, no workspace mode and no other "
                                       "mapping flag");
        split = 3;
    }
    const int lanes = (mode & RD_VJP_FLAG_LANES4) ? 4 : (mode & RD_VJP_FLAG_LANES) ? 8 : 0;
    if (lanes && (split != 0 || joint_frames))
        return rd_fail(RD_ERR_ARG, "rnea_vjp: RD_VJP_FLAG_LANES excludes RD_VJP_FLAG_TWO_WARPS, "
                                   "RD_VJP_FLAG_ONE_THREAD and RD_VJP_FLAG_JOINT_FRAMES");
    mode &= 0xff;
    const size_t need = (size_t)m->n * kVjpStateScalars * (size_t)B * sizeof(T);
    if (mode == RD_VJP_AUTO) {
        // Measured at n = 32: in FP32 re-deriving the state beats the extra
        // workspace traffic (B = 65536: 51 us vs 78 us); in FP64 the FP64 pipe is
        // the bound and storing saves work (B = 8192: 421 us vs 512 us).
        mode = (sizeof(T) == 8 && ws && ws_bytes >= need) ? RD_VJP_STORE : RD_VJP_RECOMPUTE;
    }
    if (mode == RD_VJP_STORE) {
        if (lanes)
            return rd_fail(RD_ERR_ARG, "rnea_vjp: RD_VJP_FLAG_LANES runs in recompute mode only");
        if (!ws || ws_bytes < need)
            return rd_fail(RD_ERR_ARG, "rnea_vjp: store mode needs a %zu-byte workspace (%zu given)",
                           need, ws_bytes);
        if (!vjp_aligned16(ws)) return rd_fail(RD_ERR_ARG, "rnea_vjp: workspace not 16-byte aligned");
        return launch_vjp_any<T, kVjpStore>(m, B, q, qd, qdd, w, gq, gqd, gqdd, ws, base18, fast,
                                            joint_frames, split == 2 ? 2 : split, 0, s);
    }
    if (mode == RD_VJP_RECOMPUTE)
        return launch_vjp_any<T, kVjpRecompute>(m, B, q, qd, qdd, w, gq, gqd, gqdd, nullptr,
                                                base18, fast, joint_frames, split, lanes, s);
    return rd_fail(RD_ERR_ARG, "rnea_vjp: unknown mode %d", mode);
}

}  // namespace
}  // namespace rdyn
