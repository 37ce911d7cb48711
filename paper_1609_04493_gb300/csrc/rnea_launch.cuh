// rnea_launch.cuh -- variant choice and launches of the one-thread-per-
// instance RNEA kernels; included once per element type (rnea_f32.cu,
// rnea_f64.cu) so the two instantiation sets compile in parallel.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "rdyn_internal.h"
#include "rnea_hybrid.cuh"
#include "rnea_regstate.cuh"
#include "rnea_scan.cuh"
#include "rnea_serial.cuh"

namespace rdyn {
namespace {

template <typename T>
BaseParams<T> make_base(const double b[18])
{
    BaseParams<T> p;
    for (int k = 0; k < 6; ++k) {
        p.V0[k] = (T)b[k];
        p.dV0[k] = (T)b[6 + k];
        p.Fn[k] = (T)b[12 + k];
    }
    return p;
}

int max_smem_optin(int device)
{
    static std::atomic<int> cache[64];
    if (device < 0 || device >= 64) return 48 * 1024;
    int v = cache[device].load();
    if (v == 0) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) !=
            cudaSuccess)
            v = 48 * 1024;
        cache[device].store(v);
    }
    return v;
}

// Raise a kernel's dynamic shared-memory limit once per device.
template <typename K>
cudaError_t allow_smem(K kern, int device, std::atomic<uint64_t> &done)
{
    uint64_t bit = 1ull << (device & 63);
    if (done.load() & bit) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         max_smem_optin(device));
    if (e == cudaSuccess) done.fetch_or(bit);
    return e;
}

template <typename T>
size_t serial_smem(int n, int block, int mode, bool vec)
{
    size_t s = (size_t)n * kLinkConsts * sizeof(T);
    if (vec) s += (size_t)stage_bytes_per_thread<T>() * block;
    s += (size_t)n * state_bytes_per_link<T>(mode) * block;
    return s;
}

template <typename T, int BLOCK, int MODE, bool VEC, bool FAST>
int launch_serial_k(const rd_model *m, int B, const void *q, const void *qd, const void *qdd,
                    void *tau, const double *base18, cudaStream_t stream)
{
    static std::atomic<uint64_t> configured{0};
    const int n = m->n;
    size_t smem = serial_smem<T>(n, BLOCK, MODE, VEC);
    auto kern = rnea_serial_kernel<T, BLOCK, MODE, VEC, FAST>;
    cudaError_t e = allow_smem(kern, m->device, configured);
    if (e != cudaSuccess) return rd_cuda_fail(e, "cudaFuncSetAttribute");
    const T *consts = nullptr;
    if constexpr (sizeof(T) == 4) consts = reinterpret_cast<const T *>(m->d_c32);
    else consts = reinterpret_cast<const T *>(m->d_c64);
    unsigned grid = (unsigned)((B + BLOCK - 1) / BLOCK);
    rd_note_rnea(MODE == kStore ? RD_VARIANT_SERIAL : MODE == kRecompute ? RD_VARIANT_SERIAL_RECOMPUTE
                                                                        : RD_VARIANT_SERIAL_RECOMPUTE_CS,
                 BLOCK, MODE == kStore ? n : 0);
    kern<<<grid, BLOCK, smem, stream>>>(consts, n, B, static_cast<const T *>(q),
                                        static_cast<const T *>(qd), static_cast<const T *>(qdd),
                                        static_cast<T *>(tau), make_base<T>(base18));
    e = cudaGetLastError();
    if (e != cudaSuccess) return rd_cuda_fail(e, "rnea kernel launch");
    return RD_OK;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Vector loads (and the cp.async ring) when rows are whole 16-byte chunks and
// the ring still fits; element loads otherwise.
template <typename T, int BLOCK, int MODE>
int launch_serial(const rd_model *m, int B, const void *q, const void *qd, const void *qdd,
                  void *tau, const double *base18, bool fast, cudaStream_t stream)
{
    const size_t limit = (size_t)max_smem_optin(m->device);
    bool vec = (m->n % 4 == 0) && aligned16(q) && aligned16(qd) && aligned16(qdd) &&
               aligned16(tau) && serial_smem<T>(m->n, BLOCK, MODE, true) <= limit;
    if (!vec && serial_smem<T>(m->n, BLOCK, MODE, false) > limit)
        return rd_fail(RD_ERR_ARG, "rnea_batch: %zu bytes of shared memory needed, %zu available",
                       serial_smem<T>(m->n, BLOCK, MODE, false), limit);
    if constexpr (sizeof(T) == 4) {
        if (fast)
            return vec ? launch_serial_k<T, BLOCK, MODE, true, true>(m, B, q, qd, qdd, tau, base18, stream)
                       : launch_serial_k<T, BLOCK, MODE, false, true>(m, B, q, qd, qdd, tau, base18, stream);
    }
    return vec ? launch_serial_k<T, BLOCK, MODE, true, false>(m, B, q, qd, qdd, tau, base18, stream)
               : launch_serial_k<T, BLOCK, MODE, false, false>(m, B, q, qd, qdd, tau, base18, stream);
}

template <typename T, int MODE>
int launch_mode(const rd_model *m, int block, int B, const void *q, const void *qd,
                const void *qdd, void *tau, const double *base18, bool fast, cudaStream_t s)
{
    switch (block) {
    case 32: return launch_serial<T, 32, MODE>(m, B, q, qd, qdd, tau, base18, fast, s);
    case 64: return launch_serial<T, 64, MODE>(m, B, q, qd, qdd, tau, base18, fast, s);
    case 128: return launch_serial<T, 128, MODE>(m, B, q, qd, qdd, tau, base18, fast, s);
    default: return rd_fail(RD_ERR_ARG, "rnea_batch: block size %d not built (32, 64, 128)", block);
    }
}

template <typename T, int BLOCK, bool VEC, bool FAST>
int launch_hybrid_k(const rd_model *m, int K, int B, const void *q, const void *qd,
                    const void *qdd, void *tau, const double *base18, cudaStream_t stream)
{
    static std::atomic<uint64_t> configured{0};
    const int n = m->n;
    const size_t smem = hybrid_smem_bytes<T>(n, K, BLOCK, VEC);
    auto kern = rnea_hybrid_kernel<T, BLOCK, VEC, FAST>;
    cudaError_t e = allow_smem(kern, m->device, configured);
    if (e != cudaSuccess) return rd_cuda_fail(e, "cudaFuncSetAttribute");
    const T *consts = nullptr;
    if constexpr (sizeof(T) == 4) consts = reinterpret_cast<const T *>(m->d_c32);
    else consts = reinterpret_cast<const T *>(m->d_c64);
    const unsigned grid = (unsigned)((B + BLOCK - 1) / BLOCK);
    rd_note_rnea(RD_VARIANT_SERIAL_HYBRID, BLOCK, K);
    kern<<<grid, BLOCK, smem, stream>>>(consts, n, K, B, static_cast<const T *>(q),
                                        static_cast<const T *>(qd), static_cast<const T *>(qdd),
                                        static_cast<T *>(tau), make_base<T>(base18));
    e = cudaGetLastError();
    if (e != cudaSuccess) return rd_cuda_fail(e, "rnea hybrid kernel launch");
    return RD_OK;
}

template <typename T, int BLOCK>
int launch_hybrid_b(const rd_model *m, int K, int B, const void *q, const void *qd,
                    const void *qdd, void *tau, const double *base18, bool fast, cudaStream_t s)
{
    const size_t limit = (size_t)max_smem_optin(m->device);
    const bool vec = (m->n % 4 == 0) && aligned16(q) && aligned16(qd) && aligned16(qdd) &&
                     aligned16(tau) && hybrid_smem_bytes<T>(m->n, K, BLOCK, true) <= limit;
    if (!vec && hybrid_smem_bytes<T>(m->n, K, BLOCK, false) > limit)
        return rd_fail(RD_ERR_ARG, "rnea_batch: state of %d links needs %zu bytes of shared "
                                   "memory, %zu available", K,
                       hybrid_smem_bytes<T>(m->n, K, BLOCK, false), limit);
    if constexpr (sizeof(T) == 4) {
        if (fast)
            return vec ? launch_hybrid_k<T, BLOCK, true, true>(m, K, B, q, qd, qdd, tau, base18, s)
                       : launch_hybrid_k<T, BLOCK, false, true>(m, K, B, q, qd, qdd, tau, base18, s);
    }
    return vec ? launch_hybrid_k<T, BLOCK, true, false>(m, K, B, q, qd, qdd, tau, base18, s)
               : launch_hybrid_k<T, BLOCK, false, false>(m, K, B, q, qd, qdd, tau, base18, s);
}

// Stored-state prefix of K links (rounded up to whole chunks and capped at the
// chain); the rest of the chain is recomputed in the backward sweep.
template <typename T>
int launch_hybrid(const rd_model *m, int block, int K, int B, const void *q, const void *qd,
                  const void *qdd, void *tau, const double *base18, bool fast, cudaStream_t s)
{
    const int cap = 4 * ((m->n + 3) / 4);
    K = K > cap ? cap : 4 * ((K + 3) / 4);
    switch (block) {
    case 32: return launch_hybrid_b<T, 32>(m, K, B, q, qd, qdd, tau, base18, fast, s);
    case 64: return launch_hybrid_b<T, 64>(m, K, B, q, qd, qdd, tau, base18, fast, s);
    case 128: return launch_hybrid_b<T, 128>(m, K, B, q, qd, qdd, tau, base18, fast, s);
    default: return rd_fail(RD_ERR_ARG, "rnea_batch: block size %d not built (32, 64, 128)", block);
    }
}

template <typename T, int L, int K, bool FAST>
int launch_scan_k(const rd_model *m, int B, const void *q, const void *qd, const void *qdd,
                  void *tau, const double *base18, cudaStream_t stream)
{
    static std::atomic<uint64_t> configured{0};
    const int n = m->n;
    const size_t smem = (size_t)n * kLinkConsts * sizeof(T);
    auto kern = rnea_scan_kernel<T, L, K, FAST>;
    cudaError_t e = allow_smem(kern, m->device, configured);
    if (e != cudaSuccess) return rd_cuda_fail(e, "cudaFuncSetAttribute");
    const T *consts = nullptr;
    if constexpr (sizeof(T) == 4) consts = reinterpret_cast<const T *>(m->d_c32);
    else consts = reinterpret_cast<const T *>(m->d_c64);
    const long long threads = (long long)B * L;
    const unsigned grid = (unsigned)((threads + 127) / 128);
    rd_note_rnea(RD_VARIANT_SCAN(L), 128, 0);
    kern<<<grid, 128, smem, stream>>>(consts, n, B, static_cast<const T *>(q),
                                      static_cast<const T *>(qd), static_cast<const T *>(qdd),
                                      static_cast<T *>(tau), make_base<T>(base18));
    e = cudaGetLastError();
    if (e != cudaSuccess) return rd_cuda_fail(e, "rnea scan kernel launch");
    return RD_OK;
}

template <typename T, int L, bool FAST>
int launch_scan_l(const rd_model *m, int B, const void *q, const void *qd, const void *qdd,
                  void *tau, const double *base18, cudaStream_t s)
{
    const int k = (m->n + L - 1) / L;
    if (k <= 1) return launch_scan_k<T, L, 1, FAST>(m, B, q, qd, qdd, tau, base18, s);
    if (k <= 2) return launch_scan_k<T, L, 2, FAST>(m, B, q, qd, qdd, tau, base18, s);
    if (k <= 4) return launch_scan_k<T, L, 4, FAST>(m, B, q, qd, qdd, tau, base18, s);
    if (k <= 8) return launch_scan_k<T, L, 8, FAST>(m, B, q, qd, qdd, tau, base18, s);
    return rd_fail(RD_ERR_ARG, "rnea_batch: %d lanes cannot hold %d links (at most 8 per lane)",
                   L, m->n);
}

template <typename T, bool FAST>
int launch_scan(const rd_model *m, int lanes, int B, const void *q, const void *qd,
                const void *qdd, void *tau, const double *base18, cudaStream_t s)
{
    switch (lanes) {
    case 2: return launch_scan_l<T, 2, FAST>(m, B, q, qd, qdd, tau, base18, s);
    case 4: return launch_scan_l<T, 4, FAST>(m, B, q, qd, qdd, tau, base18, s);
    case 8: return launch_scan_l<T, 8, FAST>(m, B, q, qd, qdd, tau, base18, s);
    case 16: return launch_scan_l<T, 16, FAST>(m, B, q, qd, qdd, tau, base18, s);
    case 32: return launch_scan_l<T, 32, FAST>(m, B, q, qd, qdd, tau, base18, s);
    default: return rd_fail(RD_ERR_ARG, "rnea_batch: scan lanes %d not in {2,4,8,16,32}", lanes);
    }
}

template <typename T, int BLOCK, int RL>
int launch_regstate_k(const rd_model *m, int B, const void *q, const void *qd, const void *qdd,
                      void *tau, const double *base18, cudaStream_t stream)
{
    static std::atomic<uint64_t> configured{0};
    const int n = m->n;
    const size_t smem = (size_t)n * kLinkConsts * sizeof(T) +
                        (size_t)stage_bytes_per_thread<T>() * BLOCK +
                        (size_t)(n > RL ? n - RL : 0) * state_bytes_per_link<T>(kStore) * BLOCK;
    if (smem > (size_t)max_smem_optin(m->device))  // long chain: keep no per-link state
        return launch_serial<T, 64, kRecompute>(m, B, q, qd, qdd, tau, base18, false, stream);
    auto kern = rnea_regstate_kernel<T, BLOCK, RL>;
    cudaError_t e = allow_smem(kern, m->device, configured);
    if (e != cudaSuccess) return rd_cuda_fail(e, "cudaFuncSetAttribute");
    const T *consts = nullptr;
    if constexpr (sizeof(T) == 4) consts = reinterpret_cast<const T *>(m->d_c32);
    else consts = reinterpret_cast<const T *>(m->d_c64);
    const unsigned grid = (unsigned)((B + BLOCK - 1) / BLOCK);
    rd_note_rnea(RD_VARIANT_SERIAL_REGSTATE, BLOCK, n);
    kern<<<grid, BLOCK, smem, stream>>>(consts, n, B, static_cast<const T *>(q),
                                        static_cast<const T *>(qd), static_cast<const T *>(qdd),
                                        static_cast<T *>(tau), make_base<T>(base18));
    e = cudaGetLastError();
    if (e != cudaSuccess) return rd_cuda_fail(e, "rnea regstate kernel launch");
    return RD_OK;
}

// Register-plus-shared-memory state; needs whole 16-byte chunks (else the
// shared-memory-state kernel runs instead).
template <typename T>
int launch_regstate(const rd_model *m, int block, int reglinks, int B, const void *q,
                    const void *qd, const void *qdd, void *tau, const double *base18, bool fast,
                    cudaStream_t s)
{
    const bool vec = (m->n % 4 == 0) && aligned16(q) && aligned16(qd) && aligned16(qdd) &&
                     aligned16(tau);
    if (!vec || fast)
        return launch_mode<T, kStore>(m, block ? block : 32, B, q, qd, qdd, tau, base18, fast, s);
    if (!block) block = 32;
    if (!reglinks) reglinks = 16;
#define RD_REGSTATE_CASE(BL, RLK)                                                   \
    if (block == BL && reglinks == RLK)                                             \
        return launch_regstate_k<T, BL, RLK>(m, B, q, qd, qdd, tau, base18, s);
    RD_REGSTATE_CASE(32, 8)
    RD_REGSTATE_CASE(32, 16)
    RD_REGSTATE_CASE(64, 8)
    RD_REGSTATE_CASE(64, 16)
#undef RD_REGSTATE_CASE
    return rd_fail(RD_ERR_ARG, "rnea_batch: register-state kernel not built for %d threads, "
                               "%d register links", block, reglinks);
}

template <typename T>
int dispatch(const rd_model *m, int B, const void *q, const void *qd, const void *qdd, void *tau,
             const double *base18, int variant, cudaStream_t s)
{
    const int n = m->n;
    const size_t limit = (size_t)max_smem_optin(m->device);
    const bool fast = (variant & RD_FLAG_FAST_TRIG) != 0;
    int block = (variant >> 16) & 0xf;
    if (block) block = 1 << block;
    const int reglinks = 4 * ((variant >> 20) & 0xff);  // RD_TUNE_REGLINKS / _STORED_LINKS
    const int regstate = 4 * ((variant >> 28) & 0x7);   // RD_TUNE_REG_STATE_LINKS
    const int stages = (variant & RD_TUNE_TWO_STAGE_RING) ? 2 : kStages;
    variant &= 0xfff;
    const bool dhp_rows = sizeof(T) == 4 && n % 4 == 0 && n <= 128 && aligned16(q) &&
                          aligned16(qd) && aligned16(qdd) && aligned16(tau);
    // the common-normal kernel of the next branch overtakes the scans sooner
    // (n = 32: 7.5 us against 9.3 at B = 4096; 6.9 against 5.0 at B = 1024)
    if (variant == RD_VARIANT_AUTO && B <= (dhp_rows ? 2048 : 152 * 32) && n <= 128) {
        // Fewer instances than one warp per SM: the serial recursion leaves the
        // GPU idle, and splitting each chain over lanes (the scans of Sec. III)
        // cuts latency. Measured: n = 7, B = 1024 FP64 30 us with 8 lanes vs 43
        // serial; n = 32, B = 1024 FP32 5.1 us with 16 lanes vs 8.4 serial;
        // from B = 8192 on the serial form wins.
        int lanes = 2;
        while (lanes < 16 && lanes < n) lanes <<= 1;
        while (lanes * 8 < n) lanes <<= 1;
        if constexpr (sizeof(T) == 4) {
            if (fast) return launch_scan<T, true>(m, lanes, B, q, qd, qdd, tau, base18, s);
        }
        return launch_scan<T, false>(m, lanes, B, q, qd, qdd, tau, base18, s);
    }
    if (variant == RD_VARIANT_AUTO && dhp_rows) {
        // FP32, whole 16-byte chunks: common-normal frames, constants as a kernel
        // parameter, full state for the library's K (about 22% below the
        // joint-frame kernels at n = 16..100, B = 65536; see rnea_dh_launch.cuh)
        return rd_rnea_dh_f32(m, B, q, qd, qdd, tau, base18, 1, block, fast,
                              reglinks ? reglinks : -1, 0, regstate, stages, s);
    }
    if (variant == RD_VARIANT_AUTO) {
        // Sweep on GB300 at B = 65536 (modes x block sizes x stored links):
        // per-link state in shared memory wins while it is small (FP32 n <= 32,
        // FP64 n <= 16); FP64 up to n = 32 keeps part of it in registers; up to
        // n = 64 the first links keep their state and the rest are re-derived;
        // longer chains re-derive the motion of every link in the backward sweep.
        if (n <= (sizeof(T) == 4 ? 32 : 16) && serial_smem<T>(n, 32, kStore, true) <= limit / 4) {
            variant = RD_VARIANT_SERIAL;
            // FP64 n = 16: 393 us with 32 threads vs 408 with 64
            if (!block) block = (sizeof(T) == 8 || n > 16) ? 32 : 64;
        } else if (n <= 64 && (sizeof(T) == 4 || n > 32)) {
            // 32 < n <= 64: state for the first links only. FP64 n = 48: 1492 us
            // with 12 stored links vs 1719 stateless; n = 64: 2068 vs 2143 with 8;
            // FP32 n = 48 / 64: 45.8 / 60.6 us with 8 vs 47.3 / 61.8.
            const int K = reglinks ? reglinks : (sizeof(T) == 8 && n <= 48 ? 12 : 8);
            return launch_hybrid<T>(m, block ? block : 64, K, B, q, qd, qdd, tau, base18, fast, s);
        } else if (sizeof(T) == 8 && n <= 32) {
            // FP64, 16 < n <= 32: the first 16 links' state in registers
            // (812 us vs 934 us for cos/sin-only state at n = 32)
            if (n % 4 == 0) {
                return launch_regstate<T>(m, block ? block : 32, reglinks ? reglinks : 16, B, q,
                                          qd, qdd, tau, base18, fast, s);
            }
            variant = RD_VARIANT_SERIAL_RECOMPUTE_CS;
            if (!block) block = 32;
        } else {
            variant = RD_VARIANT_SERIAL_RECOMPUTE;
            if (!block) block = sizeof(T) == 4 ? 64 : 32;
        }
    }
    if (variant == RD_VARIANT_SERIAL) {
        if (!block) {
            block = serial_smem<T>(n, 64, kStore, false) <= limit / 2 ? 64 : 32;
            if (serial_smem<T>(n, 32, kStore, false) > limit)
                return rd_fail(RD_ERR_ARG, "rnea_batch: per-link state of %d links does not fit in "
                                           "shared memory; use RD_VARIANT_SERIAL_RECOMPUTE", n);
        }
        return launch_mode<T, kStore>(m, block, B, q, qd, qdd, tau, base18, fast, s);
    }
    if (variant == RD_VARIANT_SERIAL_REGSTATE)
        return launch_regstate<T>(m, block, reglinks, B, q, qd, qdd, tau, base18, fast, s);
    if (variant == RD_VARIANT_SERIAL_DH || variant == RD_VARIANT_SERIAL_DH_RECOMPUTE ||
        variant == RD_VARIANT_SERIAL_DH_TMEM) {
        const int stored = variant != RD_VARIANT_SERIAL_DH_RECOMPUTE;
        const int tmem = variant == RD_VARIANT_SERIAL_DH_TMEM;
        const int kfull = reglinks ? reglinks : -1;
        if constexpr (sizeof(T) == 4)
            return rd_rnea_dh_f32(m, B, q, qd, qdd, tau, base18, stored, block, fast, kfull, tmem,
                                  regstate, stages, s);
        else
            return rd_rnea_dh_f64(m, B, q, qd, qdd, tau, base18, stored, block, fast, kfull, tmem,
                                  regstate, stages, s);
    }
    if (variant == RD_VARIANT_SERIAL_DF) {
        if constexpr (sizeof(T) == 8)
            return rd_rnea_df_f64(m, B, q, qd, qdd, tau, base18, block, s);
        else
            return rd_fail(RD_ERR_DTYPE, "rnea_batch: RD_VARIANT_SERIAL_DF takes RD_F64 data");
    }
    if (variant == RD_VARIANT_SERIAL_HYBRID) {
        if (!block) block = 32;
        const int K = reglinks ? reglinks : 16;
        return launch_hybrid<T>(m, block, K, B, q, qd, qdd, tau, base18, fast, s);
    }
    if (!block) block = 64;
    if (variant == RD_VARIANT_SERIAL_RECOMPUTE)
        return launch_mode<T, kRecompute>(m, block, B, q, qd, qdd, tau, base18, fast, s);
    if (variant == RD_VARIANT_SERIAL_RECOMPUTE_CS)
        return launch_mode<T, kRecomputeCS>(m, block, B, q, qd, qdd, tau, base18, fast, s);
    if ((variant & 0xf00) == 0x100) {
        const int lanes = variant & 0xff;
        if constexpr (sizeof(T) == 4) {
            if (fast) return launch_scan<T, true>(m, lanes, B, q, qd, qdd, tau, base18, s);
        }
        return launch_scan<T, false>(m, lanes, B, q, qd, qdd, tau, base18, s);
    }
    return rd_fail(RD_ERR_ARG, "rnea_batch: unknown variant 0x%x", variant);
}

}  // namespace
}  // namespace rdyn
