// rnea_dh_launch.cuh -- launches of the common-normal-frame RNEA kernels
// (rnea_dh.cuh); included once per element type (rnea_dh_f32.cu,
// rnea_dh_f64.cu).
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "rdyn_internal.h"
#include "rnea_dht.cuh"
#include "rnea_dhp.cuh"

namespace rdyn {
namespace {

int dh_smem_optin(int device)
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

template <typename T>
size_t dh_smem(int n, int block, int mode, bool vec)
{
    size_t s = (size_t)n * kDhConsts * sizeof(T);
    if (vec) s += (size_t)stage_bytes_per_thread<T>() * block;
    s += (size_t)n * state_bytes_per_link<T>(mode) * block;
    return s;
}

template <typename T, int BLOCK, int MODE, bool VEC, bool FAST>
int launch_dh_k(const rd_model *m, int B, const void *q, const void *qd, const void *qdd,
                void *tau, const BaseParams<T> &base, size_t smem, cudaStream_t stream)
{
    static std::atomic<uint64_t> configured{0};
    auto kern = rnea_dh_kernel<T, BLOCK, MODE, VEC, FAST>;
    const uint64_t bit = 1ull << (m->device & 63);
    if (!(configured.load() & bit)) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             dh_smem_optin(m->device));
        if (e != cudaSuccess) return rd_cuda_fail(e, "cudaFuncSetAttribute");
        configured.fetch_or(bit);
    }
    const T *consts = nullptr;
    if constexpr (sizeof(T) == 4) consts = m->d_dh32;
    else consts = m->d_dh64;
    const unsigned grid = (unsigned)((B + BLOCK - 1) / BLOCK);
    rd_note_rnea(MODE == kStore ? RD_VARIANT_SERIAL_DH : RD_VARIANT_SERIAL_DH_RECOMPUTE, BLOCK,
                 MODE == kStore ? m->n : 0);
    kern<<<grid, BLOCK, smem, stream>>>(consts, m->n, B, static_cast<const T *>(q),
                                        static_cast<const T *>(qd), static_cast<const T *>(qdd),
                                        static_cast<T *>(tau), base);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return rd_cuda_fail(e, "rnea common-normal kernel launch");
    return RD_OK;
}

inline bool dh_aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

template <typename T, int BLOCK, int MODE>
int launch_dh_b(const rd_model *m, int B, const void *q, const void *qd, const void *qdd,
                void *tau, const BaseParams<T> &base, bool fast, cudaStream_t s)
{
    const size_t limit = (size_t)dh_smem_optin(m->device);
    const bool vec = (m->n % 4 == 0) && dh_aligned16(q) && dh_aligned16(qd) &&
                     dh_aligned16(qdd) && dh_aligned16(tau) &&
                     dh_smem<T>(m->n, BLOCK, MODE, true) <= limit;
    const size_t smem = dh_smem<T>(m->n, BLOCK, MODE, vec);
    if (smem > limit)
        return rd_fail(RD_ERR_ARG, "rnea_batch: %zu bytes of shared memory needed, %zu available",
                       smem, limit);
    if constexpr (sizeof(T) == 4) {
        if (fast)
            return vec ? launch_dh_k<T, BLOCK, MODE, true, true>(m, B, q, qd, qdd, tau, base, smem, s)
                       : launch_dh_k<T, BLOCK, MODE, false, true>(m, B, q, qd, qdd, tau, base, smem, s);
    }
    return vec ? launch_dh_k<T, BLOCK, MODE, true, false>(m, B, q, qd, qdd, tau, base, smem, s)
               : launch_dh_k<T, BLOCK, MODE, false, false>(m, B, q, qd, qdd, tau, base, smem, s);
}

template <typename T, int MODE>
int launch_dh_mode(const rd_model *m, int block, int B, const void *q, const void *qd,
                   const void *qdd, void *tau, const BaseParams<T> &base, bool fast,
                   cudaStream_t s)
{
    switch (block) {
    case 32: return launch_dh_b<T, 32, MODE>(m, B, q, qd, qdd, tau, base, fast, s);
    case 64: return launch_dh_b<T, 64, MODE>(m, B, q, qd, qdd, tau, base, fast, s);
    case 128: return launch_dh_b<T, 128, MODE>(m, B, q, qd, qdd, tau, base, fast, s);
    default: return rd_fail(RD_ERR_ARG, "rnea_batch: block size %d not built (32, 64, 128)", block);
    }
}

template <typename T, int NMAX, int BLOCK, int TRIG, int RL = 0, int STG = kStages>
int launch_dhp_k(const rd_model *m, int K, int B, const void *q, const void *qd, const void *qdd,
                 void *tau, const BaseParams<T> &base, size_t smem, cudaStream_t stream)
{
    static std::atomic<uint64_t> configured{0};
    auto kern = rnea_dhp_kernel<T, NMAX, BLOCK, TRIG, RL, STG>;
    const uint64_t bit = 1ull << (m->device & 63);
    if (!(configured.load() & bit)) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             dh_smem_optin(m->device));
        if (e != cudaSuccess) return rd_cuda_fail(e, "cudaFuncSetAttribute");
        configured.fetch_or(bit);
    }
    DhParamConsts<T, NMAX> pc;
    for (int k = 0; k < m->n * kDhConsts; ++k) pc.c[k] = (T)m->host_dh64[k];
    for (int k = m->n * kDhConsts; k < NMAX * kDhConsts; ++k) pc.c[k] = T(0);
    const unsigned grid = (unsigned)((B + BLOCK - 1) / BLOCK);
    rd_note_rnea(RD_RNEA_KERNEL_DH_PARAM, BLOCK, K, RL, STG);
    kern<<<grid, BLOCK, smem, stream>>>(pc, m->n, K, B, static_cast<const T *>(q),
                                        static_cast<const T *>(qd), static_cast<const T *>(qdd),
                                        static_cast<T *>(tau), base);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return rd_cuda_fail(e, "rnea common-normal kernel launch");
    return RD_OK;
}

template <typename T, int NMAX, int TRIG>
int launch_dhp_b(const rd_model *m, int block, int K, int B, const void *q, const void *qd,
                 const void *qdd, void *tau, const BaseParams<T> &base, size_t smem,
                 cudaStream_t s)
{
    switch (block) {
    case 32: return launch_dhp_k<T, NMAX, 32, TRIG>(m, K, B, q, qd, qdd, tau, base, smem, s);
    case 64: return launch_dhp_k<T, NMAX, 64, TRIG>(m, K, B, q, qd, qdd, tau, base, smem, s);
    case 128: return launch_dhp_k<T, NMAX, 128, TRIG>(m, K, B, q, qd, qdd, tau, base, smem, s);
    default: return rd_fail(RD_ERR_ARG, "rnea_batch: block size %d not built (32, 64, 128)", block);
    }
}

int dh_device_attr(int device, cudaDeviceAttr attr, int fallback)
{
    int v = 0;
    if (cudaDeviceGetAttribute(&v, attr, device) != cudaSuccess || v <= 0) return fallback;
    return v;
}

// Default K for the parameter-constant kernel (32-thread blocks). On GB300 at
// B = 65536 the fastest K at every length was the largest that still leaves 7
// blocks per SM, so the batch runs in at most two waves (n = 16: K = 16, 10.8 us;
// n = 32: K = 24, 23.2 us; n = 64: K = 12, 46.7 us; n = 100: K = 0, 71.2 us,
// against 14.8 / 29.7 / 60.2 / 92.0 us for the joint-frame kernels). When the
// whole batch fits in one wave with more state, the larger K is taken.
template <typename T>
int dhp_default_k(const rd_model *m, int B)
{
    static std::atomic<int> smem_sm[64], sms[64];
    const int d = m->device & 63;
    if (smem_sm[d].load() == 0) {
        smem_sm[d].store(dh_device_attr(m->device, cudaDevAttrMaxSharedMemoryPerMultiprocessor, 100 * 1024));
        sms[d].store(dh_device_attr(m->device, cudaDevAttrMultiProcessorCount, 1));
    }
    const int n = m->n;
    auto blocks_per_sm = [&](int K) {
        const size_t per_block = dhp_smem_per_thread<T>(n, K) * 32 + 1024;  // + the block's reserve
        const long long b = (long long)smem_sm[d].load() / (long long)per_block;
        return b > 32 ? 32 : (int)b;
    };
    const long long blocks = (B + 31) / 32;
    int best = 0;
    for (int K = 0; K <= n; K += 4) {
        const int per_sm = blocks_per_sm(K);
        if (per_sm >= 7 || (long long)per_sm * sms[d].load() >= blocks) best = K;
    }
    return best;
}

// Parameter-constant kernel with full state for the first K links (K a multiple
// of 4, at most n; K < 0: library default); needs n % 4 == 0, n <= 128 and
// 16-byte aligned rows.
template <typename T>
bool dhp_eligible(const rd_model *m, const void *q, const void *qd, const void *qdd,
                  const void *tau)
{
    return m->n % 4 == 0 && m->n <= 128 && dh_aligned16(q) && dh_aligned16(qd) &&
           dh_aligned16(qdd) && dh_aligned16(tau);
}

// Library default for FP32, n <= 32, 32-thread blocks: every link stored (K =
// n), the first RL of them in registers, the joint values staged through a
// ring of `stages` chunks. Measured on GB300 (µs at B = 65536; the previous
// default of 24 or n links in shared memory / the choice): n = 8: 5.68 / 5.17
// (RL = 8, all in registers); 12: 7.43 / 7.02 (8, two-chunk ring); 16: 10.30 /
// 9.18 (8, two); 20: 13.50 / 11.63 (8, two); 24: 15.76 / 14.47 (8, three); 28:
// 18.54 / 17.39 (8, two); 32: 21.78 / 20.25 (8, three; two: 20.96). Where RL =
// 4 with the two-chunk ring holds the whole batch in half a wave it leads (n =
// 16, B = 16384: 4.09 against 4.50 with 8; n = 32, B = 16384: 6.75 against
// 7.14); near a full wave 8 does (n = 16, B = 65536: 9.18 against 9.39). 12 and
// 16 register links never led: more blocks per SM, longer unrolled code.
template <int TRIG>
void dhp_default_kr(const rd_model *m, int B, int &K, int &RL, int &stages)
{
    const int n = m->n;
    K = n;
    stages = kStages;
    if (n <= 8) {
        RL = n;
        return;
    }
    // resident blocks per SM of the RL = 4, two-chunk kernel at this n, queried
    // once per device, length and sin/cos variant (stored + 1; 0 = not yet known)
    static std::atomic<int> known[64][33][2];
    std::atomic<int> &slot = known[m->device & 63][n][TRIG == kTrigSfu ? 1 : 0];
    int per_sm = slot.load() - 1;
    if (per_sm < 0) {
        per_sm = 0;
        const size_t smem = dhp_smem_per_thread<float>(n, n, 4, 2) * 32;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, rnea_dhp_kernel<float, 32, 32, TRIG, 4, 2>, 32, smem);
        slot.store(per_sm + 1);
    }
    const long long sms = dh_device_attr(m->device, cudaDevAttrMultiProcessorCount, 1);
    if ((long long)per_sm * sms >= 2 * ((long long)(B + 31) / 32)) {
        RL = 4;
        stages = 2;
        return;
    }
    RL = 8;
    stages = (n == 24 || n == 32) ? kStages : 2;
}

// FP32, n <= 32, 32-thread blocks: the first RL of the K stored links keep
// their state in registers (RL = 4, 8, 12 or 16; K >= RL)
template <int TRIG>
int launch_dhp_reg(const rd_model *m, int RL, int stages, int K, int B, const void *q,
                   const void *qd, const void *qdd, void *tau, const BaseParams<float> &base,
                   size_t smem, cudaStream_t s)
{
    if (stages == 2) {
        switch (RL) {
        case 0: return launch_dhp_k<float, 32, 32, TRIG, 0, 2>(m, K, B, q, qd, qdd, tau, base, smem, s);
        case 4: return launch_dhp_k<float, 32, 32, TRIG, 4, 2>(m, K, B, q, qd, qdd, tau, base, smem, s);
        case 8: return launch_dhp_k<float, 32, 32, TRIG, 8, 2>(m, K, B, q, qd, qdd, tau, base, smem, s);
        default: break;
        }
        return rd_fail(RD_ERR_ARG, "rnea_batch: the two-stage ring is built for 0, 4 or 8 register "
                                   "links (%d asked)", RL);
    }
    switch (RL) {
    case 4: return launch_dhp_k<float, 32, 32, TRIG, 4>(m, K, B, q, qd, qdd, tau, base, smem, s);
    case 8: return launch_dhp_k<float, 32, 32, TRIG, 8>(m, K, B, q, qd, qdd, tau, base, smem, s);
    case 12: return launch_dhp_k<float, 32, 32, TRIG, 12>(m, K, B, q, qd, qdd, tau, base, smem, s);
    case 16: return launch_dhp_k<float, 32, 32, TRIG, 16>(m, K, B, q, qd, qdd, tau, base, smem, s);
    default: return rd_fail(RD_ERR_ARG, "rnea_batch: %d register links not built (4, 8, 12, 16)", RL);
    }
}

template <typename T>
int launch_dhp(const rd_model *m, int block, int K, int B, const void *q, const void *qd,
               const void *qdd, void *tau, const BaseParams<T> &base, bool fast, cudaStream_t s,
               int RL = 0, int stages = kStages)
{
    const int n = m->n;
    if constexpr (sizeof(T) == 4) {
        if (K < 0 && RL == 0 && stages == kStages && block == 32 && n <= 32) {
            if (fast) dhp_default_kr<kTrigSfu>(m, B, K, RL, stages);
            else dhp_default_kr<kTrigPoly>(m, B, K, RL, stages);
        }
    }
    if (K < 0) K = dhp_default_k<T>(m, B);
    K = K > n ? n : 4 * (K / 4);
    if (RL || stages != kStages) {
        if (sizeof(T) != 4 || n > 32 || block != 32 || RL % 4 || RL < 0 || RL > 16 || RL > K)
            return rd_fail(RD_ERR_ARG, "rnea_batch: register state and the two-stage ring need "
                                       "FP32, n <= 32, 32-thread blocks and 4, 8, 12 or 16 "
                                       "register links, at most the %d stored", K);
    }
    const size_t smem = dhp_smem_per_thread<T>(n, K, RL, stages) * (size_t)block;
    if (smem > (size_t)dh_smem_optin(m->device))
        return rd_fail(RD_ERR_ARG, "rnea_batch: state of %d links needs %zu bytes of shared "
                                   "memory, %d available", K, smem, dh_smem_optin(m->device));
    if constexpr (sizeof(T) == 4) {
        if (RL || stages != kStages)
            return fast ? launch_dhp_reg<kTrigSfu>(m, RL, stages, K, B, q, qd, qdd, tau, base, smem, s)
                        : launch_dhp_reg<kTrigPoly>(m, RL, stages, K, B, q, qd, qdd, tau, base, smem, s);
    }
    const bool sfu = sizeof(T) == 4 && fast;
    if (n <= 32)
        return sfu ? launch_dhp_b<T, 32, kTrigSfu>(m, block, K, B, q, qd, qdd, tau, base, smem, s)
                   : launch_dhp_b<T, 32, kTrigPoly>(m, block, K, B, q, qd, qdd, tau, base, smem, s);
    return sfu ? launch_dhp_b<T, 128, kTrigSfu>(m, block, K, B, q, qd, qdd, tau, base, smem, s)
               : launch_dhp_b<T, 128, kTrigPoly>(m, block, K, B, q, qd, qdd, tau, base, smem, s);
}

// ---- TMEM-state kernel (FP32, n <= 32, n % 4 == 0, aligned rows)

template <int TRIG, int STAGES>
int launch_dht_k(const rd_model *m, int K, int TL, int B, const void *q, const void *qd,
                 const void *qdd, void *tau, const BaseParams<float> &base, size_t smem,
                 cudaStream_t stream)
{
    static std::atomic<uint64_t> configured{0};
    auto kern = rnea_dht_kernel<32, TRIG, STAGES>;
    const uint64_t bit = 1ull << (m->device & 63);
    if (!(configured.load() & bit)) {
        // the opt-in limit covers static and dynamic shared memory together
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, kern);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     dh_smem_optin(m->device) - (int)fa.sharedSizeBytes);
        if (e != cudaSuccess) return rd_cuda_fail(e, "cudaFuncSetAttribute");
        configured.fetch_or(bit);
    }
    DhParamConsts<float, 32> pc;
    for (int k = 0; k < m->n * kDhConsts; ++k) pc.c[k] = (float)m->host_dh64[k];
    for (int k = m->n * kDhConsts; k < 32 * kDhConsts; ++k) pc.c[k] = 0.0f;
    // four blocks per SM, each with an equal share of the batch in rounds of
    // at most 128 instances
    static std::atomic<int> sms[64];
    const int d = m->device & 63;
    if (sms[d].load() == 0) sms[d].store(dh_device_attr(m->device, cudaDevAttrMultiProcessorCount, 1));
    const long long max_grid = 4LL * sms[d].load(), min_grid = ((long long)B + 31) / 32;
    const long long grid = max_grid < min_grid ? max_grid : min_grid;
    const long long per_block = ((long long)B + grid - 1) / grid;
    const long long rounds = (per_block + kDhtThreads - 1) / kDhtThreads;
    const long long per_round = (per_block + rounds - 1) / rounds;
    rd_note_rnea(RD_RNEA_KERNEL_DH_TMEM, kDhtThreads, K);
    kern<<<(unsigned)grid, kDhtThreads, smem, stream>>>(pc, m->n, K, TL, B, (int)per_block,
                                              (int)per_round, static_cast<const float *>(q),
                                              static_cast<const float *>(qd),
                                              static_cast<const float *>(qdd),
                                              static_cast<float *>(tau), base);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return rd_cuda_fail(e, "rnea TMEM-state kernel launch");
    return RD_OK;
}

// Shared memory a block may use with four blocks per SM, and the padding that
// keeps a fifth from fitting (each block holds 128 of the SM's 512 TMEM columns).
inline void dht_smem_bounds(int device, size_t &max_block, size_t &min_block)
{
    static std::atomic<int> smem_sm[64];
    const int d = device & 63;
    if (smem_sm[d].load() == 0)
        smem_sm[d].store(dh_device_attr(device, cudaDevAttrMaxSharedMemoryPerMultiprocessor, 0));
    const size_t sm = (size_t)smem_sm[d].load();
    const size_t reserve = 1024 + 16;  // per-block reserve and the static TMEM-address word
    max_block = sm / 4 > reserve ? sm / 4 - reserve : 0;
    min_block = sm / 5 + 16 > reserve ? ((sm / 5 + 16 - reserve) + 15) / 16 * 16 : 0;
}

// K < 0: the largest K whose state fits four blocks per SM (two-stage ring if
// the three-stage one does not fit); K >= 0: that K with the deepest ring that fits.
inline int launch_dht(const rd_model *m, int K, int B, const void *q, const void *qd,
                      const void *qdd, void *tau, const BaseParams<float> &base, bool fast,
                      cudaStream_t s)
{
    const int n = m->n;
    size_t max_block, min_block;
    dht_smem_bounds(m->device, max_block, min_block);
    auto need = [&](int k, int stages) {
        return dht_smem_per_thread(n, k, k < kDhtMaxTmemLinks ? k : kDhtMaxTmemLinks, stages) *
               kDhtThreads;
    };
    int stages = 0;
    if (K < 0) {
        for (int k = n; k >= 0 && !stages; k -= 4)
            for (int st = 3; st >= 2 && !stages; --st)
                if (need(k, st) <= max_block) {
                    K = k;
                    stages = st;
                }
    } else {
        K = K > n ? n : 4 * (K / 4);
        for (int st = 3; st >= 2 && !stages; --st)
            if (need(K, st) <= max_block) stages = st;
    }
    if (!stages)
        return rd_fail(RD_ERR_ARG, "rnea_batch: TMEM-state kernel: state of %d links does not fit "
                                   "four blocks per SM", K);
    const int TL = K < kDhtMaxTmemLinks ? K : kDhtMaxTmemLinks;
    size_t smem = need(K, stages);
    if (smem < min_block) smem = min_block;
    if (stages == 3)
        return fast ? launch_dht_k<kTrigSfu, 3>(m, K, TL, B, q, qd, qdd, tau, base, smem, s)
                    : launch_dht_k<kTrigPoly, 3>(m, K, TL, B, q, qd, qdd, tau, base, smem, s);
    return fast ? launch_dht_k<kTrigSfu, 2>(m, K, TL, B, q, qd, qdd, tau, base, smem, s)
                : launch_dht_k<kTrigPoly, 2>(m, K, TL, B, q, qd, qdd, tau, base, smem, s);
}

// stored: state for the first K links (kfull; < 0 = library default), else
// none. Rows with n % 4 == 0, n <= 128 and 16-byte alignment take the
// parameter-constant kernel; others the shared-memory-constant kernel, with
// every link's state (stored) or none.
template <typename T>
int dh_launch(const rd_model *m, int B, const void *q, const void *qd, const void *qdd,
              void *tau, const double *base18, bool stored, int block, bool fast, int kfull,
              bool tmem, int reg_links, int stages, cudaStream_t s)
{
    double b[18];
    rd_convert_base_dh(m, base18, b);
    BaseParams<T> base;
    for (int k = 0; k < 6; ++k) {
        base.V0[k] = (T)b[k];
        base.dV0[k] = (T)b[6 + k];
        base.Fn[k] = (T)b[12 + k];
    }
    if constexpr (sizeof(T) == 4) {
        if (tmem) {
            if (!dhp_eligible<T>(m, q, qd, qdd, tau) || m->n > 32)
                return rd_fail(RD_ERR_ARG, "rnea_batch: the TMEM-state kernel needs FP32, "
                                           "n %% 4 == 0, n <= 32 and 16-byte aligned rows");
            return launch_dht(m, stored ? kfull : 0, B, q, qd, qdd, tau, base, fast, s);
        }
    }
    if ((reg_links || stages != kStages) && (!stored || tmem || !dhp_eligible<T>(m, q, qd, qdd, tau)))
        return rd_fail(RD_ERR_ARG, "rnea_batch: register state is for the stored-state "
                                   "common-normal kernel (n %% 4 == 0, aligned rows)");
    if (dhp_eligible<T>(m, q, qd, qdd, tau))
        return launch_dhp<T>(m, block ? block : 32, stored ? kfull : 0, B, q, qd, qdd, tau, base,
                             fast, s, reg_links, stages);
    if (stored) {
        if (!block)
            block = dh_smem<T>(m->n, 64, kStore, true) <= (size_t)dh_smem_optin(m->device) / 4 ? 64 : 32;
        return launch_dh_mode<T, kStore>(m, block, B, q, qd, qdd, tau, base, fast, s);
    }
    return launch_dh_mode<T, kRecompute>(m, block ? block : 64, B, q, qd, qdd, tau, base, fast, s);
}

}  // namespace
}  // namespace rdyn
