// rdyn_rnea.cu -- rnea_batch / rnea_batch_host: argument checks, variant
// choice and launches of the inverse-dynamics kernels (Algorithm 1).
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "rdyn_internal.h"
#include "rnea_serial.cuh"

using namespace rdyn;

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
size_t serial_smem(int n, int block, int mode)
{
    size_t s = (size_t)n * kLinkConsts * sizeof(T);
    if (mode == kStore) s += (size_t)n * state_bytes_per_link<T>() * block;
    return s;
}

template <typename T, int BLOCK, int MODE>
int launch_serial(const rd_model *m, int B, const void *q, const void *qd, const void *qdd,
                  void *tau, const double *base18, cudaStream_t stream)
{
    static std::atomic<uint64_t> configured{0};
    const int n = m->n;
    size_t smem = serial_smem<T>(n, BLOCK, MODE);
    if (smem > (size_t)max_smem_optin(m->device))
        return rd_fail(RD_ERR_ARG, "rnea_batch: %zu bytes of shared memory needed, %d available",
                       smem, max_smem_optin(m->device));
    auto kern = rnea_serial_kernel<T, BLOCK, MODE>;
    cudaError_t e = allow_smem(kern, m->device, configured);
    if (e != cudaSuccess) return rd_cuda_fail(e, "cudaFuncSetAttribute");
    const T *consts = nullptr;
    if constexpr (sizeof(T) == 4) consts = reinterpret_cast<const T *>(m->d_c32);
    else consts = reinterpret_cast<const T *>(m->d_c64);
    unsigned grid = (unsigned)((B + BLOCK - 1) / BLOCK);
    kern<<<grid, BLOCK, smem, stream>>>(consts, n, B, static_cast<const T *>(q),
                                        static_cast<const T *>(qd), static_cast<const T *>(qdd),
                                        static_cast<T *>(tau), make_base<T>(base18));
    e = cudaGetLastError();
    if (e != cudaSuccess) return rd_cuda_fail(e, "rnea kernel launch");
    return RD_OK;
}

template <typename T>
int dispatch(const rd_model *m, int B, const void *q, const void *qd, const void *qdd, void *tau,
             const double *base18, int variant, cudaStream_t s)
{
    const int n = m->n;
    const int limit = max_smem_optin(m->device);
    if (variant == RD_VARIANT_AUTO) {
        // one thread per instance; keep per-link state in shared memory when at
        // least two warps' worth fits, else re-derive it in the backward sweep
        variant = serial_smem<T>(n, 64, kStore) <= (size_t)limit ? RD_VARIANT_SERIAL
                                                                 : RD_VARIANT_SERIAL_RECOMPUTE;
    }
    if (variant == RD_VARIANT_SERIAL) {
        if (serial_smem<T>(n, 64, kStore) <= (size_t)limit / 2)
            return launch_serial<T, 64, kStore>(m, B, q, qd, qdd, tau, base18, s);
        if (serial_smem<T>(n, 32, kStore) <= (size_t)limit)
            return launch_serial<T, 32, kStore>(m, B, q, qd, qdd, tau, base18, s);
        return rd_fail(RD_ERR_ARG, "rnea_batch: per-link state of %d links does not fit in "
                                   "shared memory; use RD_VARIANT_SERIAL_RECOMPUTE", n);
    }
    if (variant == RD_VARIANT_SERIAL_RECOMPUTE)
        return launch_serial<T, 128, kRecompute>(m, B, q, qd, qdd, tau, base18, s);
    return rd_fail(RD_ERR_ARG, "rnea_batch: unknown variant 0x%x", variant);
}

}  // namespace

extern "C" int rnea_batch(const rd_model *m, int B, int dtype, const void *q, const void *qd,
                          const void *qdd, void *tau, const double *base, int variant,
                          void *stream)
{
    g_rd_error.clear();
    if (!m) return rd_fail(RD_ERR_ARG, "rnea_batch: null model");
    if (B < 0) return rd_fail(RD_ERR_RANGE, "rnea_batch: B = %d < 0", B);
    if (dtype != RD_F32 && dtype != RD_F64)
        return rd_fail(RD_ERR_DTYPE, "rnea_batch: dtype %d is not RD_F32 or RD_F64", dtype);
    if (B == 0) return RD_OK;
    if (!q || !qd || !qdd || !tau) return rd_fail(RD_ERR_ARG, "rnea_batch: null batch pointer");
    if (tau == q || tau == qd || tau == qdd)
        return rd_fail(RD_ERR_ARG, "rnea_batch: tau aliases an input");
    double b18[18];
    rd_convert_base(m, base, b18);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (dtype == RD_F32) return dispatch<float>(m, B, q, qd, qdd, tau, b18, variant, s);
    return dispatch<double>(m, B, q, qd, qdd, tau, b18, variant, s);
}

extern "C" int rnea_batch_host(rd_model *m, int B, int dtype, const void *q, const void *qd,
                               const void *qdd, void *tau, const double *base, int variant,
                               void *stream)
{
    g_rd_error.clear();
    if (!m) return rd_fail(RD_ERR_ARG, "rnea_batch_host: null model");
    if (B < 0) return rd_fail(RD_ERR_RANGE, "rnea_batch_host: B = %d < 0", B);
    if (dtype != RD_F32 && dtype != RD_F64)
        return rd_fail(RD_ERR_DTYPE, "rnea_batch_host: dtype %d is not RD_F32 or RD_F64", dtype);
    if (B == 0) return RD_OK;
    if (!q || !qd || !qdd || !tau)
        return rd_fail(RD_ERR_ARG, "rnea_batch_host: null batch pointer");
    const size_t esz = dtype == RD_F32 ? 4 : 8;
    const size_t arr = (size_t)B * m->n * esz;
    const size_t slot = (arr + 255) & ~(size_t)255;
    std::lock_guard<std::mutex> lk(m->io_mu);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (m->io_bytes < 4 * slot) {
        if (m->d_io) {
            e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return rd_cuda_fail(e, "cudaStreamSynchronize");
            cudaFree(m->d_io);
            m->d_io = nullptr;
            m->io_bytes = 0;
        }
        e = cudaMalloc(&m->d_io, 4 * slot);
        if (e != cudaSuccess) return rd_fail(RD_ERR_ALLOC, "rnea_batch_host: %s",
                                             cudaGetErrorString(e));
        m->io_bytes = 4 * slot;
    }
    char *d = static_cast<char *>(m->d_io);
    void *dq = d, *dqd = d + slot, *dqdd = d + 2 * slot, *dtau = d + 3 * slot;
    e = cudaMemcpyAsync(dq, q, arr, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dqd, qd, arr, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dqdd, qdd, arr, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return rd_cuda_fail(e, "rnea_batch_host: copy to device");
    int rc = rnea_batch(m, B, dtype, dq, dqd, dqdd, dtau, base, variant, stream);
    if (rc) return rc;
    e = cudaMemcpyAsync(tau, dtau, arr, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return rd_cuda_fail(e, "rnea_batch_host: copy to host");
    return RD_OK;
}
