// rdyn_rnea.cu -- rnea_batch / rnea_batch_host: argument checks, variant
// choice and launches of the inverse-dynamics kernels (Algorithm 1).
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "rdyn_internal.h"


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
    if (dtype == RD_F32) return rd_rnea_dispatch_f32(m, B, q, qd, qdd, tau, b18, variant, s);
    return rd_rnea_dispatch_f64(m, B, q, qd, qdd, tau, b18, variant, s);
}

namespace {

// Device-visible address of a pinned (page-locked or registered) host buffer,
// or nullptr when the pointer is not one.
const void *pinned_device_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
    return a.devicePointer;
}

}  // namespace

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
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    // Pinned host arrays: the kernel reads and writes them in place over the
    // host link (coherent on Grace-Blackwell), no staging copies.
    const void *dq = pinned_device_ptr(q), *dqd = pinned_device_ptr(qd),
               *dqdd = pinned_device_ptr(qdd), *dtau = pinned_device_ptr(tau);
    if (dq && dqd && dqdd && dtau) {
        int rc = rnea_batch(m, B, dtype, dq, dqd, dqdd, const_cast<void *>(dtau), base, variant,
                            stream);
        if (rc) return rc;
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return rd_cuda_fail(e, "rnea_batch_host: synchronize");
        return RD_OK;
    }
    // Otherwise stage through device buffers owned by the model.
    const size_t esz = dtype == RD_F32 ? 4 : 8;
    const size_t arr = (size_t)B * m->n * esz;
    const size_t slot = (arr + 255) & ~(size_t)255;
    std::lock_guard<std::mutex> lk(m->io_mu);
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
    void *sq = d, *sqd = d + slot, *sqdd = d + 2 * slot, *stau = d + 3 * slot;
    e = cudaMemcpyAsync(sq, q, arr, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sqd, qd, arr, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sqdd, qdd, arr, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return rd_cuda_fail(e, "rnea_batch_host: copy to device");
    int rc = rnea_batch(m, B, dtype, sq, sqd, sqdd, stau, base, variant, stream);
    if (rc) return rc;
    e = cudaMemcpyAsync(tau, stau, arr, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return rd_cuda_fail(e, "rnea_batch_host: copy to host");
    return RD_OK;
}
