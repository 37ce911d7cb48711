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

// Rows per chunk of the host-array pipeline (B = 65536, n = 32 in FP32: 212 us
// per call with two chunks of 32768 rows, 223 with 16384, 248 with 8192: every
// chunk adds host-side calls and a copy start-up that outweigh the overlap).
#ifndef RD_HOST_CHUNK_ROWS
#define RD_HOST_CHUNK_ROWS 32768
#endif
constexpr int kHostMaxChunks = 16;

namespace {

// Three-stage pipeline over row chunks on (io_in, s, io_out): the inputs of
// chunk c+1 stream in while chunk c is computed and chunk c-1 streams out, so
// the inbound copies run back to back. A stream-wait captures the event as last
// recorded, so one pair of events serves every chunk. Enqueues only.
int enqueue_host_pipeline(rd_model *m, int B, int dtype, const void *q, const void *qd,
                          const void *qdd, void *tau, const double *base, int variant,
                          cudaStream_t s, size_t slot)
{
    const size_t row = (size_t)m->n * (dtype == RD_F32 ? 4 : 8);
    char *d = static_cast<char *>(m->d_io);
    char *dq = d, *dqd = d + slot, *dqdd = d + 2 * slot, *dtau = d + 3 * slot;
    // whole chunks of at least RD_HOST_CHUNK_ROWS rows (above the batch size
    // below which AUTO picks the lane-parallel scan), so the kernel chosen per
    // chunk, and with it the rounding, is the one the whole batch would get
    const long long nch = (long long)B / RD_HOST_CHUNK_ROWS;
    const int chunks = nch < 1 ? 1 : (nch > kHostMaxChunks ? kHostMaxChunks : (int)nch);
    cudaError_t e = cudaEventRecord(m->io_fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(m->io_in, m->io_fork, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(m->io_out, m->io_fork, 0);
    if (e != cudaSuccess) return rd_cuda_fail(e, "rnea_batch_host: fork");
    for (int c = 0; c < chunks; ++c) {
        const int b0 = (int)((long long)B * c / chunks), b1 = (int)((long long)B * (c + 1) / chunks);
        const size_t o = (size_t)b0 * row, len = (size_t)(b1 - b0) * row;
        e = cudaMemcpyAsync(dq + o, static_cast<const char *>(q) + o, len, cudaMemcpyHostToDevice, m->io_in);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dqd + o, static_cast<const char *>(qd) + o, len, cudaMemcpyHostToDevice, m->io_in);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dqdd + o, static_cast<const char *>(qdd) + o, len, cudaMemcpyHostToDevice, m->io_in);
        if (e == cudaSuccess) e = cudaEventRecord(m->io_in_done, m->io_in);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, m->io_in_done, 0);
        if (e != cudaSuccess) return rd_cuda_fail(e, "rnea_batch_host: copy to device");
        int rc = rnea_batch(m, b1 - b0, dtype, dq + o, dqd + o, dqdd + o, dtau + o, base, variant, s);
        if (rc) return rc;
        e = cudaEventRecord(m->io_kern_done, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(m->io_out, m->io_kern_done, 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(static_cast<char *>(tau) + o, dtau + o, len, cudaMemcpyDeviceToHost, m->io_out);
        if (e != cudaSuccess) return rd_cuda_fail(e, "rnea_batch_host: copy to host");
    }
    e = cudaEventRecord(m->io_join, m->io_out);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, m->io_join, 0);
    if (e != cudaSuccess) return rd_cuda_fail(e, "rnea_batch_host: join");
    return RD_OK;
}

// Device address of a host range the GPU can read and write in place (mapped
// pinned memory, as cudaHostAlloc gives under unified addressing), or null.
// Both ends of the range must resolve, to consecutive device addresses.
void *mapped_host_range(const void *p, size_t bytes)
{
    cudaPointerAttributes a, b;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
    const char *last = static_cast<const char *>(p) + bytes - 1;
    if (cudaPointerGetAttributes(&b, last) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (b.type != cudaMemoryTypeHost ||
        static_cast<char *>(b.devicePointer) != static_cast<char *>(a.devicePointer) + bytes - 1)
        return nullptr;
    return a.devicePointer;
}

// AUTO on FP32 rows the host-memory kernel takes (n % 4 == 0, n <= 64): the
// device addresses of all four arrays when each is mapped pinned memory on a
// 16-byte boundary.
bool host_in_place(const rd_model *m, int B, int dtype, const void *q, const void *qd,
                   const void *qdd, void *tau, int variant, void *dev[4])
{
    if (variant != RD_VARIANT_AUTO || dtype != RD_F32 || m->n % 4 != 0 || m->n > 64) return false;
    const size_t bytes = (size_t)B * (size_t)m->n * sizeof(float);
    const void *h[4] = {q, qd, qdd, tau};
    for (int k = 0; k < 4; ++k) {
        dev[k] = mapped_host_range(h[k], bytes);
        if (!dev[k] || (reinterpret_cast<uintptr_t>(dev[k]) & 15u)) return false;
    }
    return true;
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
    if (tau == q || tau == qd || tau == qdd)
        return rd_fail(RD_ERR_ARG, "rnea_batch_host: tau aliases an input");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool copy = (variant & RD_FLAG_HOST_COPY) != 0;
    variant &= ~RD_FLAG_HOST_COPY;
    void *dev[4];
    if (!copy && host_in_place(m, B, dtype, q, qd, qdd, tau, variant, dev)) {
        // the kernel moves the rows over the host link itself (rnea_dhz.cuh)
        double b18[18];
        rd_convert_base(m, base, b18);
        int rc = rd_rnea_dhz_f32(m, B, dev[0], dev[1], dev[2], dev[3], b18, s);
        if (rc) return rc;
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return rd_cuda_fail(e, "rnea_batch_host: synchronize");
        return RD_OK;
    }
    const size_t esz = dtype == RD_F32 ? 4 : 8;
    const size_t arr = (size_t)B * (size_t)m->n * esz;
    const size_t slot = (arr + 255) & ~(size_t)255;
    std::lock_guard<std::mutex> lk(m->io_mu);
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
    if (!m->io_in) {
        e = cudaStreamCreateWithFlags(&m->io_in, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&m->io_out, cudaStreamNonBlocking);
        cudaEvent_t *evs[4] = {&m->io_fork, &m->io_join, &m->io_in_done, &m->io_kern_done};
        for (int k = 0; k < 4 && e == cudaSuccess; ++k)
            e = cudaEventCreateWithFlags(evs[k], cudaEventDisableTiming);
        if (e != cudaSuccess) return rd_cuda_fail(e, "rnea_batch_host: stream set-up");
    }
    int rc = enqueue_host_pipeline(m, B, dtype, q, qd, qdd, tau, base, variant, s, slot);
    if (rc) return rc;
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return rd_cuda_fail(e, "rnea_batch_host: synchronize");
    return RD_OK;
}
