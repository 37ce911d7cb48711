// rdyn_vjp_noalloc.cu -- rnea_vjp_noalloc: the adjoint in its store mode with
// the workspace taken from a fixed-size array inside the library, so the call
// allocates nothing.
//
// Who needs this: callers that cannot or may not allocate device memory at
// the point of the call, such as a real-time control loop with a
// no-allocation rule, a plug-in running inside another framework that owns
// the device memory pool, or code that must not touch the allocator on its
// fast path. They still pass their own inputs and outputs; only the
// scratch space of the store mode comes from here.
//
// The scratch is a file-scope __device__ array of RD_VJP_NOALLOC_SCRATCH_BYTES.
// Every device that loads the library holds it until the process exits. On
// the host its name is only a stand-in: the kernel gets the device address,
// looked up once per device with cudaGetSymbolAddress while that device is
// current.
#include <cuda_runtime.h>

#include <mutex>

#include "rdyn_internal.h"

namespace {

__device__ __align__(256) unsigned char g_vjp_scratch[RD_VJP_NOALLOC_SCRATCH_BYTES];

std::mutex g_scratch_mu;
void *g_scratch_ptr[64] = {};

// Device address of the scratch array on the current device (looked up on the
// first call per device and kept for the life of the process; a
// cudaDeviceReset while the library is in use would leave it stale).
int scratch_address(int device, void **out)
{
    if (device < 0 || device >= 64)
        return rd_fail(RD_ERR_ARG, "rnea_vjp_noalloc: device %d out of range", device);
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_ptr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_vjp_scratch);
        if (e != cudaSuccess) return rd_cuda_fail(e, "rnea_vjp_noalloc: cudaGetSymbolAddress");
        g_scratch_ptr[device] = p;
    }
    *out = g_scratch_ptr[device];
    return RD_OK;
}

}  // namespace

extern "C" int rnea_vjp_noalloc(const rd_model *m, int B, int dtype, const void *q,
                                const void *qd, const void *qdd, const void *w, void *gq,
                                void *gqd, void *gqdd, const double *base, void *stream)
{
    g_rd_error.clear();
    if (!m) return rd_fail(RD_ERR_ARG, "rnea_vjp_noalloc: null model");
    if (B < 0) return rd_fail(RD_ERR_RANGE, "rnea_vjp_noalloc: B = %d < 0", B);
    if (dtype != RD_F32 && dtype != RD_F64)
        return rd_fail(RD_ERR_DTYPE, "rnea_vjp_noalloc: dtype %d is not RD_F32 or RD_F64", dtype);
    const size_t need = (size_t)m->n * 20 * (size_t)B * (dtype == RD_F32 ? 4 : 8);
    if (need > (size_t)RD_VJP_NOALLOC_SCRATCH_BYTES)
        return rd_fail(RD_ERR_RANGE,
                       "rnea_vjp_noalloc: B = %d states of %d links need %zu bytes of scratch; "
                       "the fixed scratch holds %zu (use rnea_vjp with a workspace)",
                       B, m->n, need, (size_t)RD_VJP_NOALLOC_SCRATCH_BYTES);
    if (B == 0) return RD_OK;
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return rd_cuda_fail(e, "rnea_vjp_noalloc: cudaGetDevice");
    void *ws = nullptr;
    int rc = scratch_address(dev, &ws);
    if (rc) return rc;
    // Every slot of the store-mode state is written by sweep 1 before sweep 2
    // reads it, so nothing in the scratch needs clearing between calls.
    return rnea_vjp(m, B, dtype, q, qd, qdd, w, gq, gqd, gqdd, base, RD_VJP_STORE, ws,
                    (size_t)RD_VJP_NOALLOC_SCRATCH_BYTES, stream);
}
