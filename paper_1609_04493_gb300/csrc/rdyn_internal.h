// rdyn_internal.h -- shared host-side declarations of librdyn.so.
#pragma once
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstddef>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/rdyn.h"
#include "spatial.cuh"

struct rd_model {
    int n = 0;
    int device = 0;
    float *d_c32 = nullptr;   // n * kLinkConsts, joint-frame constants (FP32)
    double *d_c64 = nullptr;  // same in FP64
    double TnR[9];            // joint frame of link n (for F_{n+1})
    double Tnp[3];
    float *d_dh32 = nullptr;  // n * kDhConsts, common-normal-frame constants (FP32)
    double *d_dh64 = nullptr; // same in FP64
    double GBR[9];            // base frame D_{-1} of the common-normal frames in frame 0
    double GBp[3];
    double phi_last = 0;      // D_{n-1} is the joint frame of link n turned by phi_last about z
    std::vector<double> host_dh64;  // the common-normal-frame constants on the host
    std::vector<double> host_aba64; // their FP64 forward-dynamics records (aba_dh.cuh)
    double *d_aba64 = nullptr;      // the records on the device
    float *d_abadf = nullptr;       // the records split into double-float pairs (hi, lo)
    std::vector<double> host_c64;
    // device staging for the host-pointer entry points, grown on demand
    void *d_io = nullptr;
    size_t io_bytes = 0;
    // host-array pipeline: copies in on io_in, kernels on the caller's stream,
    // copies out on io_out, chained per chunk by io_in_done / io_kern_done
    cudaStream_t io_in = nullptr, io_out = nullptr;
    cudaEvent_t io_fork = nullptr, io_join = nullptr, io_in_done = nullptr, io_kern_done = nullptr;
    std::mutex io_mu;
};

extern thread_local std::string g_rd_error;
// Kernel, block size and stored links of the calling thread's last rnea_batch
// launch (rd_rnea_last_config).
struct RdLaunchConfig {
    int kernel = 0, block = 0, stored_links = 0, register_links = 0, ring_chunks = 0;
};
extern thread_local RdLaunchConfig g_rd_last_rnea;
inline void rd_note_rnea(int kernel, int block, int stored, int register_links = 0,
                         int ring_chunks = 0)
{
    g_rd_last_rnea.kernel = kernel;
    g_rd_last_rnea.block = block;
    g_rd_last_rnea.stored_links = stored;
    g_rd_last_rnea.register_links = register_links;
    g_rd_last_rnea.ring_chunks = ring_chunks;
}
int rd_fail(int code, const char *fmt, ...);
int rd_cuda_fail(cudaError_t e, const char *what);
void rd_convert_base(const rd_model *m, const double *base, double out[18]);
void rd_convert_base_dh(const rd_model *m, const double in18[18], double out[18]);
int rd_build_dh(int n, const std::vector<double> &c64, std::vector<double> &dh64, double GBR[9],
                double GBp[3], double *phi_last);
void rd_build_aba64(int n, const std::vector<double> &dh64, std::vector<double> &out);
int rd_rnea_dh_f32(const rd_model *m, int B, const void *q, const void *qd, const void *qdd,
                   void *tau, const double *base18, int stored, int block, int fast,
                   int kfull, int tmem, int reg_links, int stages, cudaStream_t s);
int rd_rnea_dh_f64(const rd_model *m, int B, const void *q, const void *qd, const void *qdd,
                   void *tau, const double *base18, int stored, int block, int fast,
                   int kfull, int tmem, int reg_links, int stages, cudaStream_t s);
// FP32 inverse dynamics reading and writing mapped pinned host arrays (device
// addresses), n % 4 == 0, n <= 64, 16-byte aligned
int rd_rnea_dhz_f32(const rd_model *m, int B, const void *q, const void *qd, const void *qdd,
                    void *tau, const double *base18, cudaStream_t s);
// FP64 data in double-float arithmetic (RD_VARIANT_SERIAL_DF), n <= 64
int rd_rnea_df_f64(const rd_model *m, int B, const void *q, const void *qd, const void *qdd,
                   void *tau, const double *base18, int block, cudaStream_t s);
// the double-float sine and cosine of the FP64 kernels, as doubles (rd_joint_trig_df)
int rd_df_trig_launch(const double *x, double *s, double *c, int count, cudaStream_t stream);
int rd_rnea_dispatch_f32(const rd_model *m, int B, const void *q, const void *qd,
                         const void *qdd, void *tau, const double *base18, int variant,
                         cudaStream_t s);
int rd_rnea_dispatch_f64(const rd_model *m, int B, const void *q, const void *qd,
                         const void *qdd, void *tau, const double *base18, int variant,
                         cudaStream_t s);
int rd_vjp_dispatch_f32(const rd_model *m, int B, const void *q, const void *qd, const void *qdd,
                        const void *w, void *gq, void *gqd, void *gqdd, const double *base18,
                        int mode, void *ws, size_t ws_bytes, cudaStream_t s);
int rd_vjp_dispatch_f64(const rd_model *m, int B, const void *q, const void *qd, const void *qdd,
                        const void *w, void *gq, void *gqd, void *gqdd, const double *base18,
                        int mode, void *ws, size_t ws_bytes, cudaStream_t s);
int rd_aba_dispatch_f32(const rd_model *m, int B, const void *q, const void *qd, const void *tau,
                        void *qdd, int *status, void *ws, size_t ws_bytes, const double *base18,
                        int flags, cudaStream_t s);
int rd_aba_dispatch_f64(const rd_model *m, int B, const void *q, const void *qd, const void *tau,
                        void *qdd, int *status, void *ws, size_t ws_bytes, const double *base18,
                        int flags, cudaStream_t s);
// the adjoint with L lanes per instance (rnea_vjp_lane.cuh), FP32
int rd_vjp_lane_f32(const rd_model *m, int B, const void *q, const void *qd, const void *qdd,
                    const void *w, void *gq, void *gqd, void *gqdd, const double *base18,
                    bool fast_trig, int lanes, cudaStream_t s);
// forward dynamics with one warp per instance (aba_warp.cuh)
int rd_aba_warp_f32(const rd_model *m, int B, const void *q, const void *qd, const void *tau,
                    void *qdd, int *status, const double *base18, bool fp64_update,
                    bool extended_bias, cudaStream_t s);
int rd_aba_warp_f64(const rd_model *m, int B, const void *q, const void *qd, const void *tau,
                    void *qdd, int *status, const double *base18, cudaStream_t s);
// forward dynamics with two warps per 32 instances (aba_pair.cuh); withhold:
// the RD_ABA_TEST_WITHHOLD hook
int rd_aba_pair_f32(const rd_model *m, int B, const void *q, const void *qd, const void *tau,
                    void *qdd, int *status, void *ws, const double *base18, bool fp64_update,
                    bool extended_bias, bool withhold, cudaStream_t s);
int rd_aba_pair_f64(const rd_model *m, int B, const void *q, const void *qd, const void *tau,
                    void *qdd, int *status, void *ws, const double *base18, bool withhold,
                    cudaStream_t s);
// the same with the articulated-inertia recursion split over two warps
// (three warps per 32 instances, aba_tri.cuh)
int rd_aba_tri_f32(const rd_model *m, int B, const void *q, const void *qd, const void *tau,
                   void *qdd, int *status, void *ws, const double *base18, bool fp64_update,
                   bool extended_bias, cudaStream_t s);
int rd_aba_tri_f64(const rd_model *m, int B, const void *q, const void *qd, const void *tau,
                   void *qdd, int *status, void *ws, const double *base18, cudaStream_t s);
size_t rd_aba_ws_bytes_f32(int n, int B, int flags);
size_t rd_aba_ws_bytes_f64(int n, int B, int flags);
int rd_build_chain(int n, const double *M, const double *S, const double *inertia,
                   std::vector<double> &c64, double TnR[9], double Tnp[3]);
