// rdyn_model.cu -- model upload and the library's error state.
//
// rd_model_create re-expresses the user's chain (Sec. II-A: M_i, S_i, J_i)
// in joint frames: for every link a frame i' with its z axis on the joint
// axis and its origin at the point of the axis nearest to frame i's origin.
// With T_i mapping frame-i' coordinates to frame i,
//     S_i = Ad_{T_i} (0, 0, 0, 0, 0, 1),
//     exp([S_i] q) = T_i Rz(q) T_i^-1,
//     f'_{i-1,i} = T_{i-1}^-1 f_{i-1,i} T_i = (T_{i-1}^-1 M_i T_i) Rz(q),
// so each link transform becomes a constant rigid motion times a rotation
// about z, and tau_i = S_i^T F_i is the z moment of the wrench in frame i'.
// Twists and wrenches are the same physical quantities in other
// coordinates; the torques are unchanged. Base frame 0 is kept (T_0 = I).
// All of this runs once, in double precision, on the host.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "rdyn_internal.h"

thread_local std::string g_rd_error;

int rd_fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_rd_error = buf;
    return code;
}

int rd_cuda_fail(cudaError_t e, const char *what)
{
    return rd_fail(RD_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

namespace {

struct Rigid {
    double R[9];  // row-major
    double p[3];
};

Rigid compose(const Rigid &a, const Rigid &b)
{
    Rigid c;
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += a.R[3 * i + k] * b.R[3 * k + j];
            c.R[3 * i + j] = s;
        }
        double t = a.p[i];
        for (int k = 0; k < 3; ++k) t += a.R[3 * i + k] * b.p[k];
        c.p[i] = t;
    }
    return c;
}

Rigid inverse(const Rigid &a)
{
    Rigid c;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) c.R[3 * i + j] = a.R[3 * j + i];
    for (int i = 0; i < 3; ++i) {
        double t = 0;
        for (int k = 0; k < 3; ++k) t += c.R[3 * i + k] * a.p[k];
        c.p[i] = -t;
    }
    return c;
}

// Joint frame of a revolute twist S = (v, w): columns (x, y, w), origin r = w x v.
int joint_frame(int link, const double *S, Rigid &T)
{
    double w[3] = {S[3], S[4], S[5]}, v[3] = {S[0], S[1], S[2]};
    double nw = std::sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    if (!(std::fabs(nw - 1.0) <= 1e-6))
        return rd_fail(RD_ERR_ARG, "link %d: joint axis |w| = %g, expected 1", link, nw);
    for (double &x : w) x /= nw;
    double nv = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    double pitch = w[0] * v[0] + w[1] * v[1] + w[2] * v[2];
    if (!(std::fabs(pitch) <= 1e-9 * (1.0 + nv)))
        return rd_fail(RD_ERR_ARG, "link %d: twist has pitch w.v = %g; only revolute joints "
                                   "(w.v = 0) are supported", link, pitch);
    double r[3] = {w[1] * v[2] - w[2] * v[1], w[2] * v[0] - w[0] * v[2],
                   w[0] * v[1] - w[1] * v[0]};
    double a[3] = {0, 0, 0};
    if (std::fabs(w[0]) < 0.9) a[0] = 1; else a[1] = 1;
    double d = a[0] * w[0] + a[1] * w[1] + a[2] * w[2];
    double x[3] = {a[0] - d * w[0], a[1] - d * w[1], a[2] - d * w[2]};
    double nx = std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
    for (double &e : x) e /= nx;
    double y[3] = {w[1] * x[2] - w[2] * x[1], w[2] * x[0] - w[0] * x[2],
                   w[0] * x[1] - w[1] * x[0]};
    for (int i = 0; i < 3; ++i) {
        T.R[3 * i + 0] = x[i];
        T.R[3 * i + 1] = y[i];
        T.R[3 * i + 2] = w[i];
        T.p[i] = r[i];
    }
    return RD_OK;
}

// Symmetric positive semi-definite test by principal minors (a point mass,
// I_c = 0, is allowed), with a tolerance relative to the trace.
bool psd3(const double I[3][3])
{
    double tr = std::fabs(I[0][0]) + std::fabs(I[1][1]) + std::fabs(I[2][2]);
    double eps = 1e-12 * (tr + 1e-300);
    for (int i = 0; i < 3; ++i)
        if (!(I[i][i] >= -eps)) return false;
    for (int i = 0; i < 3; ++i)
        for (int j = i + 1; j < 3; ++j)
            if (!(I[i][i] * I[j][j] - I[i][j] * I[j][i] >= -eps * tr)) return false;
    double det = I[0][0] * (I[1][1] * I[2][2] - I[1][2] * I[2][1]) -
                 I[0][1] * (I[1][0] * I[2][2] - I[1][2] * I[2][0]) +
                 I[0][2] * (I[1][0] * I[2][1] - I[1][1] * I[2][0]);
    return det >= -eps * tr * tr;
}

}  // namespace

extern "C" int rd_version(void) { return 100; }

extern "C" const char *rd_last_error(void) { return g_rd_error.c_str(); }

extern "C" int rd_model_links(const rd_model *m)
{
    if (!m) return rd_fail(RD_ERR_ARG, "rd_model_links: null model");
    return m->n;
}

// Joint-frame constants of one chain (24 doubles per link, see spatial.cuh) and
// the joint frame of its last link (for F_{n+1}). Host-side, FP64.
int rd_build_chain(int n, const double *M, const double *S, const double *inertia,
                   std::vector<double> &c64, double TnR[9], double Tnp[3])
{
    if (n < 1 || n > RD_MAX_LINKS)
        return rd_fail(RD_ERR_RANGE, "n = %d outside [1, %d]", n, RD_MAX_LINKS);
    if (!M || !S || !inertia) return rd_fail(RD_ERR_ARG, "null model array");
    std::vector<Rigid> T(n + 1);
    for (int k = 0; k < 9; ++k) T[0].R[k] = (k % 4 == 0) ? 1.0 : 0.0;
    T[0].p[0] = T[0].p[1] = T[0].p[2] = 0.0;
    for (int i = 0; i < n; ++i) {
        int rc = joint_frame(i, S + 6 * i, T[i + 1]);
        if (rc) return rc;
    }
    c64.assign((size_t)n * rdyn::kLinkConsts, 0.0);
    for (int i = 0; i < n; ++i) {
        const double *in = inertia + 10 * i;
        double m = in[0];
        if (!(m > 0) || !std::isfinite(m))
            return rd_fail(RD_ERR_ARG, "link %d: mass %g must be positive", i, m);
        double Ic[3][3] = {{in[4], in[7], in[8]}, {in[7], in[5], in[9]}, {in[8], in[9], in[6]}};
        if (!psd3(Ic))
            return rd_fail(RD_ERR_ARG, "link %d: inertia about the centre of mass is not "
                                       "positive semi-definite", i);
        Rigid Mi;
        for (int k = 0; k < 9; ++k) Mi.R[k] = M[12 * i + k];
        for (int k = 0; k < 3; ++k) Mi.p[k] = M[12 * i + 9 + k];
        for (int k = 0; k < 12; ++k)
            if (!std::isfinite(M[12 * i + k]))
                return rd_fail(RD_ERR_ARG, "link %d: non-finite home transform", i);
        Rigid Mp = compose(compose(inverse(T[i]), Mi), T[i + 1]);
        const Rigid &Ti = T[i + 1];
        // c' = R^T (c - r), I' = R^T I_c R
        double dc[3] = {in[1] - Ti.p[0], in[2] - Ti.p[1], in[3] - Ti.p[2]};
        double cp[3], Ip[3][3];
        for (int a = 0; a < 3; ++a) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += Ti.R[3 * k + a] * dc[k];
            cp[a] = s;
        }
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double s = 0;
                for (int k = 0; k < 3; ++k)
                    for (int l = 0; l < 3; ++l) s += Ti.R[3 * k + a] * Ic[k][l] * Ti.R[3 * l + b];
                Ip[a][b] = s;
            }
        double *o = c64.data() + (size_t)i * rdyn::kLinkConsts;
        for (int k = 0; k < 9; ++k) o[k] = Mp.R[k];
        for (int k = 0; k < 3; ++k) o[9 + k] = Mp.p[k];
        o[12] = m;
        for (int k = 0; k < 3; ++k) o[13 + k] = cp[k];
        o[16] = Ip[0][0];
        o[17] = Ip[1][1];
        o[18] = Ip[2][2];
        o[19] = 0.5 * (Ip[0][1] + Ip[1][0]);
        o[20] = 0.5 * (Ip[0][2] + Ip[2][0]);
        o[21] = 0.5 * (Ip[1][2] + Ip[2][1]);
    }
    for (int k = 0; k < 9; ++k) TnR[k] = T[n].R[k];
    for (int k = 0; k < 3; ++k) Tnp[k] = T[n].p[k];
    return RD_OK;
}

extern "C" int rd_model_create(int n, const double *M, const double *S, const double *inertia,
                               rd_model **out)
{
    g_rd_error.clear();
    if (!out) return rd_fail(RD_ERR_ARG, "rd_model_create: out is null");
    *out = nullptr;
    if (n < 1 || n > RD_MAX_LINKS)
        return rd_fail(RD_ERR_RANGE, "rd_model_create: n = %d outside [1, %d]", n, RD_MAX_LINKS);
    if (!M || !S || !inertia) return rd_fail(RD_ERR_ARG, "rd_model_create: null model array");
    std::vector<double> c64;
    double TnR[9], Tnp[3];
    int rc = rd_build_chain(n, M, S, inertia, c64, TnR, Tnp);
    if (rc) return rc;

    rd_model *mdl = new (std::nothrow) rd_model();
    if (!mdl) return rd_fail(RD_ERR_ALLOC, "rd_model_create: host allocation failed");
    mdl->n = n;
    cudaError_t e = cudaGetDevice(&mdl->device);
    if (e != cudaSuccess) {
        delete mdl;
        return rd_cuda_fail(e, "cudaGetDevice");
    }
    for (int k = 0; k < 9; ++k) mdl->TnR[k] = TnR[k];
    for (int k = 0; k < 3; ++k) mdl->Tnp[k] = Tnp[k];
    mdl->host_c64 = c64;

    std::vector<float> c32(c64.size());
    for (size_t k = 0; k < c64.size(); ++k) c32[k] = (float)c64[k];
    size_t b64 = c64.size() * sizeof(double), b32 = c32.size() * sizeof(float);
    e = cudaMalloc(&mdl->d_c64, b64);
    if (e == cudaSuccess) e = cudaMalloc(&mdl->d_c32, b32);
    if (e == cudaSuccess) e = cudaMemcpy(mdl->d_c64, c64.data(), b64, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(mdl->d_c32, c32.data(), b32, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        rd_model_destroy(mdl);
        return e == cudaErrorMemoryAllocation ? rd_fail(RD_ERR_ALLOC, "rd_model_create: %s",
                                                        cudaGetErrorString(e))
                                              : rd_cuda_fail(e, "rd_model_create");
    }
    *out = mdl;
    return RD_OK;
}

extern "C" void rd_model_destroy(rd_model *m)
{
    if (!m) return;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != m->device) cudaSetDevice(m->device);
    if (m->d_c32) cudaFree(m->d_c32);
    if (m->d_c64) cudaFree(m->d_c64);
    if (m->d_io) cudaFree(m->d_io);
    if (m->io_in) cudaStreamDestroy(m->io_in);
    if (m->io_out) cudaStreamDestroy(m->io_out);
    if (m->io_fork) cudaEventDestroy(m->io_fork);
    if (m->io_join) cudaEventDestroy(m->io_join);
    if (m->io_in_done) cudaEventDestroy(m->io_in_done);
    if (m->io_kern_done) cudaEventDestroy(m->io_kern_done);
    if (prev >= 0 && prev != m->device) cudaSetDevice(prev);
    delete m;
}

// Boundary terms for the kernels: V_0, dV_0 stay in frame 0; F_{n+1} moves
// from frame n to frame n': f' = R^T f, n' = R^T (n - r x f).
void rd_convert_base(const rd_model *m, const double *base, double out[18])
{
    static const double dflt[18] = {0, 0, 0, 0, 0, 0, 0, 0, 9.81, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    const double *b = base ? base : dflt;
    for (int k = 0; k < 12; ++k) out[k] = b[k];
    const double *f = b + 12, *nn = b + 15;
    const double *R = m->TnR, *r = m->Tnp;
    double rxf[3] = {r[1] * f[2] - r[2] * f[1], r[2] * f[0] - r[0] * f[2],
                     r[0] * f[1] - r[1] * f[0]};
    for (int a = 0; a < 3; ++a) {
        double sf = 0, sn = 0;
        for (int k = 0; k < 3; ++k) {
            sf += R[3 * k + a] * f[k];
            sn += R[3 * k + a] * (nn[k] - rxf[k]);
        }
        out[12 + a] = sf;
        out[15 + a] = sn;
    }
}
