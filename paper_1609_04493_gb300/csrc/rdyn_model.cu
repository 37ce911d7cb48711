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
#include "spatial_dh.cuh"

thread_local std::string g_rd_error;
thread_local RdLaunchConfig g_rd_last_rnea;

extern "C" int rd_rnea_last_config(int *kernel, int *block, int *stored_links)
{
    if (!kernel || !block || !stored_links)
        return rd_fail(RD_ERR_ARG, "rd_rnea_last_config: null output");
    *kernel = g_rd_last_rnea.kernel;
    *block = g_rd_last_rnea.block;
    *stored_links = g_rd_last_rnea.stored_links;
    return RD_OK;
}

extern "C" int rd_rnea_last_state_layout(int *register_links, int *ring_chunks)
{
    if (!register_links || !ring_chunks)
        return rd_fail(RD_ERR_ARG, "rd_rnea_last_state_layout: null output");
    *register_links = g_rd_last_rnea.register_links;
    *ring_chunks = g_rd_last_rnea.ring_chunks;
    return RD_OK;
}

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

// Common-normal frames (spatial_dh.cuh) from the joint-frame constants: D_i is
// joint frame i' turned about its z axis by phi_i so that its x axis lies along
// z_i x z_{i+1} (phi_i = 0 for the last link and for parallel axes). Then the
// constant part of f_{i-1,i}, Rz(-phi_{i-1}) (A_i, b_i) Rz(phi_i), is checked to
// have the form (Rx(alpha_i) Rz(theta0_i), b_i'). D_{-1}, the base frame of the
// recursion, is D_0 at q_0 = 0; GB is its pose in frame 0. Host-side, FP64.
int rd_build_dh(int n, const std::vector<double> &c64, std::vector<double> &dh64, double GBR[9],
                double GBp[3], double *phi_last)
{
    constexpr int J = rdyn::kLinkConsts, D = rdyn::kDhConsts;
    std::vector<double> phi(n, 0.0);
    for (int i = 0; i + 1 < n; ++i) {
        const double *A = c64.data() + (size_t)(i + 1) * J;  // axis i+1 in frame i': A e_z
        const double ux = A[2], uy = A[5];
        if (std::hypot(ux, uy) > 1e-14) phi[i] = std::atan2(ux, -uy);
    }
    dh64.assign((size_t)n * D, 0.0);
    for (int i = 0; i < n; ++i) {
        const double *c = c64.data() + (size_t)i * J;
        double *o = dh64.data() + (size_t)i * D;
        const double cp = std::cos(phi[i]), sp = std::sin(phi[i]);
        if (i == 0) {
            o[0] = 1.0;  // alpha_0 = theta0_0 = 0, b_0 = 0
        } else {
            const double cm = std::cos(phi[i - 1]), sm = std::sin(phi[i - 1]);
            // Q = Rz(-phi_{i-1}) A Rz(phi_i); bD = Rz(-phi_{i-1}) b
            double T1[9], Q[9];
            for (int r = 0; r < 3; ++r) {
                const double *a = c + 3 * r;
                T1[3 * r + 0] = a[0] * cp + a[1] * sp;
                T1[3 * r + 1] = -a[0] * sp + a[1] * cp;
                T1[3 * r + 2] = a[2];
            }
            for (int k = 0; k < 3; ++k) {
                Q[0 + k] = cm * T1[0 + k] + sm * T1[3 + k];
                Q[3 + k] = -sm * T1[0 + k] + cm * T1[3 + k];
                Q[6 + k] = T1[6 + k];
            }
            const double b[3] = {c[9], c[10], c[11]};
            const double bD[3] = {cm * b[0] + sm * b[1], -sm * b[0] + cm * b[1], b[2]};
            double ca = Q[8], sa = -Q[5];
            const double h = std::hypot(ca, sa);
            ca /= h;
            sa /= h;
            // P = Rx(alpha)^T Q must be a rotation about z
            double P[9];
            for (int k = 0; k < 3; ++k) {
                P[0 + k] = Q[0 + k];
                P[3 + k] = ca * Q[3 + k] + sa * Q[6 + k];
                P[6 + k] = -sa * Q[3 + k] + ca * Q[6 + k];
            }
            const double th0 = std::atan2(P[3], P[0]);
            const double ct = std::cos(th0), st = std::sin(th0);
            const double Rz[9] = {ct, -st, 0, st, ct, 0, 0, 0, 1};
            double res = std::fabs(Q[2]);
            for (int k = 0; k < 9; ++k) res = std::fmax(res, std::fabs(P[k] - Rz[k]));
            if (!(res <= 1e-9))
                return rd_fail(RD_ERR_ARG, "link %d: common-normal frame residual %g", i, res);
            o[0] = ca;
            o[1] = sa;
            o[2] = bD[0];
            o[3] = bD[1];
            o[4] = bD[2];
            o[5] = th0;
        }
        // inertia in D_i: c_D = Rz(-phi) c', I_D = Rz(-phi) I' Rz(phi)
        o[6] = c[12];
        const double cc[3] = {c[13], c[14], c[15]};
        o[7] = cp * cc[0] + sp * cc[1];
        o[8] = -sp * cc[0] + cp * cc[1];
        o[9] = cc[2];
        const double I[3][3] = {{c[16], c[19], c[20]}, {c[19], c[17], c[21]}, {c[20], c[21], c[18]}};
        const double Rm[3][3] = {{cp, sp, 0}, {-sp, cp, 0}, {0, 0, 1}};  // Rz(-phi)
        double ID[3][3];
        for (int a = 0; a < 3; ++a)
            for (int bb = 0; bb < 3; ++bb) {
                double sum = 0;
                for (int k = 0; k < 3; ++k)
                    for (int l = 0; l < 3; ++l) sum += Rm[a][k] * I[k][l] * Rm[bb][l];
                ID[a][bb] = sum;
            }
        o[10] = ID[0][0];
        o[11] = ID[1][1];
        o[12] = ID[2][2];
        o[13] = 0.5 * (ID[0][1] + ID[1][0]);
        o[14] = 0.5 * (ID[0][2] + ID[2][0]);
        o[15] = 0.5 * (ID[1][2] + ID[2][1]);
    }
    // GB = (A_0 Rz(phi_0), b_0)
    const double *c0 = c64.data();
    const double cp = std::cos(phi[0]), sp = std::sin(phi[0]);
    for (int r = 0; r < 3; ++r) {
        const double *a = c0 + 3 * r;
        GBR[3 * r + 0] = a[0] * cp + a[1] * sp;
        GBR[3 * r + 1] = -a[0] * sp + a[1] * cp;
        GBR[3 * r + 2] = a[2];
        GBp[r] = c0[9 + r];
    }
    *phi_last = phi[n - 1];
    return RD_OK;
}

// FP64 forward-dynamics records (aba_dh.cuh) from the common-normal constants:
// the 16 constants, m c, C_o = I_c + m (|c|^2 - c c^T), cos^2 alpha, sin^2 alpha,
// cos alpha sin alpha, cos 2 alpha, sin 2 alpha; 32 per link.
void rd_build_aba64(int n, const std::vector<double> &dh64, std::vector<double> &out)
{
    out.assign((size_t)n * 32, 0.0);
    for (int i = 0; i < n; ++i) {
        const double *d = dh64.data() + (size_t)i * rdyn::kDhConsts;
        double *r = out.data() + (size_t)i * 32;
        for (int k = 0; k < rdyn::kDhConsts; ++k) r[k] = d[k];
        const double m = d[6], cx = d[7], cy = d[8], cz = d[9];
        r[16] = m * cx;
        r[17] = m * cy;
        r[18] = m * cz;
        r[19] = d[10] + m * (cy * cy + cz * cz);
        r[20] = d[11] + m * (cx * cx + cz * cz);
        r[21] = d[12] + m * (cx * cx + cy * cy);
        r[22] = d[13] - m * cx * cy;
        r[23] = d[14] - m * cx * cz;
        r[24] = d[15] - m * cy * cz;
        const double ca = d[0], sa = d[1];
        r[25] = ca * ca;
        r[26] = sa * sa;
        r[27] = ca * sa;
        r[28] = ca * ca - sa * sa;
        r[29] = 2.0 * ca * sa;
    }
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
    std::vector<double> dh64;
    rc = rd_build_dh(n, c64, dh64, mdl->GBR, mdl->GBp, &mdl->phi_last);
    if (rc) {
        delete mdl;
        return rc;
    }
    std::vector<float> dh32(dh64.begin(), dh64.end());
    mdl->host_dh64 = dh64;
    rd_build_aba64(n, dh64, mdl->host_aba64);

    std::vector<float> c32(c64.size());
    for (size_t k = 0; k < c64.size(); ++k) c32[k] = (float)c64[k];
    size_t b64 = c64.size() * sizeof(double), b32 = c32.size() * sizeof(float);
    e = cudaMalloc(&mdl->d_c64, b64);
    if (e == cudaSuccess) e = cudaMalloc(&mdl->d_c32, b32);
    if (e == cudaSuccess) e = cudaMemcpy(mdl->d_c64, c64.data(), b64, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(mdl->d_c32, c32.data(), b32, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&mdl->d_dh64, dh64.size() * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&mdl->d_dh32, dh32.size() * sizeof(float));
    if (e == cudaSuccess)
        e = cudaMemcpy(mdl->d_dh64, dh64.data(), dh64.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(mdl->d_dh32, dh32.data(), dh32.size() * sizeof(float), cudaMemcpyHostToDevice);
    // double-float pairs of the forward-dynamics records: hi = nearest float,
    // lo = nearest float of the remainder
    std::vector<float> abadf(2 * mdl->host_aba64.size());
    for (size_t k = 0; k < mdl->host_aba64.size(); ++k) {
        const double v = mdl->host_aba64[k];
        abadf[2 * k] = (float)v;
        abadf[2 * k + 1] = (float)(v - (double)(float)v);
    }
    if (e == cudaSuccess) e = cudaMalloc(&mdl->d_aba64, mdl->host_aba64.size() * sizeof(double));
    if (e == cudaSuccess)
        e = cudaMemcpy(mdl->d_aba64, mdl->host_aba64.data(), mdl->host_aba64.size() * sizeof(double),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&mdl->d_abadf, abadf.size() * sizeof(float));
    if (e == cudaSuccess)
        e = cudaMemcpy(mdl->d_abadf, abadf.data(), abadf.size() * sizeof(float), cudaMemcpyHostToDevice);
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
    if (m->d_dh32) cudaFree(m->d_dh32);
    if (m->d_dh64) cudaFree(m->d_dh64);
    if (m->d_aba64) cudaFree(m->d_aba64);
    if (m->d_abadf) cudaFree(m->d_abadf);
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

// Boundary terms in the common-normal frames, from those of rd_convert_base:
// V_0 and dV_0 move from frame 0 to D_{-1} (Ad_{GB^-1}: (R^T (v + w x p), R^T w)),
// F_{n+1} turns by -phi_last about z (D_{n-1} shares its origin with n').
void rd_convert_base_dh(const rd_model *m, const double in18[18], double out[18])
{
    const double *R = m->GBR, *p = m->GBp;
    for (int t = 0; t < 2; ++t) {
        const double *v = in18 + 6 * t, *w = in18 + 6 * t + 3;
        const double u[3] = {v[0] + w[1] * p[2] - w[2] * p[1], v[1] + w[2] * p[0] - w[0] * p[2],
                             v[2] + w[0] * p[1] - w[1] * p[0]};
        for (int a = 0; a < 3; ++a) {
            out[6 * t + a] = R[a] * u[0] + R[3 + a] * u[1] + R[6 + a] * u[2];
            out[6 * t + 3 + a] = R[a] * w[0] + R[3 + a] * w[1] + R[6 + a] * w[2];
        }
    }
    const double c = std::cos(m->phi_last), s = std::sin(m->phi_last);
    for (int t = 0; t < 2; ++t) {
        const double *x = in18 + 12 + 3 * t;
        out[12 + 3 * t + 0] = c * x[0] + s * x[1];
        out[12 + 3 * t + 1] = -s * x[0] + c * x[1];
        out[12 + 3 * t + 2] = x[2];
    }
}
