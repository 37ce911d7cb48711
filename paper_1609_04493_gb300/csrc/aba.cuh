// aba.cuh -- forward dynamics by the articulated-body algorithm (Sec. II-B,
// Eqs. abi and recursive-fd; Sec. III-D casts its linear recursions as scans),
// one thread per instance, in joint frames (S_i = e_z angular, so
// Omega_i = S^T J_hat_i S is the (w_z, w_z) entry and U_i = J_hat_i S_i the last
// column of J_hat_i).
//
//   sweep 1, base -> tip (T):  bias motion with qdd = 0 and the bias wrenches
//            F_hat_i (the forward half of tau_bias = ID(q, qd, 0, V_0, dV_0, F_{n+1})).
//   sweep 2, tip -> base:  F_i and tau_hat_i = tau_i - S^T F_i (T);
//            J_hat_i = J_i + X^T (J_hat_{i+1} - U U^T / Omega_{i+1}) X   (FP64),
//                X = Ad_{f_{i+1}^-1};   Omega_i, U_i;
//            z_hat_i = Y_{i,i+1} z_hat_{i+1} + Pi_{i,i+1} tau_hat_{i+1}
//                    = X^T (z_hat_{i+1} + U_{i+1} c_hat_{i+1}),
//            c_hat_i = (tau_hat_i - S^T z_hat_i) / Omega_i                   (FP64).
//   sweep 3, base -> tip:  a_i = Ad_{f_i^-1} lambda_{i-1},
//            qdd_i = c_hat_i - U_i^T a_i / Omega_i   (= c_hat_i - Pi_{i-1,i}^T lambda_{i-1}),
//            lambda_i = a_i + S_i qdd_i              (= Y^T_{i-1,i} lambda_{i-1} + S_i c_hat_i).
// The articulated-inertia update and the divisions by Omega (the D_i solves)
// run in FP64 whatever T is. The z_hat / lambda recursions run in FP64 by
// default (Z = double): in FP32 their accumulation over long chains cancels
// against tau_hat at the base (n = 64: round-trip residual 5e-3 of max|tau|);
// Z = T keeps them in the data precision.
// Per-link state between sweeps lives in a caller-provided workspace,
// component-major ([link][component][instance]) so a warp's accesses coalesce:
// n * 10 scalars of T (F_hat then cos, sin) and n * 8 of Z (U, c_hat, 1/Omega).
#pragma once
#include "../../include/rdyn.h"
#include "rnea_serial.cuh"

namespace rdyn {

constexpr int kAbaStateScalars = 10;

// symmetric 3x3 in the scalar D (double, or the double-float pair of df.cuh)
template <typename D>
struct Sym3 {
    D xx, yy, zz, xy, xz, yz;
};
using Sym3d = Sym3<double>;

// 6x6 symmetric [[A, Bm], [Bm^T, C]] in twist order (v, w)
template <typename D>
struct AbiT {
    Sym3<D> A;
    D Bm[9];  // row-major
    Sym3<D> C;
};
using Abi = AbiT<double>;

template <typename D>
__device__ __forceinline__ void sym_to_full(const Sym3<D> &s, D m[9])
{
    m[0] = s.xx; m[1] = s.xy; m[2] = s.xz;
    m[3] = s.xy; m[4] = s.yy; m[5] = s.yz;
    m[6] = s.xz; m[7] = s.yz; m[8] = s.zz;
}

// R X R^T for a full 3x3 X (row-major R)
__device__ __forceinline__ void rot_congr(const double R[9], const double X[9], double out[9])
{
    double T[9];  // X R^T
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            T[3 * i + j] = fma(X[3 * i], R[3 * j], fma(X[3 * i + 1], R[3 * j + 1], X[3 * i + 2] * R[3 * j + 2]));
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            out[3 * i + j] = fma(R[3 * i], T[j], fma(R[3 * i + 1], T[3 + j], R[3 * i + 2] * T[6 + j]));
}

__device__ __forceinline__ Sym3d rot_congr_sym(const double R[9], const Sym3d &s)
{
    double X[9], T[9];
    sym_to_full(s, X);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            T[3 * i + j] = fma(X[3 * i], R[3 * j], fma(X[3 * i + 1], R[3 * j + 1], X[3 * i + 2] * R[3 * j + 2]));
    auto e = [&](int i, int j) {
        return fma(R[3 * i], T[j], fma(R[3 * i + 1], T[3 + j], R[3 * i + 2] * T[6 + j]));
    };
    return Sym3d{e(0, 0), e(1, 1), e(2, 2), e(0, 1), e(0, 2), e(1, 2)};
}

// [b] X (each column crossed with b)
template <typename D>
__device__ __forceinline__ void hat_mul(const D b[3], const D X[9], D out[9])
{
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const D x0 = X[j], x1 = X[3 + j], x2 = X[6 + j];
        out[j] = fma(b[1], x2, -b[2] * x1);
        out[3 + j] = fma(b[2], x0, -b[0] * x2);
        out[6 + j] = fma(b[0], x1, -b[1] * x0);
    }
}

// X^T M X with X = Ad_{f^-1}, f = (R, b): rotate the blocks by R, then shift:
//   A' = A_r,  B' = B_r - A_r [b],  C' = C_r + [b]B_r - B_r^T[b] - [b]A_r[b].
__device__ __forceinline__ Abi abi_congruence(const Abi &M, const double R[9], const double b[3])
{
    Abi o;
    o.A = rot_congr_sym(R, M.A);
    double Br[9];
    rot_congr(R, M.Bm, Br);
    const Sym3d Cr = rot_congr_sym(R, M.C);
    double Ar[9], P[9], N[9], Q2[9], PT[9];
    sym_to_full(o.A, Ar);
    hat_mul(b, Ar, P);  // P = [b] A_r;  A_r [b] = -P^T
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) PT[3 * i + j] = P[3 * j + i];
#pragma unroll
    for (int k = 0; k < 9; ++k) o.Bm[k] = Br[k] + PT[k];
    hat_mul(b, Br, N);   // [b] B_r;  -B_r^T [b] = N^T
    hat_mul(b, PT, Q2);  // [b] P^T = -[b] A_r [b]
    o.C.xx = Cr.xx + 2.0 * N[0] + Q2[0];
    o.C.yy = Cr.yy + 2.0 * N[4] + Q2[4];
    o.C.zz = Cr.zz + 2.0 * N[8] + Q2[8];
    o.C.xy = Cr.xy + N[1] + N[3] + 0.5 * (Q2[1] + Q2[3]);
    o.C.xz = Cr.xz + N[2] + N[6] + 0.5 * (Q2[2] + Q2[6]);
    o.C.yz = Cr.yz + N[5] + N[7] + 0.5 * (Q2[5] + Q2[7]);
    return o;
}

// J about the joint-frame origin from (m, c, I_c): A = m I, B = -m[c],
// C = I_c + m (|c|^2 I - c c^T).
__device__ __forceinline__ Abi link_inertia(const double *Lc)
{
    const double m = Lc[12], cx = Lc[13], cy = Lc[14], cz = Lc[15];
    Abi J;
    J.A = Sym3d{m, m, m, 0.0, 0.0, 0.0};
    J.Bm[0] = 0.0;     J.Bm[1] = m * cz;  J.Bm[2] = -m * cy;
    J.Bm[3] = -m * cz; J.Bm[4] = 0.0;     J.Bm[5] = m * cx;
    J.Bm[6] = m * cy;  J.Bm[7] = -m * cx; J.Bm[8] = 0.0;
    const double c2 = cx * cx + cy * cy + cz * cz;
    J.C = Sym3d{Lc[16] + m * (c2 - cx * cx), Lc[17] + m * (c2 - cy * cy),
                Lc[18] + m * (c2 - cz * cz), Lc[19] - m * cx * cy, Lc[20] - m * cx * cz,
                Lc[21] - m * cy * cz};
    return J;
}

// Workspace addressing: element (link i, component k) of an instance sits at
// ws[(i * K + k) * stride + b]. A batch of one chain uses stride = B and the
// instance index b (component-major, coalesced across threads); a request of a
// fleet uses its own region with stride = 1, b = 0.
template <typename T>
__device__ __forceinline__ void aba_put(T *ws, int B, int b, int i, int k, T v)
{
    ws[((size_t)i * kAbaStateScalars + k) * (size_t)B + b] = v;
}

template <typename T>
__device__ __forceinline__ T aba_get(const T *ws, int B, int b, int i, int k)
{
    return ws[((size_t)i * kAbaStateScalars + k) * (size_t)B + b];
}

// solve-state area: U (6), c_hat, 1/Omega per link, component-major
constexpr int kAbaSolveScalars = 8;

template <typename Z>
__device__ __forceinline__ void aba_zput(Z *ws, int B, int b, int i, int k, Z v)
{
    ws[((size_t)i * kAbaSolveScalars + k) * (size_t)B + b] = v;
}

template <typename Z>
__device__ __forceinline__ Z aba_zget(const Z *ws, int B, int b, int i, int k)
{
    return ws[((size_t)i * kAbaSolveScalars + k) * (size_t)B + b];
}

// One forward-dynamics instance. sc / sd: the chain's constants (T and FP64,
// shared or global memory); qr, qdr, taur, qddr: its joint rows; ws / wsz and
// (B, b): its workspace (see aba_put). Returns 1 when an Omega_i <= 0 or a
// non-finite qdd appeared.
template <typename T, typename Z, bool VEC>
__device__ __forceinline__ int aba_instance(const T *sc, const double *sd, int n,
                                            const T *__restrict__ qr, const T *__restrict__ qdr,
                                            const T *__restrict__ taur, T *__restrict__ qddr,
                                            T *__restrict__ ws, Z *__restrict__ wsz, int B, int b,
                                            const BaseParams<T> &base)
{
    int bad = 0;

    // ---- sweep 1: bias motion (qdd = 0) and bias wrenches
    Motion<T> x;
    x.v = mk3(base.V0[0], base.V0[1], base.V0[2]);
    x.w = mk3(base.V0[3], base.V0[4], base.V0[5]);
    x.a = mk3(base.dV0[0], base.dV0[1], base.dV0[2]);
    x.al = mk3(base.dV0[3], base.dV0[4], base.dV0[5]);
    const int nchunks = (n + 3) / 4;
    for (int kc = 0; kc < nchunks; ++kc) {
        const int i0 = 4 * kc;
        const Chunk<T> cq = ld_chunk<T, VEC>(qr, i0, n), cqd = ld_chunk<T, VEC>(qdr, i0, n);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int i = i0 + j;
            if (VEC || i < n) {
                LinkC<T> L;
                load_link(sc + i * kLinkConsts, L);
                T s, c;
                sincos_t(cq.v[j], &s, &c);
                const Rot<T> R = make_rot(L.A, c, s);
                x = forward_step_R(R, mk3(L.b[0], L.b[1], L.b[2]), cqd.v[j], T(0), x);
                const Wrench<T> Fh = bias_wrench(L.m, mk3(L.c[0], L.c[1], L.c[2]), L.I, x);
                // slots 0-5: F_hat (replaced by U in sweep 2), 8-9: cos, sin
                const T vals[6] = {Fh.f.x, Fh.f.y, Fh.f.z, Fh.n.x, Fh.n.y, Fh.n.z};
#pragma unroll
                for (int k = 0; k < 6; ++k) aba_put(ws, B, b, i, k, vals[k]);
                aba_put(ws, B, b, i, 8, c);
                aba_put(ws, B, b, i, 9, s);
            }
        }
    }

    // ---- sweep 2: tau_hat, articulated inertias (FP64), z_hat, c_hat
    Wrench<T> F;
    F.f = mk3(base.Fn[0], base.Fn[1], base.Fn[2]);
    F.n = mk3(base.Fn[3], base.Fn[4], base.Fn[5]);
    Wrench<Z> z;
    z.f = z.n = mk3(Z(0), Z(0), Z(0));
    Rot<Z> RnZ;
    V3<Z> bnZ = mk3(Z(0), Z(0), Z(0));
    Abi Jh;
    double Uv[3] = {0, 0, 0}, Uw[3] = {0, 0, 0}, invOm = 0.0, chat = 0.0;
    Rot<T> Rn;
    V3<T> bn = mk3(T(0), T(0), T(0));
    double Rn64[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, bn64[3] = {0, 0, 0};
    const int last0 = ((n - 1) / 4) * 4;
    for (int i0 = last0; i0 >= 0; i0 -= 4) {
        const Chunk<T> ct = ld_chunk<T, VEC>(taur, i0, n);
#pragma unroll
        for (int j = 3; j >= 0; --j) {
            const int i = i0 + j;
            if (VEC || i < n) {
                Wrench<T> Fh;
                Fh.f = mk3(aba_get(ws, B, b, i, 0), aba_get(ws, B, b, i, 1), aba_get(ws, B, b, i, 2));
                Fh.n = mk3(aba_get(ws, B, b, i, 3), aba_get(ws, B, b, i, 4), aba_get(ws, B, b, i, 5));
                const T c = aba_get(ws, B, b, i, 8), s = aba_get(ws, B, b, i, 9);
                const double *L64 = sd + i * kLinkConsts;
                const T *Lt = sc + i * kLinkConsts;
                Abi Ji = link_inertia(L64);
                if (i == n - 1) {
                    F.f = add3(F.f, Fh.f);
                    F.n = add3(F.n, Fh.n);
                    Jh = Ji;
                } else {
                    F = carry_wrench_R(Rn, bn, F, Fh);
                    // M = J_hat_{i+1} - U U^T / Omega_{i+1}, then X^T M X + J_i
                    Abi M = Jh;
                    M.A.xx -= Uv[0] * Uv[0] * invOm; M.A.yy -= Uv[1] * Uv[1] * invOm;
                    M.A.zz -= Uv[2] * Uv[2] * invOm; M.A.xy -= Uv[0] * Uv[1] * invOm;
                    M.A.xz -= Uv[0] * Uv[2] * invOm; M.A.yz -= Uv[1] * Uv[2] * invOm;
#pragma unroll
                    for (int r = 0; r < 3; ++r)
#pragma unroll
                        for (int cc = 0; cc < 3; ++cc) M.Bm[3 * r + cc] -= Uv[r] * Uw[cc] * invOm;
                    M.C.xx -= Uw[0] * Uw[0] * invOm; M.C.yy -= Uw[1] * Uw[1] * invOm;
                    M.C.zz -= Uw[2] * Uw[2] * invOm; M.C.xy -= Uw[0] * Uw[1] * invOm;
                    M.C.xz -= Uw[0] * Uw[2] * invOm; M.C.yz -= Uw[1] * Uw[2] * invOm;
                    const Abi X = abi_congruence(M, Rn64, bn64);
                    Jh.A = Sym3d{Ji.A.xx + X.A.xx, Ji.A.yy + X.A.yy, Ji.A.zz + X.A.zz,
                                 Ji.A.xy + X.A.xy, Ji.A.xz + X.A.xz, Ji.A.yz + X.A.yz};
#pragma unroll
                    for (int k = 0; k < 9; ++k) Jh.Bm[k] = Ji.Bm[k] + X.Bm[k];
                    Jh.C = Sym3d{Ji.C.xx + X.C.xx, Ji.C.yy + X.C.yy, Ji.C.zz + X.C.zz,
                                 Ji.C.xy + X.C.xy, Ji.C.xz + X.C.xz, Ji.C.yz + X.C.yz};
                    // z_hat_i = X^T (z_hat_{i+1} + U_{i+1} c_hat_{i+1})
                    Wrench<Z> zz;
                    zz.f = mk3(z.f.x + (Z)(Uv[0] * chat), z.f.y + (Z)(Uv[1] * chat), z.f.z + (Z)(Uv[2] * chat));
                    zz.n = mk3(z.n.x + (Z)(Uw[0] * chat), z.n.y + (Z)(Uw[1] * chat), z.n.z + (Z)(Uw[2] * chat));
                    Wrench<Z> zero;
                    zero.f = zero.n = mk3(Z(0), Z(0), Z(0));
                    z = carry_wrench_R(RnZ, bnZ, zz, zero);
                }
                const double tau_hat = (double)ct.v[j] - (double)F.n.z;
                // U_i = J_hat_i S (last column), Omega_i = its w_z entry
                Uv[0] = Jh.Bm[2]; Uv[1] = Jh.Bm[5]; Uv[2] = Jh.Bm[8];
                Uw[0] = Jh.C.xz; Uw[1] = Jh.C.yz; Uw[2] = Jh.C.zz;
                const double Om = Jh.C.zz;
                if (!(Om > 0.0)) bad = 1;
                invOm = 1.0 / Om;
                chat = (tau_hat - (double)z.n.z) * invOm;
                const Z vals[8] = {(Z)Uv[0], (Z)Uv[1], (Z)Uv[2], (Z)Uw[0], (Z)Uw[1], (Z)Uw[2],
                                   (Z)chat, (Z)invOm};
#pragma unroll
                for (int k = 0; k < 8; ++k) aba_zput(wsz, B, b, i, k, vals[k]);
                // transform of link i, for the step to link i-1
                Rn = make_rot(Lt, c, s);
                bn = mk3(Lt[9], Lt[10], Lt[11]);
                const double cd = (double)c, sd_ = (double)s;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    Rn64[3 * k + 0] = fma(cd, L64[3 * k + 0], sd_ * L64[3 * k + 1]);
                    Rn64[3 * k + 1] = fma(cd, L64[3 * k + 1], -sd_ * L64[3 * k + 0]);
                    Rn64[3 * k + 2] = L64[3 * k + 2];
                }
                bn64[0] = L64[9]; bn64[1] = L64[10]; bn64[2] = L64[11];
                if constexpr (sizeof(Z) == 8) {
#pragma unroll
                    for (int k = 0; k < 9; ++k) RnZ.r[k] = (Z)Rn64[k];
                    bnZ = mk3((Z)bn64[0], (Z)bn64[1], (Z)bn64[2]);
                } else {
#pragma unroll
                    for (int k = 0; k < 9; ++k) RnZ.r[k] = (Z)Rn.r[k];
                    bnZ = mk3((Z)bn.x, (Z)bn.y, (Z)bn.z);
                }
            }
        }
    }

    // ---- sweep 3: lambda and qdd
    V3<Z> lv = mk3(Z(0), Z(0), Z(0)), lw = mk3(Z(0), Z(0), Z(0));
    for (int kc = 0; kc < nchunks; ++kc) {
        const int i0 = 4 * kc;
        Chunk<T> out;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int i = i0 + j;
            out.v[j] = T(0);
            if (VEC || i < n) {
                const T c = aba_get(ws, B, b, i, 8), s = aba_get(ws, B, b, i, 9);
                Rot<Z> R;
                V3<Z> bi;
                if constexpr (sizeof(Z) == 8) {
                    const double *L64 = sd + i * kLinkConsts;
                    R = make_rot(L64, (double)c, (double)s);
                    bi = mk3(L64[9], L64[10], L64[11]);
                } else {
                    const T *Lt = sc + i * kLinkConsts;
                    R = make_rot(Lt, c, s);
                    bi = mk3(Lt[9], Lt[10], Lt[11]);
                }
                // a = Ad_{f^-1} lambda
                const V3<Z> t = cross_add(lw, bi, lv);
                V3<Z> av = mulAT(R.r, t), aw = mulAT(R.r, lw);
                const V3<Z> uv = mk3(aba_zget(wsz, B, b, i, 0), aba_zget(wsz, B, b, i, 1), aba_zget(wsz, B, b, i, 2));
                const V3<Z> uw = mk3(aba_zget(wsz, B, b, i, 3), aba_zget(wsz, B, b, i, 4), aba_zget(wsz, B, b, i, 5));
                const Z ch = aba_zget(wsz, B, b, i, 6), iom = aba_zget(wsz, B, b, i, 7);
                const double ua = (double)uv.x * av.x + (double)uv.y * av.y + (double)uv.z * av.z +
                                  (double)uw.x * aw.x + (double)uw.y * aw.y + (double)uw.z * aw.z;
                const double qdd_i = (double)ch - (double)iom * ua;
                aw.z += (Z)qdd_i;
                lv = av;
                lw = aw;
                out.v[j] = (T)qdd_i;
                if (!(qdd_i == qdd_i)) bad = 1;
            }
        }
        st_chunk<T, VEC>(qddr, i0, n, out);
    }
    return bad;
}


// Shared memory: n * 24 constants in T, then n * 24 in FP64.
// Z: arithmetic of the z_hat / lambda recursions and storage of U, c_hat,
// 1/Omega (double by default; T when the caller asks for the spatial scans in
// the data precision).
template <typename T, typename Z, int BLOCK, bool VEC>
__global__ void __launch_bounds__(BLOCK)
aba_kernel(const T *__restrict__ consts, const double *__restrict__ consts64, int n, int B,
           const T *__restrict__ q, const T *__restrict__ qd, const T *__restrict__ tau,
           T *__restrict__ qdd_out, int *__restrict__ status, T *__restrict__ ws,
           Z *__restrict__ wsz, BaseParams<T> base)
{
    extern __shared__ __align__(16) unsigned char smem[];
    T *sc = reinterpret_cast<T *>(smem);
    double *sd = reinterpret_cast<double *>(smem + (((size_t)n * kLinkConsts * sizeof(T) + 15) & ~(size_t)15));
    const int nc = n * kLinkConsts;
    for (int k = threadIdx.x; k < nc; k += BLOCK) {
        sc[k] = consts[k];
        sd[k] = consts64[k];
    }
    __syncthreads();

    const int b = blockIdx.x * BLOCK + threadIdx.x;
    if (b >= B) return;
    const size_t row = (size_t)b * (size_t)n;
    const int bad = aba_instance<T, Z, VEC>(sc, sd, n, q + row, qd + row, tau + row, qdd_out + row,
                                            ws, wsz, B, b, base);
    if (status) status[b] = bad ? RD_WARN_SINGULAR : 0;
}

}  // namespace rdyn
