// aba_warp.cuh -- forward dynamics with one warp per instance, for batches too
// small to fill the GPU with one thread per instance.
//
// The articulated-body algorithm (Sec. II-B) in the form of Sec. III-D:
//   1. tau_bias = ID(q, qd, 0, ...) by the two scans of inverse dynamics
//      (Sec. III-B/C) across the 32 lanes, K = ceil(n / 32) links per lane:
//      segment elements, Kogge-Stone combines with shuffles, replays (as
//      rnea_scan.cuh, here in common-normal frames); tau_hat = tau - tau_bias.
//   2. The articulated inertias, Eq. (abi): a nonlinear recursion that no scan
//      speeds up, so it runs link by link, tip to base. Each link's update
//          J_hat_i = J_i + X^T (J_hat_{i+1} - U U^T / Omega) X
//      is spread over the warp instead: lane e of 21 owns the entry (a, b),
//      a <= b, and forms x_a^T P x_b with x_a = X e_a, after gathering the 21
//      entries of J_hat_{i+1} with shuffles. Every lane runs the same
//      instructions (no divergence); the entries differ only in data.
//   3. Eq. (fd-bkwd-scan): z_hat / c_hat as a backward scan of affine maps
//      z -> M z + v over the lanes' segments (suffix combine, replay), then
//      Eq. (fd-fwd-scan): lambda / qdd as a forward scan of lambda -> N lambda +
//      u (prefix combine, replay). The operands, their bracketings and this
//      segmented form are checked against the oracle on the host.
// State between the phases (per link: cos, sin, tau_hat, U, 1 / Omega) lives in
// shared memory, one slice per warp. D: double-float (FP32 data) or double;
// TB: precision of phase 1 and of the joint sin/cos (T, or DF for chains
// beyond RD_ABA_EXTENDED_BIAS_LINKS).
#pragma once
#include <type_traits>

#include "aba_dh.cuh"
#include "rdyn_internal.h"
#include "rnea_scan.cuh"

namespace rdyn {

// ---- shuffles of double-float pairs (the scalar ones are in rnea_scan.cuh).
// They sit in the pair's namespace so that the templates of rnea_scan.cuh find
// them by argument-dependent lookup.
namespace dfloat {
__device__ __forceinline__ DF shup(DF v, int d, int L)
{
    return DF(__shfl_up_sync(0xffffffffu, v.hi, d, L), __shfl_up_sync(0xffffffffu, v.lo, d, L));
}
__device__ __forceinline__ DF shdn(DF v, int d, int L)
{
    return DF(__shfl_down_sync(0xffffffffu, v.hi, d, L),
              __shfl_down_sync(0xffffffffu, v.lo, d, L));
}
}  // namespace dfloat
template <typename D>
__device__ __forceinline__ D shidx(D v, int src)
{
    if constexpr (std::is_same<D, DF>::value)
        return DF(__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src));
    else
        return __shfl_sync(0xffffffffu, v, src);
}

// lane-uniform select of a pair
template <typename D>
__device__ __forceinline__ D dsel(bool c, D a, D b)
{
    if constexpr (std::is_same<D, DF>::value) return DF(c ? a.hi : b.hi, c ? a.lo : b.lo);
    else return c ? a : b;
}

// R = Rx(alpha) Rz(theta) as a full row-major rotation
template <typename T>
__device__ __forceinline__ Rot<T> dh_full_rot(T ca, T sa, T c, T s)
{
    Rot<T> R;
    R.r[0] = c;      R.r[1] = -s;     R.r[2] = T(0.0f);
    R.r[3] = ca * s; R.r[4] = ca * c; R.r[5] = -sa;
    R.r[6] = sa * s; R.r[7] = sa * c; R.r[8] = ca;
    return R;
}

// The 21 entries (a, b), a <= b, of a symmetric 6x6 in twist order (v, w),
// one per lane; lanes 21..31 repeat (5, 5) and store nothing.
constexpr int kAbiEntries = 21;
__host__ __device__ constexpr int abi_row(int e)
{
    return e < 6 ? 0 : e < 11 ? 1 : e < 15 ? 2 : e < 18 ? 3 : e < 20 ? 4 : 5;
}
__host__ __device__ constexpr int abi_col(int e)
{
    return e < 6 ? e : e < 11 ? e - 5 : e < 15 ? e - 9 : e < 18 ? e - 12 : e < 20 ? e - 14 : 5;
}
// lane of entry (k, l), either order
__host__ __device__ constexpr int abi_lane(int k, int l)
{
    const int a = k < l ? k : l, b = k < l ? l : k;
    return a == 0 ? b : a == 1 ? 5 + b : a == 2 ? 9 + b : a == 3 ? 12 + b : a == 4 ? 14 + b : 20;
}
// J_i about the frame origin, entry by entry, from the record of aba_dh.cuh:
// A = m I, Bm = -[m c], C = C_o. Index into the record and sign (0: zero).
__host__ __device__ constexpr int abi_j_index(int e)
{
    // (0,0) m; (0,4) mcz; (0,5) mcy; (1,1) m; (1,3) mcz; (1,5) mcx; (2,2) m;
    // (2,3) mcy; (2,4) mcx; (3,3) Cxx; (3,4) Cxy; (3,5) Cxz; (4,4) Cyy; (4,5) Cyz;
    // (5,5) Czz
    return e == 0 ? 6 : e == 4 ? 18 : e == 5 ? 17 : e == 6 ? 6 : e == 8 ? 18 : e == 10 ? 16
         : e == 11 ? 6 : e == 12 ? 17 : e == 13 ? 16 : e == 15 ? 19 : e == 16 ? 22
         : e == 17 ? 23 : e == 18 ? 20 : e == 19 ? 24 : e == 20 ? 21 : 6;
}
__host__ __device__ constexpr int abi_j_sign(int e)
{
    return (e == 0 || e == 4 || e == 6 || e == 10 || e == 11 || e == 12 || e >= 15) ? 1
         : (e == 5 || e == 8 || e == 13) ? -1 : 0;
}

// Per-warp shared state, per link k: cos, sin (D), tau_hat, U (6), 1 / Omega.
template <typename D>
struct AbaWarpLink {
    D c, s, that, u[6], iom;
};

// ---- phase 1: tau_bias by lane scans in common-normal frames (precision TB).
// Lane l owns links [l K, l K + K). Writes cos, sin and tau_hat = tau - tau_bias
// of its links to the warp's shared state.
template <typename T, typename D, typename TB, int K>
__device__ __forceinline__ void aba_warp_bias(const T *__restrict__ sc, const DF *__restrict__ sdf,
                                              int n, const T *__restrict__ qr,
                                              const T *__restrict__ qdr,
                                              const T *__restrict__ taur,
                                              const BaseParams<T> &base, AbaWarpLink<D> *st)
{
    constexpr bool kExt = !std::is_same<TB, T>::value;
    constexpr int L = 32;
    const int l = threadIdx.x & 31;
    const int s0 = l * K;
    const TB zero = dcvt<TB>(T(0));

    // link data of the segment
    TB jc[K], js[K], jqd[K];
    auto consts = [&](int i, TB &ca, TB &sa, V3<TB> &b) {
        if constexpr (kExt) {
            const DF *r = sdf + i * kAbaDh64;
            ca = r[0]; sa = r[1]; b = mk3(r[2], r[3], r[4]);
        } else {
            const T *p = sc + i * kDhConsts;
            ca = p[0]; sa = p[1]; b = mk3(p[2], p[3], p[4]);
        }
    };
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int i = s0 + j;
        jc[j] = dcvt<TB>(T(1)); js[j] = zero; jqd[j] = zero;
        if (i < n) {
            const T qi = __ldg(qr + i);
            jqd[j] = dcvt<TB>(__ldg(qdr + i));
            if constexpr (kExt) {
                df_sincos((double)qi + df_to_double(sdf[i * kAbaDh64 + 5]), &js[j], &jc[j]);
            } else {
                dh_trig<T, kTrigPoly>(qi + sc[i * kDhConsts + 5], &js[j], &jc[j]);
            }
        }
    }
    Motion<TB> xb;
    xb.v = mk3(dcvt<TB>(base.V0[0]), dcvt<TB>(base.V0[1]), dcvt<TB>(base.V0[2]));
    xb.w = mk3(dcvt<TB>(base.V0[3]), dcvt<TB>(base.V0[4]), dcvt<TB>(base.V0[5]));
    xb.a = mk3(dcvt<TB>(base.dV0[0]), dcvt<TB>(base.dV0[1]), dcvt<TB>(base.dV0[2]));
    xb.al = mk3(dcvt<TB>(base.dV0[3]), dcvt<TB>(base.dV0[4]), dcvt<TB>(base.dV0[5]));

    // forward: segment element from a zero state (lane 0: from the base state)
    FwdElem<TB> E;
    E.G = rigid_identity<TB>();
    if (l == 0) E.x = xb;
    else E.x.v = E.x.w = E.x.a = E.x.al = mk3(zero, zero, zero);
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int i = s0 + j;
        if (i < n) {
            TB ca, sa;
            V3<TB> b;
            consts(i, ca, sa, b);
            E.x = dh_forward(dh_rot(ca, sa, jc[j], js[j]), b, jqd[j], zero, E.x);
            E.G = premul_ginv(dh_full_rot(ca, sa, jc[j], js[j]), b, E.G);
        }
    }
#pragma unroll
    for (int d = 1; d < L; d <<= 1) {
        FwdElem<TB> Y;
        Y.G = shup_rigid(E.G, d, L);
        Y.x.v = shup3(E.x.v, d, L);
        Y.x.w = shup3(E.x.w, d, L);
        Y.x.a = shup3(E.x.a, d, L);
        Y.x.al = shup3(E.x.al, d, L);
        if (l >= d) E = fwd_combine(E, Y);
    }
    Motion<TB> x;
    x.v = shup3(E.x.v, 1, L);
    x.w = shup3(E.x.w, 1, L);
    x.a = shup3(E.x.a, 1, L);
    x.al = shup3(E.x.al, 1, L);
    if (l == 0) x = xb;
    Wrench<TB> Fh[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int i = s0 + j;
        Fh[j].f = Fh[j].n = mk3(zero, zero, zero);
        if (i < n) {
            TB ca, sa, m;
            V3<TB> b, cm;
            TB I[6];
            if constexpr (kExt) {
                const DF *r = sdf + i * kAbaDh64;
                ca = r[0]; sa = r[1]; b = mk3(r[2], r[3], r[4]);
                m = r[6]; cm = mk3(r[7], r[8], r[9]);
#pragma unroll
                for (int k = 0; k < 6; ++k) I[k] = r[10 + k];
            } else {
                DhLink<T> Lk;
                load_dh(sc + i * kDhConsts, Lk);
                ca = Lk.ca; sa = Lk.sa; b = Lk.b; m = Lk.m; cm = Lk.c;
#pragma unroll
                for (int k = 0; k < 6; ++k) I[k] = Lk.I[k];
            }
            x = dh_forward(dh_rot(ca, sa, jc[j], js[j]), b, jqd[j], zero, x);
            Fh[j] = bias_wrench(m, cm, I, x);
        }
    }

    // backward: element (H, b) of the segment, F_s = Ad^T_H F_e + b
    const TB c_up = shdn(jc[0], 1, L), s_up = shdn(js[0], 1, L);
    const int e = s0 + K;
    const bool tip_lane = (s0 < n) && (e >= n);
    BwdElem<TB> Bk;
    Bk.H = rigid_identity<TB>();
    Bk.b.f = Bk.b.n = mk3(zero, zero, zero);
    if (tip_lane) {
        Bk.b.f = mk3(dcvt<TB>(base.Fn[0]), dcvt<TB>(base.Fn[1]), dcvt<TB>(base.Fn[2]));
        Bk.b.n = mk3(dcvt<TB>(base.Fn[3]), dcvt<TB>(base.Fn[4]), dcvt<TB>(base.Fn[5]));
    }
    DhRot<TB> Rup = dh_rot(dcvt<TB>(T(1)), zero, dcvt<TB>(T(1)), zero);
    V3<TB> bup = mk3(zero, zero, zero);
    if (s0 < n && !tip_lane) {
        TB ca, sa;
        consts(e, ca, sa, bup);
        Rup = dh_rot(ca, sa, c_up, s_up);
        // H = g_e = (R^T, -R^T b)
        const Rot<TB> Rf = dh_full_rot(ca, sa, c_up, s_up);
#pragma unroll
        for (int k = 0; k < 9; ++k) Bk.H.R.r[k] = Rf.r[3 * (k % 3) + k / 3];
        Bk.H.p = dh_mulT(Rup, mk3(-bup.x, -bup.y, -bup.z));
    }
    if (s0 < n) {
        DhRot<TB> Rn = Rup;
        V3<TB> bn = bup;
        TB can = zero, san = zero;
        if (!tip_lane) consts(e, can, san, bn);
        Rot<TB> Rnf = dh_full_rot(can, san, c_up, s_up);
#pragma unroll
        for (int j = K - 1; j >= 0; --j) {
            const int i = s0 + j;
            if (i < n) {
                if (i == n - 1 || i == e - 1) {
                    Bk.b.f = add3(Bk.b.f, Fh[j].f);
                    Bk.b.n = add3(Bk.b.n, Fh[j].n);
                } else {
                    Bk.b = dh_carry(Rn, bn, Bk.b, Fh[j]);
                    Bk.H = postmul_ginv(Bk.H, Rnf, bn);
                }
                TB ca, sa;
                consts(i, ca, sa, bn);
                Rn = dh_rot(ca, sa, jc[j], js[j]);
                Rnf = dh_full_rot(ca, sa, jc[j], js[j]);
            }
        }
    }
#pragma unroll
    for (int d = 1; d < L; d <<= 1) {
        BwdElem<TB> Y;
        Y.H = shdn_rigid(Bk.H, d, L);
        Y.b.f = shdn3(Bk.b.f, d, L);
        Y.b.n = shdn3(Bk.b.n, d, L);
        if (l + d < L) Bk = bwd_combine(Bk, Y);
    }
    Wrench<TB> F;
    F.f = shdn3(Bk.b.f, 1, L);
    F.n = shdn3(Bk.b.n, 1, L);
    if (tip_lane) {
        F.f = mk3(dcvt<TB>(base.Fn[0]), dcvt<TB>(base.Fn[1]), dcvt<TB>(base.Fn[2]));
        F.n = mk3(dcvt<TB>(base.Fn[3]), dcvt<TB>(base.Fn[4]), dcvt<TB>(base.Fn[5]));
    }
    if (s0 < n) {
        DhRot<TB> Rn = Rup;
        V3<TB> bn = bup;
#pragma unroll
        for (int j = K - 1; j >= 0; --j) {
            const int i = s0 + j;
            if (i < n) {
                if (i == n - 1) {
                    F.f = add3(F.f, Fh[j].f);
                    F.n = add3(F.n, Fh[j].n);
                } else {
                    F = dh_carry(Rn, bn, F, Fh[j]);
                }
                const T ti = __ldg(taur + i);
                AbaWarpLink<D> &sl = st[i];
                if constexpr (kExt) sl.that = dcvt<D>(DF(ti) - F.n.z);
                else sl.that = dsub_exact<D>(ti, F.n.z);
                sl.c = dcvt<D>(jc[j]);
                sl.s = dcvt<D>(js[j]);
                TB ca, sa;
                consts(i, ca, sa, bn);
                Rn = dh_rot(ca, sa, jc[j], js[j]);
            }
        }
    }
}

// ---- phase 2: the articulated inertias, Eq. (abi), tip to base. Lane e < 21
// holds entry (a, b) of J_hat_i. Each link gathers all 21 by shuffles, records
// U_i = J_hat_i S_i and 1 / Omega_i, forms P = J_hat_i - U U^T / Omega_i (zero
// w_z row and column, so a 5 x 5 block) and its own entry of
//     J_hat_{i-1} = J_{i-1} + X^T P X,   X = Ad_{f_{i-1,i}^-1},
// as x_a^T (P x_b) with x_a = X e_a: for a < 3, (row a of R, 0); for a >= 3,
// (R^T (e_{a-3} x b), row a-3 of R), R = Rx(alpha_i) Rz(theta_i) and b_i.
// Returns true on every lane when an Omega_i <= 0 (or is not a number).
template <typename D>
__device__ __forceinline__ bool aba_warp_abi(const D *__restrict__ sd, int n, AbaWarpLink<D> *st)
{
    const int lane = threadIdx.x & 31;
    const int e = lane < kAbiEntries ? lane : kAbiEntries - 1;
    const int a = abi_row(e), bcol = abi_col(e);
    const int jidx = abi_j_index(e), jsgn = abi_j_sign(e);
    const D zero = dcvt<D>(0.0f);
    auto jentry = [&](int i) -> D {
        const D v = sd[i * kAbaDh64 + jidx];
        return jsgn > 0 ? v : jsgn < 0 ? -v : zero;
    };
    // x_k = X e_k from the rows of R and b
    auto column = [&](const D R[9], const D b[3], int k, D x[6]) {
        const int r = k < 3 ? k : k - 3;
        const D r0 = dsel(r == 0, R[0], dsel(r == 1, R[3], R[6]));
        const D r1 = dsel(r == 0, R[1], dsel(r == 1, R[4], R[7]));
        const D r2 = dsel(r == 0, R[2], dsel(r == 1, R[5], R[8]));
        // u = e_r x b
        const D u0 = dsel(r == 0, zero, dsel(r == 1, b[2], -b[1]));
        const D u1 = dsel(r == 0, -b[2], dsel(r == 1, zero, b[0]));
        const D u2 = dsel(r == 0, b[1], dsel(r == 1, -b[0], zero));
        const D t0 = fma(R[0], u0, fma(R[3], u1, R[6] * u2));
        const D t1 = fma(R[1], u0, fma(R[4], u1, R[7] * u2));
        const D t2 = fma(R[2], u0, fma(R[5], u1, R[8] * u2));
        const bool lin = k < 3;
        x[0] = dsel(lin, r0, t0);
        x[1] = dsel(lin, r1, t1);
        x[2] = dsel(lin, r2, t2);
        x[3] = dsel(lin, zero, r0);
        x[4] = dsel(lin, zero, r1);
        x[5] = dsel(lin, zero, r2);
    };
    bool bad = false;
    D own = jentry(n - 1);  // entry of J_hat_{n-1} = J_{n-1}
#pragma unroll 1
    for (int i = n - 1;; --i) {
        D jj[kAbiEntries];
#pragma unroll
        for (int k = 0; k < kAbiEntries; ++k) jj[k] = shidx(own, k);
        const D Om = jj[abi_lane(5, 5)];
        if (!dpositive(Om)) bad = true;
        const D iom = drecip(Om);
        D U[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) U[k] = jj[abi_lane(k, 5)];
        if (lane < 6) {
            D u = U[0];
#pragma unroll
            for (int k = 1; k < 6; ++k) u = dsel(lane == k, U[k], u);
            st[i].u[lane] = u;
        }
        if (lane == 6) st[i].iom = iom;
        if (i == 0) break;
        // J_hat_{i-1}: X is the transform of link i
        const D *ri = sd + i * kAbaDh64;
        const DhRot<D> Rd = dh_rot(ri[0], ri[1], st[i].c, st[i].s);
        const D R[9] = {Rd.c, -Rd.s, zero, Rd.sca, Rd.cca, -Rd.sa, Rd.ssa, Rd.csa, Rd.ca};
        const D bv[3] = {ri[2], ri[3], ri[4]};
        D xa[6], xb[6];
        column(R, bv, a, xa);
        column(R, bv, bcol, xb);
        D w[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) w[k] = U[k] * iom;
        D r = jentry(i - 1);
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            D y = zero;
#pragma unroll
            for (int m = 0; m < 5; ++m) y = fma(fma(-w[k], U[m], jj[abi_lane(k, m)]), xb[m], y);
            r = fma(xa[k], y, r);
        }
        own = r;
    }
    return __any_sync(0xffffffffu, bad);
}

// X_k^T z for a wrench-like z = (f, n): (R f, b x (R f) + R n)
template <typename D>
__device__ __forceinline__ void xt_apply(const DhRot<D> &R, const V3<D> &b, D z[6])
{
    const V3<D> f = dh_mul(R, mk3(z[0], z[1], z[2]));
    const V3<D> m = cross_add(b, f, dh_mul(R, mk3(z[3], z[4], z[5])));
    z[0] = f.x; z[1] = f.y; z[2] = f.z; z[3] = m.x; z[4] = m.y; z[5] = m.z;
}

// X_k x for a motion x = (v, w): (R^T (v + w x b), R^T w)
template <typename D>
__device__ __forceinline__ void x_apply(const DhRot<D> &R, const V3<D> &b, D x[6])
{
    const V3<D> w = mk3(x[3], x[4], x[5]);
    const V3<D> v = dh_mulT(R, cross_add(w, b, mk3(x[0], x[1], x[2])));
    const V3<D> ww = dh_mulT(R, w);
    x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = ww.x; x[4] = ww.y; x[5] = ww.z;
}

// (M, v) <- (M M', M v' + v) for 6 x 6 M (row-major) and 6-vectors
template <typename D>
__device__ __forceinline__ void affine_compose(D M[36], D v[6], const D Mp[36], const D vp[6])
{
    D R[36], rv[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            D acc = M[6 * i] * Mp[j];
#pragma unroll
            for (int k = 1; k < 6; ++k) acc = fma(M[6 * i + k], Mp[6 * k + j], acc);
            R[6 * i + j] = acc;
        }
        D acc = v[i];
#pragma unroll
        for (int k = 0; k < 6; ++k) acc = fma(M[6 * i + k], vp[k], acc);
        rv[i] = acc;
    }
#pragma unroll
    for (int k = 0; k < 36; ++k) M[k] = R[k];
#pragma unroll
    for (int k = 0; k < 6; ++k) v[k] = rv[k];
}

// ---- phase 3: Eq. (fd-bkwd-scan) then Eq. (fd-fwd-scan) as scans of affine
// maps over the lanes' segments. Backward, link k maps z_k to
//     z_{k-1} = X_k^T (z_k + U_k c_k),  c_k = (tau_hat_k - S_k^T z_k) / Omega_k,
// from z_{n-1} = 0; forward, with a_k = X_k lambda_{k-1},
//     qdd_k = c_k - U_k^T a_k / Omega_k,  lambda_k = a_k + S_k qdd_k,
// from lambda_{-1} = 0. Writes qdd; returns true if any is not a number.
template <typename T, typename D, int K>
__device__ __forceinline__ bool aba_warp_solve(const D *__restrict__ sd, int n,
                                               const AbaWarpLink<D> *st, T *__restrict__ qddr)
{
    constexpr int L = 32;
    const int l = threadIdx.x & 31;
    const int s0 = l * K;
    const D zero = dcvt<D>(0.0f), one = dcvt<D>(1.0f);
    auto xform = [&](int k, DhRot<D> &R, V3<D> &b) {
        const D *r = sd + k * kAbaDh64;
        R = dh_rot(r[0], r[1], st[k].c, st[k].s);
        b = mk3(r[2], r[3], r[4]);
    };

    // backward: (M, v) of the segment, z_{s0-1} = M z_{e-1} + v
    D M[36], v[6];
#pragma unroll
    for (int k = 0; k < 36; ++k) M[k] = (k % 7 == 0) ? one : zero;
#pragma unroll
    for (int k = 0; k < 6; ++k) v[k] = zero;
#pragma unroll
    for (int j = K - 1; j >= 0; --j) {
        const int k = s0 + j;
        if (k < n) {
            DhRot<D> R;
            V3<D> b;
            xform(k, R, b);
            const AbaWarpLink<D> &sk = st[k];
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                D z[6];
                const D t = -(M[30 + c] * sk.iom);
#pragma unroll
                for (int r = 0; r < 6; ++r) z[r] = fma(sk.u[r], t, M[6 * r + c]);
                xt_apply(R, b, z);
#pragma unroll
                for (int r = 0; r < 6; ++r) M[6 * r + c] = z[r];
            }
            const D t = (sk.that - v[5]) * sk.iom;
#pragma unroll
            for (int r = 0; r < 6; ++r) v[r] = fma(sk.u[r], t, v[r]);
            xt_apply(R, b, v);
        }
    }
    // inclusive suffix combine, lower o upper
#pragma unroll
    for (int d = 1; d < L; d <<= 1) {
        D Mp[36], vp[6];
#pragma unroll
        for (int k = 0; k < 36; ++k) Mp[k] = shdn(M[k], d, L);
#pragma unroll
        for (int k = 0; k < 6; ++k) vp[k] = shdn(v[k], d, L);
        if (l + d < L) affine_compose(M, v, Mp, vp);
    }
    // z entering from above: the next lane's suffix applied to z_{n-1} = 0
    D z[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const D t = shdn(v[k], 1, L);
        z[k] = l + 1 < L ? t : zero;
    }
    D ch[K];
#pragma unroll
    for (int j = K - 1; j >= 0; --j) {
        const int k = s0 + j;
        ch[j] = zero;
        if (k < n) {
            DhRot<D> R;
            V3<D> b;
            xform(k, R, b);
            const AbaWarpLink<D> &sk = st[k];
            ch[j] = (sk.that - z[5]) * sk.iom;
#pragma unroll
            for (int r = 0; r < 6; ++r) z[r] = fma(sk.u[r], ch[j], z[r]);
            xt_apply(R, b, z);
        }
    }

    // forward: (N, u) of the segment, lambda_{e-1} = N lambda_{s0-1} + u
    D N[36], u[6];
#pragma unroll
    for (int k = 0; k < 36; ++k) N[k] = (k % 7 == 0) ? one : zero;
#pragma unroll
    for (int k = 0; k < 6; ++k) u[k] = zero;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int k = s0 + j;
        if (k < n) {
            DhRot<D> R;
            V3<D> b;
            xform(k, R, b);
            const AbaWarpLink<D> &sk = st[k];
#pragma unroll
            for (int c = 0; c < 7; ++c) {
                D x[6];
#pragma unroll
                for (int r = 0; r < 6; ++r) x[r] = c < 6 ? N[6 * r + c] : u[r];
                x_apply(R, b, x);
                D ua = sk.u[0] * x[0];
#pragma unroll
                for (int r = 1; r < 6; ++r) ua = fma(sk.u[r], x[r], ua);
                x[5] = fma(-sk.iom, ua, x[5]);
                if (c == 6) x[5] = x[5] + ch[j];
#pragma unroll
                for (int r = 0; r < 6; ++r) {
                    if (c < 6) N[6 * r + c] = x[r];
                    else u[r] = x[r];
                }
            }
        }
    }
    // inclusive prefix combine, later o earlier
#pragma unroll
    for (int d = 1; d < L; d <<= 1) {
        D Np[36], up[6];
#pragma unroll
        for (int k = 0; k < 36; ++k) Np[k] = shup(N[k], d, L);
#pragma unroll
        for (int k = 0; k < 6; ++k) up[k] = shup(u[k], d, L);
        if (l >= d) affine_compose(N, u, Np, up);
    }
    D lam[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const D t = shup(u[k], 1, L);
        lam[k] = l > 0 ? t : zero;
    }
    bool nan = false;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int k = s0 + j;
        if (k < n) {
            DhRot<D> R;
            V3<D> b;
            xform(k, R, b);
            const AbaWarpLink<D> &sk = st[k];
            x_apply(R, b, lam);
            D ua = sk.u[0] * lam[0];
#pragma unroll
            for (int r = 1; r < 6; ++r) ua = fma(sk.u[r], lam[r], ua);
            const D q = fma(-sk.iom, ua, ch[j]);
            lam[5] = lam[5] + q;
            if (disnan(q)) nan = true;
            qddr[k] = dcvt<T>(q);
        }
    }
    return __any_sync(0xffffffffu, nan);
}

// One warp per instance, WARPS instances per block; shared memory holds
// n AbaWarpLink<D> per warp.
template <typename T, typename D, typename TB, int K, int WARPS>
__global__ void __launch_bounds__(32 * WARPS)
aba_warp_kernel(const T *__restrict__ sc, const D *__restrict__ sd, const DF *__restrict__ sdf,
                int n, int B, const T *__restrict__ q, const T *__restrict__ qd,
                const T *__restrict__ tau, T *__restrict__ qdd_out, int *__restrict__ status,
                BaseParams<T> base)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5;
    const int inst = blockIdx.x * WARPS + warp;
    if (inst >= B) return;  // whole warps leave together
    AbaWarpLink<D> *st = reinterpret_cast<AbaWarpLink<D> *>(smem) + (size_t)warp * n;
    const size_t row = (size_t)inst * (size_t)n;
    aba_warp_bias<T, D, TB, K>(sc, sdf, n, q + row, qd + row, tau + row, base, st);
    __syncwarp();
    const bool bad = aba_warp_abi<D>(sd, n, st);
    __syncwarp();
    const bool nan = aba_warp_solve<T, D, K>(sd, n, st, qdd_out + row);
    if (status && (threadIdx.x & 31) == 0) status[inst] = (bad || nan) ? RD_WARN_SINGULAR : 0;
}

// One warp per instance: 4 instances per block, K links per lane.
template <typename T, typename D, typename TB, int K>
int launch_aba_warp_k(const rd_model *m, int B, const void *q, const void *qd, const void *tau,
                      void *qdd, int *status, const double *base18, cudaStream_t stream)
{
    constexpr int WARPS = 4;
    const int n = m->n;
    double bb[18];
    rd_convert_base_dh(m, base18, bb);
    BaseParams<T> bp;
    for (int k = 0; k < 6; ++k) {
        bp.V0[k] = (T)bb[k];
        bp.dV0[k] = (T)bb[6 + k];
        bp.Fn[k] = (T)bb[12 + k];
    }
    const T *sc = nullptr;
    if constexpr (sizeof(T) == 4) sc = reinterpret_cast<const T *>(m->d_dh32);
    else sc = reinterpret_cast<const T *>(m->d_dh64);
    const D *sd = nullptr;
    if constexpr (std::is_same<D, double>::value) sd = m->d_aba64;
    else sd = reinterpret_cast<const D *>(m->d_abadf);
    const DF *sdf = reinterpret_cast<const DF *>(m->d_abadf);
    const size_t smem = (size_t)WARPS * n * sizeof(AbaWarpLink<D>);
    const unsigned grid = (unsigned)((B + WARPS - 1) / WARPS);
    aba_warp_kernel<T, D, TB, K, WARPS><<<grid, 32 * WARPS, smem, stream>>>(
        sc, sd, sdf, n, B, static_cast<const T *>(q), static_cast<const T *>(qd),
        static_cast<const T *>(tau), static_cast<T *>(qdd), status, bp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return rd_cuda_fail(e, "aba warp-per-instance kernel launch");
    return RD_OK;
}

template <typename T, typename D, typename TB>
int launch_aba_warp(const rd_model *m, int B, const void *q, const void *qd, const void *tau,
                    void *qdd, int *status, const double *base18, cudaStream_t s)
{
    if (m->n <= 32) return launch_aba_warp_k<T, D, TB, 1>(m, B, q, qd, tau, qdd, status, base18, s);
    if (m->n <= 64) return launch_aba_warp_k<T, D, TB, 2>(m, B, q, qd, tau, qdd, status, base18, s);
    return launch_aba_warp_k<T, D, TB, 4>(m, B, q, qd, tau, qdd, status, base18, s);
}

}  // namespace rdyn
