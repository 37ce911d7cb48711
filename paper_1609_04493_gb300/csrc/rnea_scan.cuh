// rnea_scan.cuh -- lane-parallel inverse dynamics: the two scans of Sec. III
// across the lanes of a warp.
//
// L consecutive lanes share one instance; lane l owns links [l K, l K + K).
//
// Forward (Sec. III-B, Eq. scan-id-vel-acc). The operand of a link is the
// semigroup element (g_i, xi1_i, xi2_i) = (f_{i-1,i}^-1, S_i qdd_i, S_i qd_i),
// combined later-on-the-left:
//   (g, x1, x2) (+) (g', x1', x2') = (g g', Ad_g x1' + x1 - ad_{x2} Ad_g x2',
//                                     Ad_g x2' + x2),
// and an element acts on a state (dV, V) as
//   (dV, V) -> (Ad_g dV - ad_{x2} Ad_g V + x1, Ad_g V + x2).
// Each lane folds its segment into one element: G = g_{e-1}...g_s, and
// (x1, x2) = the recursion run over the segment from a zero state (lane 0
// starts from the base state instead, so its element already carries the
// boundary). A Kogge-Stone scan with shuffles gives every lane the product of
// the elements below it, whose (x1, x2) is the true state entering its
// segment; the lane then replays its segment from that state, forming F_hat.
//
// Backward (Sec. III-C, Eq. id-bkwd-scan). A segment maps the wrench entering
// from above, F_e, to F_s = Ad^T_H F_e + b with H = g_e g_{e-1} ... g_{s+1};
// elements compose as (H, b) o (H', b') = (H' H, Ad^T_H b' + b). A suffix scan
// with shuffles gives each lane the true F_e; a replay of the segment then
// yields F_i and tau_i = S_i^T F_i.
#pragma once
#include "rnea_serial.cuh"

namespace rdyn {

template <typename T>
struct Rigid3 {
    Rot<T> R;
    V3<T> p;
};

template <typename T>
__device__ __forceinline__ Rigid3<T> rigid_identity()
{
    Rigid3<T> g;
#pragma unroll
    for (int k = 0; k < 9; ++k) g.R.r[k] = (k % 4 == 0) ? T(1) : T(0);
    g.p = mk3(T(0), T(0), T(0));
    return g;
}

// row-major 3x3 products
template <typename T>
__device__ __forceinline__ Rot<T> rot_mul(const Rot<T> &a, const Rot<T> &b)
{
    Rot<T> c;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            c.r[3 * i + j] = fma(a.r[3 * i + 0], b.r[j],
                                 fma(a.r[3 * i + 1], b.r[3 + j], a.r[3 * i + 2] * b.r[6 + j]));
    return c;
}

// a^T b
template <typename T>
__device__ __forceinline__ Rot<T> rot_tmul(const Rot<T> &a, const Rot<T> &b)
{
    Rot<T> c;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            c.r[3 * i + j] = fma(a.r[i], b.r[j], fma(a.r[3 + i], b.r[3 + j], a.r[6 + i] * b.r[6 + j]));
    return c;
}

// a b^T
template <typename T>
__device__ __forceinline__ Rot<T> rot_mult(const Rot<T> &a, const Rot<T> &b)
{
    Rot<T> c;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            c.r[3 * i + j] = fma(a.r[3 * i], b.r[3 * j],
                                 fma(a.r[3 * i + 1], b.r[3 * j + 1], a.r[3 * i + 2] * b.r[3 * j + 2]));
    return c;
}

// Ad_G (v, w) = (R v + p x R w, R w)
template <typename T>
__device__ __forceinline__ void Ad_apply(const Rigid3<T> &G, V3<T> v, V3<T> w, V3<T> &ov, V3<T> &ow)
{
    ow = mulA(G.R.r, w);
    ov = cross_add(G.p, ow, mulA(G.R.r, v));
}

// Ad^T_H (f, n) = (R^T f, R^T (n + f x p))
template <typename T>
__device__ __forceinline__ Wrench<T> AdT_apply(const Rigid3<T> &H, const Wrench<T> &F)
{
    Wrench<T> o;
    o.f = mulAT(H.R.r, F.f);
    o.n = mulAT(H.R.r, cross_add(F.f, H.p, F.n));
    return o;
}

// Forward element: G and the state (x1 = dV part (a, al), x2 = V part (v, w)).
template <typename T>
struct FwdElem {
    Rigid3<T> G;
    Motion<T> x;
};

// later (+) earlier
template <typename T>
__device__ __forceinline__ FwdElem<T> fwd_combine(const FwdElem<T> &L, const FwdElem<T> &E)
{
    FwdElem<T> o;
    o.G.R = rot_mul(L.G.R, E.G.R);
    o.G.p = add3(mulA(L.G.R.r, E.G.p), L.G.p);
    V3<T> av, aw, dv, dw;
    Ad_apply(L.G, E.x.v, E.x.w, av, aw);     // Ad_G x2'
    Ad_apply(L.G, E.x.a, E.x.al, dv, dw);    // Ad_G x1'
    o.x.v = add3(av, L.x.v);
    o.x.w = add3(aw, L.x.w);
    // - ad_{x2}(Ad_G x2'), ad_{(v2,w2)}(v, w) = (w2 x v + v2 x w, w2 x w)
    V3<T> adv = cross_add(L.x.v, aw, cross3(L.x.w, av));
    V3<T> adw = cross3(L.x.w, aw);
    o.x.a = sub3(add3(dv, L.x.a), adv);
    o.x.al = sub3(add3(dw, L.x.al), adw);
    return o;
}

template <typename T>
struct BwdElem {
    Rigid3<T> H;
    Wrench<T> b;
};

// lower o upper: (H, b) o (H', b') = (H' H, Ad^T_H b' + b)
template <typename T>
__device__ __forceinline__ BwdElem<T> bwd_combine(const BwdElem<T> &Lo, const BwdElem<T> &Up)
{
    BwdElem<T> o;
    o.H.R = rot_mul(Up.H.R, Lo.H.R);
    o.H.p = add3(mulA(Up.H.R.r, Lo.H.p), Up.H.p);
    Wrench<T> t = AdT_apply(Lo.H, Up.b);
    o.b.f = add3(t.f, Lo.b.f);
    o.b.n = add3(t.n, Lo.b.n);
    return o;
}

template <typename T>
__device__ __forceinline__ T shup(T v, int d, int L)
{
    return __shfl_up_sync(0xffffffffu, v, d, L);
}

template <typename T>
__device__ __forceinline__ T shdn(T v, int d, int L)
{
    return __shfl_down_sync(0xffffffffu, v, d, L);
}

template <typename T>
__device__ __forceinline__ V3<T> shup3(V3<T> a, int d, int L)
{
    return mk3(shup(a.x, d, L), shup(a.y, d, L), shup(a.z, d, L));
}

template <typename T>
__device__ __forceinline__ V3<T> shdn3(V3<T> a, int d, int L)
{
    return mk3(shdn(a.x, d, L), shdn(a.y, d, L), shdn(a.z, d, L));
}

template <typename T>
__device__ __forceinline__ Rigid3<T> shup_rigid(const Rigid3<T> &g, int d, int L)
{
    Rigid3<T> o;
#pragma unroll
    for (int k = 0; k < 9; ++k) o.R.r[k] = shup(g.R.r[k], d, L);
    o.p = shup3(g.p, d, L);
    return o;
}

template <typename T>
__device__ __forceinline__ Rigid3<T> shdn_rigid(const Rigid3<T> &g, int d, int L)
{
    Rigid3<T> o;
#pragma unroll
    for (int k = 0; k < 9; ++k) o.R.r[k] = shdn(g.R.r[k], d, L);
    o.p = shdn3(g.p, d, L);
    return o;
}

// g_i = f_{i-1,i}^-1 = (R^T, -R^T b); returns g_i * G.
template <typename T>
__device__ __forceinline__ Rigid3<T> premul_ginv(const Rot<T> &R, V3<T> b, const Rigid3<T> &G)
{
    Rigid3<T> o;
    o.R = rot_tmul(R, G.R);
    o.p = mulAT(R.r, sub3(G.p, b));
    return o;
}

// H * g_j with g_j = (R^T, -R^T b): (R_H R^T, -R_H R^T b + p_H)
template <typename T>
__device__ __forceinline__ Rigid3<T> postmul_ginv(const Rigid3<T> &H, const Rot<T> &R, V3<T> b)
{
    Rigid3<T> o;
    o.R = rot_mult(H.R, R);
    o.p = sub3(H.p, mulA(o.R.r, b));
    return o;
}

// Grid: one instance per L consecutive lanes, 32 / L instances per warp.
template <typename T, int L, int K, bool FAST>
__global__ void __launch_bounds__(128)
rnea_scan_kernel(const T *__restrict__ consts, int n, int B, const T *__restrict__ q,
                 const T *__restrict__ qd, const T *__restrict__ qdd, T *__restrict__ tau,
                 BaseParams<T> base)
{
    extern __shared__ __align__(16) unsigned char smem[];
    T *sc = reinterpret_cast<T *>(smem);
    const int nc = n * kLinkConsts;
    for (int k = threadIdx.x; k < nc; k += blockDim.x) sc[k] = consts[k];
    __syncthreads();

    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int inst = gtid / L;
    const int l = threadIdx.x % L;
    const bool live = inst < B;
    const size_t row = (size_t)(live ? inst : B - 1) * (size_t)n;
    const int s0 = l * K;

    // joint values of the segment
    T jq[K], jqd[K], jqdd[K], jc[K], js[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int i = s0 + j;
        jq[j] = i < n ? __ldg(q + row + i) : T(0);
        jqd[j] = i < n ? __ldg(qd + row + i) : T(0);
        jqdd[j] = i < n ? __ldg(qdd + row + i) : T(0);
        joint_trig<T, FAST>(jq[j], &js[j], &jc[j]);
    }

    // ---- forward: segment element (lane 0 starts from the base state)
    FwdElem<T> E;
    E.G = rigid_identity<T>();
    if (l == 0) {
        E.x.v = mk3(base.V0[0], base.V0[1], base.V0[2]);
        E.x.w = mk3(base.V0[3], base.V0[4], base.V0[5]);
        E.x.a = mk3(base.dV0[0], base.dV0[1], base.dV0[2]);
        E.x.al = mk3(base.dV0[3], base.dV0[4], base.dV0[5]);
    } else {
        E.x.v = E.x.w = E.x.a = E.x.al = mk3(T(0), T(0), T(0));
    }
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int i = s0 + j;
        if (i < n) {
            LinkXf<T> X;
            load_xf(sc + i * kLinkConsts, X);
            const Rot<T> R = make_rot(X.A, jc[j], js[j]);
            const V3<T> b = mk3(X.b[0], X.b[1], X.b[2]);
            E.x = forward_step_R(R, b, jqd[j], jqdd[j], E.x);
            E.G = premul_ginv(R, b, E.G);
        }
    }
    // inclusive Kogge-Stone scan over the L lanes (later on the left)
#pragma unroll
    for (int d = 1; d < L; d <<= 1) {
        FwdElem<T> Y;
        Y.G = shup_rigid(E.G, d, L);
        Y.x.v = shup3(E.x.v, d, L);
        Y.x.w = shup3(E.x.w, d, L);
        Y.x.a = shup3(E.x.a, d, L);
        Y.x.al = shup3(E.x.al, d, L);
        if (l >= d) E = fwd_combine(E, Y);
    }
    // state entering this segment = state part of the previous lane's prefix
    Motion<T> x;
    x.v = shup3(E.x.v, 1, L);
    x.w = shup3(E.x.w, 1, L);
    x.a = shup3(E.x.a, 1, L);
    x.al = shup3(E.x.al, 1, L);
    if (l == 0) {
        x.v = mk3(base.V0[0], base.V0[1], base.V0[2]);
        x.w = mk3(base.V0[3], base.V0[4], base.V0[5]);
        x.a = mk3(base.dV0[0], base.dV0[1], base.dV0[2]);
        x.al = mk3(base.dV0[3], base.dV0[4], base.dV0[5]);
    }
    // replay the segment: true motion and bias wrenches
    Wrench<T> Fh[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int i = s0 + j;
        if (i < n) {
            LinkC<T> Lc;
            load_link(sc + i * kLinkConsts, Lc);
            const Rot<T> R = make_rot(Lc.A, jc[j], js[j]);
            x = forward_step_R(R, mk3(Lc.b[0], Lc.b[1], Lc.b[2]), jqd[j], jqdd[j], x);
            Fh[j] = bias_wrench(Lc.m, mk3(Lc.c[0], Lc.c[1], Lc.c[2]), Lc.I, x);
        } else {
            Fh[j].f = Fh[j].n = mk3(T(0), T(0), T(0));
        }
    }

    // ---- backward: (c, s) of the first link above this segment, from lane l+1
    const T c_up = shdn(jc[0], 1, L), s_up = shdn(js[0], 1, L);
    const int e = s0 + K;  // first link above the segment
    const bool tip_lane = (s0 < n) && (e >= n);
    BwdElem<T> Bk;
    Bk.H = rigid_identity<T>();
    Bk.b.f = Bk.b.n = mk3(T(0), T(0), T(0));
    if (tip_lane) {
        Bk.b.f = mk3(base.Fn[0], base.Fn[1], base.Fn[2]);
        Bk.b.n = mk3(base.Fn[3], base.Fn[4], base.Fn[5]);
    }
    if (s0 < n) {
        // transform of link e (for segments below the tip)
        Rot<T> Rup;
        V3<T> bup = mk3(T(0), T(0), T(0));
        if (!tip_lane) {
            LinkXf<T> X;
            load_xf(sc + e * kLinkConsts, X);
            Rup = make_rot(X.A, c_up, s_up);
            bup = mk3(X.b[0], X.b[1], X.b[2]);
            Bk.H.R = Rup;  // g_e = (Rup^T, -Rup^T bup): H = g_e
#pragma unroll
            for (int k = 0; k < 9; ++k) Bk.H.R.r[k] = Rup.r[3 * (k % 3) + k / 3];
            Bk.H.p = mk3(T(0), T(0), T(0));
            Bk.H.p = sub3(Bk.H.p, mulAT(Rup.r, bup));
        }
        Rot<T> Rn = Rup;
        V3<T> bn = bup;
#pragma unroll
        for (int j = K - 1; j >= 0; --j) {
            const int i = s0 + j;
            if (i < n) {
                if (i == n - 1 || i == e - 1) {
                    Bk.b.f = add3(Bk.b.f, Fh[j].f);
                    Bk.b.n = add3(Bk.b.n, Fh[j].n);
                } else {
                    Bk.b = carry_wrench_R(Rn, bn, Bk.b, Fh[j]);
                    Bk.H = postmul_ginv(Bk.H, Rn, bn);
                }
                LinkXf<T> X;
                load_xf(sc + i * kLinkConsts, X);
                Rn = make_rot(X.A, jc[j], js[j]);
                bn = mk3(X.b[0], X.b[1], X.b[2]);
            }
        }
    }
    // inclusive suffix scan (lower o upper)
#pragma unroll
    for (int d = 1; d < L; d <<= 1) {
        BwdElem<T> Y;
        Y.H = shdn_rigid(Bk.H, d, L);
        Y.b.f = shdn3(Bk.b.f, d, L);
        Y.b.n = shdn3(Bk.b.n, d, L);
        if (l + d < L) Bk = bwd_combine(Bk, Y);
    }
    // true wrench entering from above = b of the next lane's suffix
    Wrench<T> F;
    F.f = shdn3(Bk.b.f, 1, L);
    F.n = shdn3(Bk.b.n, 1, L);
    if (tip_lane) {
        F.f = mk3(base.Fn[0], base.Fn[1], base.Fn[2]);
        F.n = mk3(base.Fn[3], base.Fn[4], base.Fn[5]);
    }
    // replay the segment downward
    if (s0 < n) {
        Rot<T> Rn;
        V3<T> bn = mk3(T(0), T(0), T(0));
        if (!tip_lane) {
            LinkXf<T> X;
            load_xf(sc + e * kLinkConsts, X);
            Rn = make_rot(X.A, c_up, s_up);
            bn = mk3(X.b[0], X.b[1], X.b[2]);
        }
        T out[K];
#pragma unroll
        for (int j = K - 1; j >= 0; --j) {
            const int i = s0 + j;
            out[j] = T(0);
            if (i < n) {
                if (i == n - 1) {
                    F.f = add3(F.f, Fh[j].f);
                    F.n = add3(F.n, Fh[j].n);
                } else {
                    F = carry_wrench_R(Rn, bn, F, Fh[j]);
                }
                out[j] = F.n.z;
                LinkXf<T> X;
                load_xf(sc + i * kLinkConsts, X);
                Rn = make_rot(X.A, jc[j], js[j]);
                bn = mk3(X.b[0], X.b[1], X.b[2]);
            }
        }
        if (live) {
#pragma unroll
            for (int j = 0; j < K; ++j)
                if (s0 + j < n) tau[row + s0 + j] = out[j];
        }
    }
}

}  // namespace rdyn
