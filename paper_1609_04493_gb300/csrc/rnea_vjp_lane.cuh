// rnea_vjp_lane.cuh -- the adjoint of inverse dynamics (rnea_vjp_dh.cuh) with
// L lanes per instance, for batches too small to fill the GPU with one thread
// per instance. Lane l owns links [l K, l K + K).
//
// Forward, the scan of Sec. III-B with the adjoint weight as a third channel:
// the element (G, x1, x2, x3) acts on (dV, V, Fb) as
//     (Ad_G dV - ad_x2 Ad_G V + x1, Ad_G V + x2, Ad_G Fb + x3),
// so Fb_i = Ad_{f_i^-1} Fb_{i-1} + S_i w_i composes like V without the ad term.
// Each lane folds its segment from a zero state (lane 0 from the base state),
// a Kogge-Stone prefix over the L lanes gives the state entering each segment,
// and a replay yields V_i, dV_i, Fb_i, kept in shared memory with cos, sin.
//
// Backward, the state y_i = (F_i, dVbar_i, Vbar_i) of the reverse sweep is
// affine in y_{i+1}:
//     y_i = M(A, X) y_{i+1} + c_i,   A = Ad_{f_{i+1}^-1},  X = S_{i+1} qd_{i+1},
//     M(A, X) y = (A^T F, A^T dVbar, A^T (Vbar - ad_X^T dVbar)),
// with the local seeds c_i = (F_hat_i, J_i Fb_i, ad_Fb^T J_i V_i - J_i ad_V Fb)
// (for the top link A = I, X = 0). A segment is one element (H, X, bF, bD, bV)
// with A = Ad_H; elements compose, lower o upper, as
//     (H_up H_lo, Ad_{H_up} X_lo + X_up,
//      Ad^T_{H_lo} bF_up + bF_lo, Ad^T_{H_lo} bD_up + bD_lo,
//      Ad^T_{H_lo} (bV_up - ad^T_{X_lo} bD_up) + bV_lo)
// (tests/test_adjoint_segments_cpu.py checks this against 18 x 18 products and
// every bracketing against the serial values). A lane's fold is the serial
// reverse sweep over its links from a zero state, tracking H and X; a suffix
// combine gives the state entering each segment from above; the replay is the
// serial reverse sweep from that state, with the gradients
//     gqdd_i = S^T dVbar_i,  gqd_i = S^T Vbar_i - <dVbar_i, ad_S V_i>,
//     gq_i = -<Vbar_i, ad_S V_i> - <dVbar_i, ad_S dV_i> - <F_i, ad_S Fb_i>.
// Common-normal frames, constants as a kernel parameter; n % 4 == 0, n <= L K,
// 16-byte aligned rows.
#pragma once
#include "rnea_scan.cuh"
#include "rnea_vjp_dh.cuh"

namespace rdyn {

template <typename T>
struct FwdElem3 {
    Rigid3<T> G;
    Motion<T> x;
    V3<T> fv, fw;
};

// later (+) earlier, with the Fb channel
template <typename T>
__device__ __forceinline__ FwdElem3<T> fwd3_combine(const FwdElem3<T> &Lt, const FwdElem3<T> &E)
{
    FwdElem<T> a, e;
    a.G = Lt.G;
    a.x = Lt.x;
    e.G = E.G;
    e.x = E.x;
    const FwdElem<T> c = fwd_combine(a, e);
    FwdElem3<T> o;
    o.G = c.G;
    o.x = c.x;
    V3<T> fv, fw;
    Ad_apply(Lt.G, E.fv, E.fw, fv, fw);
    o.fv = add3(fv, Lt.fv);
    o.fw = add3(fw, Lt.fw);
    return o;
}

template <typename T>
struct AdjElem {
    Rigid3<T> H;
    V3<T> xv, xw;
    Wrench<T> bF, bD, bV;
};

template <typename T>
__device__ __forceinline__ Wrench<T> wadd(const Wrench<T> &a, const Wrench<T> &b)
{
    return Wrench<T>{add3(a.f, b.f), add3(a.n, b.n)};
}

// ad^T_X w for X = (xv, xw), w = (f, n): (-xw x f, -xv x f - xw x n)
template <typename T>
__device__ __forceinline__ Wrench<T> adT_apply(V3<T> xv, V3<T> xw, const Wrench<T> &w)
{
    Wrench<T> o;
    o.f = cross3(w.f, xw);
    o.n = cross_add(w.f, xv, cross3(w.n, xw));
    return o;
}

// lower o upper
template <typename T>
__device__ __forceinline__ AdjElem<T> adj_combine(const AdjElem<T> &Lo, const AdjElem<T> &Up)
{
    AdjElem<T> o;
    o.H.R = rot_mul(Up.H.R, Lo.H.R);
    o.H.p = add3(mulA(Up.H.R.r, Lo.H.p), Up.H.p);
    V3<T> av, aw;
    Ad_apply(Up.H, Lo.xv, Lo.xw, av, aw);
    o.xv = add3(av, Up.xv);
    o.xw = add3(aw, Up.xw);
    o.bF = wadd(AdT_apply(Lo.H, Up.bF), Lo.bF);
    o.bD = wadd(AdT_apply(Lo.H, Up.bD), Lo.bD);
    const Wrench<T> ad = adT_apply(Lo.xv, Lo.xw, Up.bD);
    const Wrench<T> y{sub3(Up.bV.f, ad.f), sub3(Up.bV.n, ad.n)};
    o.bV = wadd(AdT_apply(Lo.H, y), Lo.bV);
    return o;
}

template <typename T>
__device__ __forceinline__ Wrench<T> shdn_w(const Wrench<T> &w, int d, int L)
{
    return Wrench<T>{shdn3(w.f, d, L), shdn3(w.n, d, L)};
}

// the seeds of link i from its motion and adjoint weight (rnea_vjp_dh.cuh)
template <typename T>
__device__ __forceinline__ void vjp_seeds(const DhLink<T> &L, const Motion<T> &x, V3<T> fbv,
                                          V3<T> fbw, Wrench<T> &Fh, Wrench<T> &dVl,
                                          Wrench<T> &Vl)
{
    Fh = bias_wrench(L.m, L.c, L.I, x);
    J_apply(L.m, L.c, L.I, fbv, fbw, dVl.f, dVl.n);
    V3<T> jvf, jvn;
    J_apply(L.m, L.c, L.I, x.v, x.w, jvf, jvn);
    const V3<T> adv = cross_add(x.v, fbw, cross3(x.w, fbv));
    const V3<T> adw = cross3(x.w, fbw);
    V3<T> jaf, jan;
    J_apply(L.m, L.c, L.I, adv, adw, jaf, jan);
    Vl.f = sub3(scale3(T(-1), cross3(fbw, jvf)), jaf);
    Vl.n = sub3(scale3(T(-1), cross_add(fbv, jvf, cross3(fbw, jvn))), jan);
}

// one step of the reverse sweep from link i+1 (transform Rn, bn; joint rate
// qdn) to link i: F, dVbar, Vbar (top: no carry)
template <typename T>
__device__ __forceinline__ void vjp_reverse_step(bool top, const DhRot<T> &Rn, V3<T> bn, T qdn,
                                                 const Wrench<T> &Fh, const Wrench<T> &dVl,
                                                 const Wrench<T> &Vl, Wrench<T> &F,
                                                 Wrench<T> &dVb, Wrench<T> &Vb)
{
    if (top) {
        F = wadd(F, Fh);
        dVb = wadd(dVb, dVl);
        Vb = wadd(Vb, Vl);
    } else {
        Wrench<T> Yb = Vb;  // Vbar_{i+1} - ad^T_{S qd_{i+1}} dVbar_{i+1}
        Yb.f.x = fma(-qdn, dVb.f.y, Yb.f.x);
        Yb.f.y = fma(qdn, dVb.f.x, Yb.f.y);
        Yb.n.x = fma(-qdn, dVb.n.y, Yb.n.x);
        Yb.n.y = fma(qdn, dVb.n.x, Yb.n.y);
        F = dh_carry(Rn, bn, F, Fh);
        Vb = dh_carry(Rn, bn, Yb, Vl);
        dVb = dh_carry(Rn, bn, dVb, dVl);
    }
}

// per-link state of a lane in shared memory, [link][component][thread]
constexpr int kVjpLaneScalars = 18;
// The lanes of a warp read different links' constants at once: from the
// kernel-parameter bank those reads serialise, so each block copies them to
// shared memory first, 20 scalars apart (80 bytes in FP32: the 16-byte reads of
// eight consecutive links then fall in distinct banks).
constexpr int kVjpLaneConstStride = 20;

// Segments of up to 4 links fit in 128 registers without spilling, which
// leaves room for four 128-thread blocks per SM (a batch of 8192 instances at 8
// lanes then runs in one wave); longer segments keep their registers.
template <typename T, int NMAX, int L, int K, int BLOCK, int TRIG>
__global__ void __launch_bounds__(BLOCK, K <= 4 ? 512 / BLOCK : 1)
rnea_vjp_lane_kernel(const __grid_constant__ DhParamConsts<T, NMAX> pc, int n, int B,
                     const T *__restrict__ q, const T *__restrict__ qd,
                     const T *__restrict__ qdd, const T *__restrict__ wv, T *__restrict__ gq,
                     T *__restrict__ gqd, T *__restrict__ gqdd, BaseParams<T> base)
{
    static_assert(K % 4 == 0, "whole 16-byte chunks per lane");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sconst = reinterpret_cast<T *>(smem_raw);
    T *sm = sconst + NMAX * kVjpLaneConstStride;
    const int tid = threadIdx.x;
    for (int k = tid; k < n * kDhConsts; k += BLOCK)
        sconst[(k / kDhConsts) * kVjpLaneConstStride + k % kDhConsts] = pc.c[k];
    __syncthreads();
    const T *sc = sconst;
    const int l = tid % L;
    const int inst = (blockIdx.x * BLOCK + tid) / L;
    const bool live = inst < B;
    const size_t row = (size_t)(live ? inst : B - 1) * (size_t)n;
    const int s0 = l * K;
    const T zero = T(0);
    auto put = [&](int j, int k, T v) { sm[(j * kVjpLaneScalars + k) * BLOCK + tid] = v; };
    auto get = [&](int j, int k) { return sm[(j * kVjpLaneScalars + k) * BLOCK + tid]; };

    // joint values of the segment
    T jq[K], jqd[K], jqdd[K], jw[K], jc[K], js[K];
#pragma unroll
    for (int c = 0; c < K / 4; ++c) {
        Chunk<T> a = {}, b = {}, d = {}, e = {};
        if (s0 + 4 * c < n) {
            ld_row_chunk(q + row, s0 + 4 * c, a);
            ld_row_chunk(qd + row, s0 + 4 * c, b);
            ld_row_chunk(qdd + row, s0 + 4 * c, d);
            ld_row_chunk(wv + row, s0 + 4 * c, e);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            jq[4 * c + j] = a.v[j];
            jqd[4 * c + j] = b.v[j];
            jqdd[4 * c + j] = d.v[j];
            jw[4 * c + j] = e.v[j];
        }
    }
#pragma unroll
    for (int j = 0; j < K; ++j) {
        jc[j] = T(1);
        js[j] = zero;
        if (s0 + j < n) dh_trig<T, TRIG>(jq[j] + sc[(s0 + j) * kVjpLaneConstStride + 5], &js[j], &jc[j]);
    }
    Motion<T> xb;
    xb.v = mk3(base.V0[0], base.V0[1], base.V0[2]);
    xb.w = mk3(base.V0[3], base.V0[4], base.V0[5]);
    xb.a = mk3(base.dV0[0], base.dV0[1], base.dV0[2]);
    xb.al = mk3(base.dV0[3], base.dV0[4], base.dV0[5]);

    // ---- forward: fold, prefix combine, replay
    FwdElem3<T> E;
    E.G = rigid_identity<T>();
    if (l == 0) E.x = xb;
    else E.x.v = E.x.w = E.x.a = E.x.al = mk3(zero, zero, zero);
    E.fv = E.fw = mk3(zero, zero, zero);
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int i = s0 + j;
        if (i < n) {
            DhXf<T> X;
            load_dh_xf(sc + i * kVjpLaneConstStride, X);
            const DhRot<T> R = dh_rot(X.ca, X.sa, jc[j], js[j]);
            E.x = dh_forward(R, X.b, jqd[j], jqdd[j], E.x);
            fb_forward_dh(R, X.b, jw[j], E.fv, E.fw);
            Rot<T> Rf;
            Rf.r[0] = jc[j];          Rf.r[1] = -js[j];         Rf.r[2] = zero;
            Rf.r[3] = R.sca;          Rf.r[4] = R.cca;          Rf.r[5] = -X.sa;
            Rf.r[6] = R.ssa;          Rf.r[7] = R.csa;          Rf.r[8] = X.ca;
            E.G = premul_ginv(Rf, X.b, E.G);
        }
    }
#pragma unroll
    for (int d = 1; d < L; d <<= 1) {
        FwdElem3<T> Y;
        Y.G = shup_rigid(E.G, d, L);
        Y.x.v = shup3(E.x.v, d, L);
        Y.x.w = shup3(E.x.w, d, L);
        Y.x.a = shup3(E.x.a, d, L);
        Y.x.al = shup3(E.x.al, d, L);
        Y.fv = shup3(E.fv, d, L);
        Y.fw = shup3(E.fw, d, L);
        if (l >= d) E = fwd3_combine(E, Y);
    }
    Motion<T> x;
    x.v = shup3(E.x.v, 1, L);
    x.w = shup3(E.x.w, 1, L);
    x.a = shup3(E.x.a, 1, L);
    x.al = shup3(E.x.al, 1, L);
    V3<T> fbv = shup3(E.fv, 1, L), fbw = shup3(E.fw, 1, L);
    if (l == 0) {
        x = xb;
        fbv = fbw = mk3(zero, zero, zero);
    }
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int i = s0 + j;
        if (i < n) {
            DhXf<T> X;
            load_dh_xf(sc + i * kVjpLaneConstStride, X);
            const DhRot<T> R = dh_rot(X.ca, X.sa, jc[j], js[j]);
            x = dh_forward(R, X.b, jqd[j], jqdd[j], x);
            fb_forward_dh(R, X.b, jw[j], fbv, fbw);
            const T vals[18] = {x.v.x, x.v.y, x.v.z, x.w.x, x.w.y, x.w.z, x.a.x, x.a.y, x.a.z,
                                x.al.x, x.al.y, x.al.z, fbv.x, fbv.y, fbv.z, fbw.x, fbw.y, fbw.z};
#pragma unroll
            for (int k = 0; k < 18; ++k) put(j, k, vals[k]);
        }
    }

    // ---- backward: the transform and rate of link e = s0 + K (lane l+1's first)
    const int e = s0 + K;
    const T c_up = shdn(jc[0], 1, L), s_up = shdn(js[0], 1, L), qd_up = shdn(jqd[0], 1, L);
    DhRot<T> Rup = dh_rot(T(1), zero, T(1), zero);
    V3<T> bup = mk3(zero, zero, zero);
    if (e < n) {
        DhXf<T> X;
        load_dh_xf(sc + e * kVjpLaneConstStride, X);
        Rup = dh_rot(X.ca, X.sa, c_up, s_up);
        bup = X.b;
    }
    auto load_motion = [&](int j, Motion<T> &xm, V3<T> &fv, V3<T> &fw) {
        xm.v = mk3(get(j, 0), get(j, 1), get(j, 2));
        xm.w = mk3(get(j, 3), get(j, 4), get(j, 5));
        xm.a = mk3(get(j, 6), get(j, 7), get(j, 8));
        xm.al = mk3(get(j, 9), get(j, 10), get(j, 11));
        fv = mk3(get(j, 12), get(j, 13), get(j, 14));
        fw = mk3(get(j, 15), get(j, 16), get(j, 17));
    };
    // fold: the reverse sweep over the segment from zero, tracking H and X
    AdjElem<T> A;
    A.H = rigid_identity<T>();
    A.xv = A.xw = mk3(zero, zero, zero);
    A.bF.f = A.bF.n = A.bD.f = A.bD.n = A.bV.f = A.bV.n = mk3(zero, zero, zero);
    {
        DhRot<T> Rn = Rup;
        V3<T> bn = bup;
        T qdn = qd_up;
#pragma unroll
        for (int j = K - 1; j >= 0; --j) {
            const int i = s0 + j;
            if (i < n) {
                DhLink<T> Lk;
                load_dh(sc + i * kVjpLaneConstStride, Lk);
                Motion<T> xm;
                V3<T> fv, fw;
                load_motion(j, xm, fv, fw);
                Wrench<T> Fh, dVl, Vl;
                vjp_seeds(Lk, xm, fv, fw, Fh, dVl, Vl);
                const bool top = i == n - 1;
                if (!top) {
                    // H <- H g_{i+1}, X <- Ad_H X_{i+1} + X, X_{i+1} = qd_{i+1} e_z (angular)
                    V3<T> av, aw;
                    Ad_apply(A.H, mk3(zero, zero, zero), mk3(zero, zero, qdn), av, aw);
                    A.xv = add3(av, A.xv);
                    A.xw = add3(aw, A.xw);
                    Rot<T> Rf;
                    Rf.r[0] = Rn.c;   Rf.r[1] = -Rn.s;  Rf.r[2] = zero;
                    Rf.r[3] = Rn.sca; Rf.r[4] = Rn.cca; Rf.r[5] = -Rn.sa;
                    Rf.r[6] = Rn.ssa; Rf.r[7] = Rn.csa; Rf.r[8] = Rn.ca;
                    A.H = postmul_ginv(A.H, Rf, bn);
                }
                vjp_reverse_step(top, Rn, bn, qdn, Fh, dVl, Vl, A.bF, A.bD, A.bV);
                Rn = dh_rot(Lk.ca, Lk.sa, jc[j], js[j]);
                bn = Lk.b;
                qdn = jqd[j];
            }
        }
    }
    // suffix combine, lower o upper
#pragma unroll
    for (int d = 1; d < L; d <<= 1) {
        AdjElem<T> Y;
        Y.H = shdn_rigid(A.H, d, L);
        Y.xv = shdn3(A.xv, d, L);
        Y.xw = shdn3(A.xw, d, L);
        Y.bF = shdn_w(A.bF, d, L);
        Y.bD = shdn_w(A.bD, d, L);
        Y.bV = shdn_w(A.bV, d, L);
        if (l + d < L) A = adj_combine(A, Y);
    }
    // state entering from above: the next lane's suffix applied to
    // y_top = (F_{n+1}, 0, 0)
    Wrench<T> Ftop;
    Ftop.f = mk3(base.Fn[0], base.Fn[1], base.Fn[2]);
    Ftop.n = mk3(base.Fn[3], base.Fn[4], base.Fn[5]);
    AdjElem<T> U;
    U.H = shdn_rigid(A.H, 1, L);
    U.bF = shdn_w(A.bF, 1, L);
    U.bD = shdn_w(A.bD, 1, L);
    U.bV = shdn_w(A.bV, 1, L);
    Wrench<T> F, dVb, Vb;
    if (l + 1 < L) {
        F = wadd(AdT_apply(U.H, Ftop), U.bF);
        dVb = U.bD;
        Vb = U.bV;
    } else {
        F = Ftop;
        dVb.f = dVb.n = Vb.f = Vb.n = mk3(zero, zero, zero);
    }
    // replay with the gradients
    if (s0 < n) {
        DhRot<T> Rn = Rup;
        V3<T> bn = bup;
        T qdn = qd_up;
        T oq[K], oqd[K], oqdd[K];
#pragma unroll
        for (int j = K - 1; j >= 0; --j) {
            const int i = s0 + j;
            oq[j] = oqd[j] = oqdd[j] = zero;
            if (i < n) {
                DhLink<T> Lk;
                load_dh(sc + i * kVjpLaneConstStride, Lk);
                Motion<T> xm;
                V3<T> fv, fw;
                load_motion(j, xm, fv, fw);
                Wrench<T> Fh, dVl, Vl;
                vjp_seeds(Lk, xm, fv, fw, Fh, dVl, Vl);
                vjp_reverse_step(i == n - 1, Rn, bn, qdn, Fh, dVl, Vl, F, dVb, Vb);
                oqdd[j] = dVb.n.z;
                oqd[j] = Vb.n.z - (dot_ez_cross(dVb.f, xm.v) + dot_ez_cross(dVb.n, xm.w));
                oq[j] = -(dot_ez_cross(Vb.f, xm.v) + dot_ez_cross(Vb.n, xm.w)) -
                        (dot_ez_cross(dVb.f, xm.a) + dot_ez_cross(dVb.n, xm.al)) -
                        (dot_ez_cross(F.f, fv) + dot_ez_cross(F.n, fw));
                Rn = dh_rot(Lk.ca, Lk.sa, jc[j], js[j]);
                bn = Lk.b;
                qdn = jqd[j];
            }
        }
        if (live) {
#pragma unroll
            for (int c = 0; c < K / 4; ++c) {
                if (s0 + 4 * c < n) {
                    Chunk<T> a, b, d;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        a.v[j] = oq[4 * c + j];
                        b.v[j] = oqd[4 * c + j];
                        d.v[j] = oqdd[4 * c + j];
                    }
                    st_chunk<T, true>(gq + row, s0 + 4 * c, n, a);
                    st_chunk<T, true>(gqd + row, s0 + 4 * c, n, b);
                    st_chunk<T, true>(gqdd + row, s0 + 4 * c, n, d);
                }
            }
        }
    }
}

}  // namespace rdyn
