// rnea_vjp_dh.cuh -- the adjoint of the two scans (rnea_vjp.cuh) in the
// common-normal frames of spatial_dh.cuh, with the link constants passed as a
// __grid_constant__ kernel parameter and FP32 sin/cos from trig_poly.cuh.
//
// The recursions are those of rnea_vjp.cuh; only the frames change. In a frame
// D_i the joint twist is still e_z (angular) and q_i enters the link transform
// as its last factor Rz(q_i), so d Ad_{f_i^-1} / dq_i = -ad_S Ad_{f_i^-1} and the
// gradient formulas carry over unchanged:
//   gqdd_i = S^T dVbar_i,
//   gqd_i  = S^T Vbar_i - <dVbar_i, ad_S V_i>,
//   gq_i   = -<Vbar_i, ad_S V_i> - <dVbar_i, ad_S dV_i> - <F_i, ad_S Fb_i>.
// Joint values and weights are read into registers one chunk ahead. For
// n % 4 == 0, n <= NMAX and 16-byte aligned rows.
#pragma once
#include "rnea_dhp.cuh"
#include "rnea_vjp.cuh"

namespace rdyn {

// Fb_i = Ad_{f^-1} Fb_{i-1} + S w  (the velocity step without the ad term)
template <typename T>
__device__ __forceinline__ void fb_forward_dh(const DhRot<T> &R, V3<T> b, T w, V3<T> &fv,
                                              V3<T> &fw)
{
    fv = dh_mulT(R, cross_add(fw, b, fv));
    fw = dh_mulT(R, fw);
    fw.z += w;
}

// inverse: Fb_{i-1} = Ad_f (Fb_i - S w)
template <typename T>
__device__ __forceinline__ void fb_backward_dh(const DhRot<T> &R, V3<T> b, T w, V3<T> &fv,
                                               V3<T> &fw)
{
    V3<T> ww = fw;
    ww.z -= w;
    const V3<T> pw = dh_mul(R, ww);
    fv = cross_add(b, pw, dh_mul(R, fv));
    fw = pw;
}

template <typename T, int NMAX, int BLOCK, int MODE, int TRIG>
__global__ void __launch_bounds__(BLOCK)
rnea_vjp_dh_kernel(const __grid_constant__ DhParamConsts<T, NMAX> pc, int n, int B,
                   const T *__restrict__ q, const T *__restrict__ qd, const T *__restrict__ qdd,
                   const T *__restrict__ wv, T *__restrict__ gq, T *__restrict__ gqd,
                   T *__restrict__ gqdd, T *__restrict__ ws, BaseParams<T> base)
{
    const T *sc = pc.c;
    // kVjpStoreShared: the per-link state in shared memory, [link][k][thread]
    extern __shared__ __align__(16) unsigned char vjp_smem[];
    T *sst = reinterpret_cast<T *>(vjp_smem);
    constexpr bool kStored = MODE == kVjpStore || MODE == kVjpStoreShared;
    auto st_put = [&](int i, int k, T v) {
        if constexpr (MODE == kVjpStoreShared)
            sst[((size_t)i * kVjpStateScalars + k) * BLOCK + threadIdx.x] = v;
        else
            ws_put(ws, B, blockIdx.x * BLOCK + threadIdx.x, i, k, v);
    };
    auto st_get = [&](int i, int k) -> T {
        if constexpr (MODE == kVjpStoreShared)
            return sst[((size_t)i * kVjpStateScalars + k) * BLOCK + threadIdx.x];
        else
            return ws_get(ws, B, blockIdx.x * BLOCK + threadIdx.x, i, k);
    };
    const int b = blockIdx.x * BLOCK + threadIdx.x;
    if (b >= B) return;
    const size_t row = (size_t)b * (size_t)n;
    const T *qr = q + row, *qdr = qd + row, *qddr = qdd + row, *wr = wv + row;

    Motion<T> x;
    x.v = mk3(base.V0[0], base.V0[1], base.V0[2]);
    x.w = mk3(base.V0[3], base.V0[4], base.V0[5]);
    x.a = mk3(base.dV0[0], base.dV0[1], base.dV0[2]);
    x.al = mk3(base.dV0[3], base.dV0[4], base.dV0[5]);
    V3<T> fbv = mk3(T(0), T(0), T(0)), fbw = mk3(T(0), T(0), T(0));

    // ---- sweep 1: base -> tip
    const int nchunks = n / 4;
    Chunk<T> cq, cqd, cqdd, cw, nq = {}, nqd = {}, nqdd = {}, nw = {};
    ld_row_chunk(qr, 0, cq);
    ld_row_chunk(qdr, 0, cqd);
    ld_row_chunk(qddr, 0, cqdd);
    ld_row_chunk(wr, 0, cw);
    for (int kc = 0; kc < nchunks; ++kc) {
        const int i0 = 4 * kc;
        if (kc + 1 < nchunks) {
            ld_row_chunk(qr, i0 + 4, nq);
            ld_row_chunk(qdr, i0 + 4, nqd);
            ld_row_chunk(qddr, i0 + 4, nqdd);
            ld_row_chunk(wr, i0 + 4, nw);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int i = i0 + j;
            DhXf<T> X;
            load_dh_xf(sc + i * kDhConsts, X);
            T s, c;
            dh_trig<T, TRIG>(cq.v[j] + X.th0, &s, &c);
            const DhRot<T> R = dh_rot(X.ca, X.sa, c, s);
            x = dh_forward(R, X.b, cqd.v[j], cqdd.v[j], x);
            fb_forward_dh(R, X.b, cw.v[j], fbv, fbw);
            if constexpr (kStored) {
                const T vals[kVjpStateScalars] = {x.v.x,  x.v.y,  x.v.z,  x.w.x,  x.w.y,
                                                  x.w.z,  x.a.x,  x.a.y,  x.a.z,  x.al.x,
                                                  x.al.y, x.al.z, fbv.x,  fbv.y,  fbv.z,
                                                  fbw.x,  fbw.y,  fbw.z,  c,      s};
#pragma unroll
                for (int k = 0; k < kVjpStateScalars; ++k) st_put(i, k, vals[k]);
            }
        }
        cq = nq;
        cqd = nqd;
        cqdd = nqdd;
        cw = nw;
    }

    // ---- sweep 2: tip -> base
    Wrench<T> F;
    F.f = mk3(base.Fn[0], base.Fn[1], base.Fn[2]);
    F.n = mk3(base.Fn[3], base.Fn[4], base.Fn[5]);
    Wrench<T> Vb, dVb;  // adjoints of V_{i+1}, dV_{i+1} (covectors)
    DhRot<T> Rn = dh_rot(T(1), T(0), T(1), T(0));
    V3<T> bn = mk3(T(0), T(0), T(0));
    T qdn = T(0);
    const int last0 = n - 4;
    ld_row_chunk(qdr, last0, cqd);
    if constexpr (MODE == kVjpRecompute) {
        ld_row_chunk(qr, last0, cq);
        ld_row_chunk(qddr, last0, cqdd);
        ld_row_chunk(wr, last0, cw);
    }
    for (int i0 = last0; i0 >= 0; i0 -= 4) {
        if (i0 > 0) {
            ld_row_chunk(qdr, i0 - 4, nqd);
            if constexpr (MODE == kVjpRecompute) {
                ld_row_chunk(qr, i0 - 4, nq);
                ld_row_chunk(qddr, i0 - 4, nqdd);
                ld_row_chunk(wr, i0 - 4, nw);
            }
        }
        Chunk<T> oq, oqd, oqdd;
#pragma unroll
        for (int j = 3; j >= 0; --j) {
            const int i = i0 + j;
            DhLink<T> L;
            load_dh(sc + i * kDhConsts, L);
            T s, c;
            if constexpr (kStored) {
                x.v = mk3(st_get(i, 0), st_get(i, 1), st_get(i, 2));
                x.w = mk3(st_get(i, 3), st_get(i, 4), st_get(i, 5));
                x.a = mk3(st_get(i, 6), st_get(i, 7), st_get(i, 8));
                x.al = mk3(st_get(i, 9), st_get(i, 10), st_get(i, 11));
                fbv = mk3(st_get(i, 12), st_get(i, 13), st_get(i, 14));
                fbw = mk3(st_get(i, 15), st_get(i, 16), st_get(i, 17));
                c = st_get(i, 18);
                s = st_get(i, 19);
            } else {
                dh_trig<T, TRIG>(cq.v[j] + L.th0, &s, &c);
            }
            const DhRot<T> R = dh_rot(L.ca, L.sa, c, s);
            const Wrench<T> Fh = bias_wrench(L.m, L.c, L.I, x);
            if (i == n - 1) {
                F.f = add3(F.f, Fh.f);
                F.n = add3(F.n, Fh.n);
            } else {
                F = dh_carry(Rn, bn, F, Fh);
            }
            // local seeds from F_hat = J dV - ad^T_V (J V)
            Wrench<T> dVl, Vl;
            J_apply(L.m, L.c, L.I, fbv, fbw, dVl.f, dVl.n);           // J Fb
            V3<T> jvf, jvn;
            J_apply(L.m, L.c, L.I, x.v, x.w, jvf, jvn);               // J V
            const V3<T> adv = cross_add(x.v, fbw, cross3(x.w, fbv));   // ad_V Fb
            const V3<T> adw = cross3(x.w, fbw);
            V3<T> jaf, jan;
            J_apply(L.m, L.c, L.I, adv, adw, jaf, jan);               // J ad_V Fb
            Vl.f = sub3(scale3(T(-1), cross3(fbw, jvf)), jaf);
            Vl.n = sub3(scale3(T(-1), cross_add(fbv, jvf, cross3(fbw, jvn))), jan);
            if (i == n - 1) {
                Vb = Vl;
                dVb = dVl;
            } else {
                Wrench<T> Yb = Vb;  // Vbar_{i+1} - ad^T_{S qd_{i+1}} dVbar_{i+1}
                Yb.f.x = fma(-qdn, dVb.f.y, Yb.f.x);
                Yb.f.y = fma(qdn, dVb.f.x, Yb.f.y);
                Yb.n.x = fma(-qdn, dVb.n.y, Yb.n.x);
                Yb.n.y = fma(qdn, dVb.n.x, Yb.n.y);
                Vb = dh_carry(Rn, bn, Yb, Vl);
                dVb = dh_carry(Rn, bn, dVb, dVl);
            }
            oqdd.v[j] = dVb.n.z;
            oqd.v[j] = Vb.n.z - (dot_ez_cross(dVb.f, x.v) + dot_ez_cross(dVb.n, x.w));
            oq.v[j] = -(dot_ez_cross(Vb.f, x.v) + dot_ez_cross(Vb.n, x.w)) -
                      (dot_ez_cross(dVb.f, x.a) + dot_ez_cross(dVb.n, x.al)) -
                      (dot_ez_cross(F.f, fbv) + dot_ez_cross(F.n, fbw));
            if constexpr (MODE == kVjpRecompute) {
                if (i > 0) {
                    x = dh_recover(R, L.b, cqd.v[j], cqdd.v[j], x);
                    fb_backward_dh(R, L.b, cw.v[j], fbv, fbw);
                }
            }
            Rn = R;
            bn = L.b;
            qdn = cqd.v[j];
        }
        st_chunk<T, true>(gq + row, i0, n, oq);
        st_chunk<T, true>(gqd + row, i0, n, oqd);
        st_chunk<T, true>(gqdd + row, i0, n, oqdd);
        cqd = nqd;
        if constexpr (MODE == kVjpRecompute) {
            cq = nq;
            cqdd = nqdd;
            cw = nw;
        }
    }
}

}  // namespace rdyn
