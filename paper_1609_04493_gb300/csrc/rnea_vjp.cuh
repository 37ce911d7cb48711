// rnea_vjp.cuh -- adjoint of the two scans: the vector-Jacobian product
//     (gq, gqd, gqdd) = d(w^T tau)/d(q, qd, qdd)
// for a batch, one thread per instance.
//
// Reverse mode through Eqs. (id-forward) and (id-backward), in joint frames
// (S = e_z angular). With bars for adjoints:
//   tau_i = S^T F_i and F_{i-1} = Ad^T_{f_i^-1} F_i + F_hat_{i-1} give a
//   twist-like adjoint of the wrenches that runs base -> tip,
//       Fb_i = Ad_{f_i^-1} Fb_{i-1} + S w_i,          F_hat_bar_i = Fb_i;
//   F_hat = J dV - ad^T_V (J V) seeds
//       dVbar_i += J Fb_i,   Vbar_i += ad^T_{Fb_i}(J V_i) - J ad_{V_i} Fb_i;
//   the forward recursion is then reversed tip -> base:
//       Ybar_{i+1} = Vbar_{i+1} - ad^T_{S qd_{i+1}} dVbar_{i+1},
//       Vbar_i  += Ad^T_{f_{i+1}^-1} Ybar_{i+1},
//       dVbar_i += Ad^T_{f_{i+1}^-1} dVbar_{i+1};
//   and with d Ad_{f_i^-1}/dq_i = -ad_S Ad_{f_i^-1} the gradients are
//       gqdd_i = S^T dVbar_i,
//       gqd_i  = S^T Vbar_i - <dVbar_i, ad_S V_i>,
//       gq_i   = -<Vbar_i, ad_S V_i> - <dVbar_i, ad_S dV_i> - <F_i, ad_S Fb_i>.
// Sweep 1 (base -> tip) computes V, dV and Fb; sweep 2 (tip -> base) the
// wrenches, the adjoints and the gradients. What sweep 2 needs of sweep 1:
//   kVjpStore     -- V, dV, Fb, cos, sin of every link (20 scalars) go to a
//                    caller-provided workspace, component-major so that a warp's
//                    accesses are contiguous;
//   kVjpRecompute -- nothing is kept: sweep 2 inverts the forward step for
//                    (V, dV) and the Fb recursion for Fb.
#pragma once
#include "rnea_serial.cuh"

namespace rdyn {

// kVjpStoreShared: as kVjpStore, with the 20 scalars per link in the block's
// shared memory instead of a workspace (common-normal kernel, small batches).
enum VjpMode { kVjpStore = 0, kVjpRecompute = 1, kVjpStoreShared = 2 };
constexpr int kVjpStateScalars = 20;

// J u = (p, c x p + I_c u_w), p = m (u_v + u_w x c)  (spatial inertia about the
// joint-frame origin, from the centre-of-mass data)
template <typename T>
__device__ __forceinline__ void J_apply(T m, V3<T> c, const T *I, V3<T> uv, V3<T> uw, V3<T> &of,
                                        V3<T> &on)
{
    V3<T> p = scale3(m, cross_add(uw, c, uv));
    of = p;
    on = cross_add(c, p, sym_mul(I, uw));
}

// <a, ad_S b> over one 3-part with S = e_z: a . (e_z x b) = a_y b_x - a_x b_y
template <typename T>
__device__ __forceinline__ T dot_ez_cross(V3<T> a, V3<T> b)
{
    return fma(a.y, b.x, -a.x * b.y);
}

// Fb_i = Ad_{f^-1} Fb_{i-1} + S w  (same operation as the velocity step)
template <typename T>
__device__ __forceinline__ void fb_forward(const Rot<T> &R, V3<T> b, T w, V3<T> &fv, V3<T> &fw)
{
    V3<T> t = cross_add(fw, b, fv);
    fv = mulAT(R.r, t);
    fw = mulAT(R.r, fw);
    fw.z += w;
}

// inverse: Fb_{i-1} = Ad_f (Fb_i - S w)
template <typename T>
__device__ __forceinline__ void fb_backward(const Rot<T> &R, V3<T> b, T w, V3<T> &fv, V3<T> &fw)
{
    V3<T> ww = fw;
    ww.z -= w;
    V3<T> pw = mulA(R.r, ww);
    fv = cross_add(b, pw, mulA(R.r, fv));
    fw = pw;
}

template <typename T>
__device__ __forceinline__ void ws_put(T *ws, int B, int b, int i, int k, T v)
{
    ws[((size_t)i * kVjpStateScalars + k) * (size_t)B + b] = v;
}

template <typename T>
__device__ __forceinline__ T ws_get(const T *ws, int B, int b, int i, int k)
{
    return ws[((size_t)i * kVjpStateScalars + k) * (size_t)B + b];
}

template <typename T, int BLOCK, int MODE, bool VEC, bool FAST>
__global__ void __launch_bounds__(BLOCK)
rnea_vjp_kernel(const T *__restrict__ consts, int n, int B, const T *__restrict__ q,
                const T *__restrict__ qd, const T *__restrict__ qdd, const T *__restrict__ wv,
                T *__restrict__ gq, T *__restrict__ gqd, T *__restrict__ gqdd,
                T *__restrict__ ws, BaseParams<T> base)
{
    extern __shared__ __align__(16) unsigned char smem[];
    T *sc = reinterpret_cast<T *>(smem);
    const int nc = n * kLinkConsts;
    for (int k = threadIdx.x; k < nc; k += BLOCK) sc[k] = consts[k];
    __syncthreads();

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
    const int nchunks = (n + 3) / 4;
    for (int kc = 0; kc < nchunks; ++kc) {
        const int i0 = 4 * kc;
        const Chunk<T> cq = ld_chunk<T, VEC>(qr, i0, n), cqd = ld_chunk<T, VEC>(qdr, i0, n),
                       cqdd = ld_chunk<T, VEC>(qddr, i0, n), cw = ld_chunk<T, VEC>(wr, i0, n);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int i = i0 + j;
            if (VEC || i < n) {
                LinkXf<T> X;
                load_xf(sc + i * kLinkConsts, X);
                T s, c;
                joint_trig<T, FAST>(cq.v[j], &s, &c);
                const Rot<T> R = make_rot(X.A, c, s);
                const V3<T> bi = mk3(X.b[0], X.b[1], X.b[2]);
                x = forward_step_R(R, bi, cqd.v[j], cqdd.v[j], x);
                fb_forward(R, bi, cw.v[j], fbv, fbw);
                if constexpr (MODE == kVjpStore) {
                    const T vals[kVjpStateScalars] = {x.v.x,  x.v.y,  x.v.z,  x.w.x,  x.w.y,
                                                      x.w.z,  x.a.x,  x.a.y,  x.a.z,  x.al.x,
                                                      x.al.y, x.al.z, fbv.x,  fbv.y,  fbv.z,
                                                      fbw.x,  fbw.y,  fbw.z,  c,      s};
#pragma unroll
                    for (int k = 0; k < kVjpStateScalars; ++k) ws_put(ws, B, b, i, k, vals[k]);
                }
            }
        }
    }

    // ---- sweep 2: tip -> base
    Wrench<T> F;
    F.f = mk3(base.Fn[0], base.Fn[1], base.Fn[2]);
    F.n = mk3(base.Fn[3], base.Fn[4], base.Fn[5]);
    Wrench<T> Vb, dVb;  // adjoints of V_{i+1}, dV_{i+1} (covectors)
    Rot<T> Rn;
    V3<T> bn = mk3(T(0), T(0), T(0));
    T qdn = T(0);
    const int last0 = ((n - 1) / 4) * 4;
    for (int i0 = last0; i0 >= 0; i0 -= 4) {
        const Chunk<T> cq = ld_chunk<T, VEC>(qr, i0, n), cqd = ld_chunk<T, VEC>(qdr, i0, n),
                       cqdd = ld_chunk<T, VEC>(qddr, i0, n), cw = ld_chunk<T, VEC>(wr, i0, n);
        Chunk<T> oq, oqd, oqdd;
#pragma unroll
        for (int j = 3; j >= 0; --j) {
            const int i = i0 + j;
            oq.v[j] = oqd.v[j] = oqdd.v[j] = T(0);
            if (VEC || i < n) {
                LinkC<T> L;
                load_link(sc + i * kLinkConsts, L);
                T s, c;
                if constexpr (MODE == kVjpStore) {
                    x.v = mk3(ws_get(ws, B, b, i, 0), ws_get(ws, B, b, i, 1), ws_get(ws, B, b, i, 2));
                    x.w = mk3(ws_get(ws, B, b, i, 3), ws_get(ws, B, b, i, 4), ws_get(ws, B, b, i, 5));
                    x.a = mk3(ws_get(ws, B, b, i, 6), ws_get(ws, B, b, i, 7), ws_get(ws, B, b, i, 8));
                    x.al = mk3(ws_get(ws, B, b, i, 9), ws_get(ws, B, b, i, 10), ws_get(ws, B, b, i, 11));
                    fbv = mk3(ws_get(ws, B, b, i, 12), ws_get(ws, B, b, i, 13), ws_get(ws, B, b, i, 14));
                    fbw = mk3(ws_get(ws, B, b, i, 15), ws_get(ws, B, b, i, 16), ws_get(ws, B, b, i, 17));
                    c = ws_get(ws, B, b, i, 18);
                    s = ws_get(ws, B, b, i, 19);
                } else {
                    joint_trig<T, FAST>(cq.v[j], &s, &c);
                }
                const Rot<T> R = make_rot(L.A, c, s);
                const V3<T> bi = mk3(L.b[0], L.b[1], L.b[2]);
                const V3<T> cm = mk3(L.c[0], L.c[1], L.c[2]);
                const Wrench<T> Fh = bias_wrench(L.m, cm, L.I, x);
                if (i == n - 1) {
                    F.f = add3(F.f, Fh.f);
                    F.n = add3(F.n, Fh.n);
                } else {
                    F = carry_wrench_R(Rn, bn, F, Fh);
                }
                // local seeds from F_hat
                Wrench<T> dVl, Vl;
                J_apply(L.m, cm, L.I, fbv, fbw, dVl.f, dVl.n);             // J Fb
                V3<T> jvf, jvn;
                J_apply(L.m, cm, L.I, x.v, x.w, jvf, jvn);                 // J V
                // ad_V Fb = (w x Fb_v + v x Fb_w, w x Fb_w)
                const V3<T> adv = cross_add(x.v, fbw, cross3(x.w, fbv));
                const V3<T> adw = cross3(x.w, fbw);
                V3<T> jaf, jan;
                J_apply(L.m, cm, L.I, adv, adw, jaf, jan);                 // J ad_V Fb
                // ad^T_Fb (J V) = (-Fb_w x (JV)_f, -Fb_v x (JV)_f - Fb_w x (JV)_n)
                Vl.f = sub3(scale3(T(-1), cross3(fbw, jvf)), jaf);
                Vl.n = sub3(scale3(T(-1), cross_add(fbv, jvf, cross3(fbw, jvn))), jan);
                if (i == n - 1) {
                    Vb = Vl;
                    dVb = dVl;
                } else {
                    // Ybar = Vbar_{i+1} - ad^T_{S qd_{i+1}} dVbar_{i+1},
                    // ad^T_{S qd} x = -qd (e_z x x_f, e_z x x_n)
                    Wrench<T> Yb = Vb;
                    Yb.f.x = fma(-qdn, dVb.f.y, Yb.f.x);
                    Yb.f.y = fma(qdn, dVb.f.x, Yb.f.y);
                    Yb.n.x = fma(-qdn, dVb.n.y, Yb.n.x);
                    Yb.n.y = fma(qdn, dVb.n.x, Yb.n.y);
                    Vb = carry_wrench_R(Rn, bn, Yb, Vl);
                    dVb = carry_wrench_R(Rn, bn, dVb, dVl);
                }
                // gradients of link i
                oqdd.v[j] = dVb.n.z;
                oqd.v[j] = Vb.n.z - (dot_ez_cross(dVb.f, x.v) + dot_ez_cross(dVb.n, x.w));
                oq.v[j] = -(dot_ez_cross(Vb.f, x.v) + dot_ez_cross(Vb.n, x.w)) -
                          (dot_ez_cross(dVb.f, x.a) + dot_ez_cross(dVb.n, x.al)) -
                          (dot_ez_cross(F.f, fbv) + dot_ez_cross(F.n, fbw));
                if constexpr (MODE == kVjpRecompute) {
                    if (i > 0) {
                        x = backward_recover_R(R, bi, cqd.v[j], cqdd.v[j], x);
                        fb_backward(R, bi, cw.v[j], fbv, fbw);
                    }
                }
                Rn = R;
                bn = bi;
                qdn = cqd.v[j];
            }
        }
        st_chunk<T, VEC>(gq + row, i0, n, oq);
        st_chunk<T, VEC>(gqd + row, i0, n, oqd);
        st_chunk<T, VEC>(gqdd + row, i0, n, oqdd);
    }
}

}  // namespace rdyn
