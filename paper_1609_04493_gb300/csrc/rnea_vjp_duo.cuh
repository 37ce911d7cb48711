// rnea_vjp_duo.cuh -- the FP32 adjoint of rnea_vjp_dh.cuh with each instance's
// work split over the two warps of a 64-thread block and the per-link state in
// shared memory, for batches too small to give every scheduler a warp.
//
// At such batches the one-thread kernel is bound by one warp's issue rate
// (about 14k instructions per instance at an IPC near 0.5), not by the depth of
// its dependent chains. The adjoint's reverse sweep carries three covectors:
// the wrench F_i (Eq. id-backward), dVbar and Vbar. F and dVbar depend on
// nothing but the stored state and their own seeds; Vbar needs dVbar of the
// link above (Ybar = Vbar - ad^T_{S qd} dVbar). So the sweeps split with no
// exchange inside them:
// * Sweep 1 (base -> tip). Warp A runs the motion recursion (V_i, dV_i) and
//   keeps V, dV, cos, sin of every link in shared memory; warp B runs the
//   adjoint-weight recursion Fb_i = Ad_{f^-1} Fb_{i-1} + S w_i (each warp
//   evaluates the joint's sin/cos itself) and keeps Fb.
// * Sweep 2 (tip -> base), after a block barrier: warp A the bias wrench, the
//   carry of F and that of dVbar, writing gqdd and its terms of gqd and gq;
//   warp B the seeds of Vbar (J V, ad_V Fb, J ad_V Fb) and its carry, with its
//   own copy of the dVbar carry (the same operations on the same operands),
//   writing its terms of gqd and gq.
// * After a second barrier warp A forms gq and warp B gqd from the terms, in
//   the one-thread kernel's order of operations.
// Shared memory per block: 20 + 5 scalars per link and lane (about 100 KB at
// n = 32, two blocks per SM). Lanes past the batch recompute the last row and
// store nothing, so every thread reaches both barriers.
#pragma once
#include "rnea_vjp_dh.cuh"

namespace rdyn {

constexpr int kVjpDuoTerms = 5;  // per link: Vbar_z, Vbar term of gq (B); dVbar terms of gqd, gq, F term of gq (A)

// bytes of dynamic shared memory of one block
__host__ __device__ constexpr size_t vjp_duo_smem(int n)
{
    return (size_t)n * (kVjpStateScalars + kVjpDuoTerms) * 32 * sizeof(float);
}

template <int NMAX, int TRIG>
__global__ void __launch_bounds__(64)
rnea_vjp_duo_kernel(const __grid_constant__ DhParamConsts<float, NMAX> pc, int n, int B,
                    const float *__restrict__ q, const float *__restrict__ qd,
                    const float *__restrict__ qdd, const float *__restrict__ wv,
                    float *__restrict__ gq, float *__restrict__ gqd, float *__restrict__ gqdd,
                    BaseParams<float> base)
{
    extern __shared__ __align__(16) unsigned char duo_smem[];
    float *sst = reinterpret_cast<float *>(duo_smem);              // [link][20][32]
    float *stm = sst + (size_t)n * kVjpStateScalars * 32;          // [link][5][32]
    const float *sc = pc.c;
    const int lane = threadIdx.x & 31;
    const bool warp_a = threadIdx.x < 32;
    const int b_raw = blockIdx.x * 32 + lane;
    const bool live = b_raw < B;
    const size_t row = (size_t)(live ? b_raw : B - 1) * (size_t)n;
    const float *qr = q + row, *qdr = qd + row, *qddr = qdd + row, *wr = wv + row;
    auto st_put = [&](int i, int k, float v) { sst[((size_t)i * kVjpStateScalars + k) * 32 + lane] = v; };
    auto st_get = [&](int i, int k) -> float { return sst[((size_t)i * kVjpStateScalars + k) * 32 + lane]; };
    auto tm_put = [&](int i, int k, float v) { stm[((size_t)i * kVjpDuoTerms + k) * 32 + lane] = v; };
    auto tm_get = [&](int i, int k) -> float { return stm[((size_t)i * kVjpDuoTerms + k) * 32 + lane]; };
    const int nchunks = n / 4;

    // ---- sweep 1: base -> tip
    if (warp_a) {
        Motion<float> x;
        x.v = mk3(base.V0[0], base.V0[1], base.V0[2]);
        x.w = mk3(base.V0[3], base.V0[4], base.V0[5]);
        x.a = mk3(base.dV0[0], base.dV0[1], base.dV0[2]);
        x.al = mk3(base.dV0[3], base.dV0[4], base.dV0[5]);
        Chunk<float> cq, cqd, cqdd, nq = {}, nqd = {}, nqdd = {};
        ld_row_chunk(qr, 0, cq);
        ld_row_chunk(qdr, 0, cqd);
        ld_row_chunk(qddr, 0, cqdd);
        for (int kc = 0; kc < nchunks; ++kc) {
            const int i0 = 4 * kc;
            if (kc + 1 < nchunks) {
                ld_row_chunk(qr, i0 + 4, nq);
                ld_row_chunk(qdr, i0 + 4, nqd);
                ld_row_chunk(qddr, i0 + 4, nqdd);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int i = i0 + j;
                DhXf<float> X;
                load_dh_xf(sc + i * kDhConsts, X);
                float s, c;
                dh_trig<float, TRIG>(cq.v[j] + X.th0, &s, &c);
                x = dh_forward(dh_rot(X.ca, X.sa, c, s), X.b, cqd.v[j], cqdd.v[j], x);
                const float vals[12] = {x.v.x, x.v.y, x.v.z, x.w.x, x.w.y, x.w.z,
                                        x.a.x, x.a.y, x.a.z, x.al.x, x.al.y, x.al.z};
#pragma unroll
                for (int k = 0; k < 12; ++k) st_put(i, k, vals[k]);
                st_put(i, 18, c);
                st_put(i, 19, s);
            }
            cq = nq;
            cqd = nqd;
            cqdd = nqdd;
        }
    } else {
        V3<float> fbv = mk3(0.0f, 0.0f, 0.0f), fbw = mk3(0.0f, 0.0f, 0.0f);
        Chunk<float> cq, cw, nq = {}, nw = {};
        ld_row_chunk(qr, 0, cq);
        ld_row_chunk(wr, 0, cw);
        for (int kc = 0; kc < nchunks; ++kc) {
            const int i0 = 4 * kc;
            if (kc + 1 < nchunks) {
                ld_row_chunk(qr, i0 + 4, nq);
                ld_row_chunk(wr, i0 + 4, nw);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int i = i0 + j;
                DhXf<float> X;
                load_dh_xf(sc + i * kDhConsts, X);
                float s, c;
                dh_trig<float, TRIG>(cq.v[j] + X.th0, &s, &c);
                fb_forward_dh(dh_rot(X.ca, X.sa, c, s), X.b, cw.v[j], fbv, fbw);
                st_put(i, 12, fbv.x);
                st_put(i, 13, fbv.y);
                st_put(i, 14, fbv.z);
                st_put(i, 15, fbw.x);
                st_put(i, 16, fbw.y);
                st_put(i, 17, fbw.z);
            }
            cq = nq;
            cw = nw;
        }
    }
    __syncthreads();

    // ---- sweep 2: tip -> base, from the stored state
    DhRot<float> Rn = dh_rot(1.0f, 0.0f, 1.0f, 0.0f);
    V3<float> bn = mk3(0.0f, 0.0f, 0.0f);
    Wrench<float> dVb;  // adjoint of dV_{i+1}
    if (warp_a) {
        Wrench<float> F;
        F.f = mk3(base.Fn[0], base.Fn[1], base.Fn[2]);
        F.n = mk3(base.Fn[3], base.Fn[4], base.Fn[5]);
        for (int i0 = n - 4; i0 >= 0; i0 -= 4) {
            Chunk<float> oqdd;
#pragma unroll
            for (int j = 3; j >= 0; --j) {
                const int i = i0 + j;
                DhLink<float> L;
                load_dh(sc + i * kDhConsts, L);
                Motion<float> x;
                x.v = mk3(st_get(i, 0), st_get(i, 1), st_get(i, 2));
                x.w = mk3(st_get(i, 3), st_get(i, 4), st_get(i, 5));
                x.a = mk3(st_get(i, 6), st_get(i, 7), st_get(i, 8));
                x.al = mk3(st_get(i, 9), st_get(i, 10), st_get(i, 11));
                const V3<float> fbv = mk3(st_get(i, 12), st_get(i, 13), st_get(i, 14));
                const V3<float> fbw = mk3(st_get(i, 15), st_get(i, 16), st_get(i, 17));
                const float c = st_get(i, 18), s = st_get(i, 19);
                const DhRot<float> R = dh_rot(L.ca, L.sa, c, s);
                const Wrench<float> Fh = bias_wrench(L.m, L.c, L.I, x);
                Wrench<float> dVl;
                J_apply(L.m, L.c, L.I, fbv, fbw, dVl.f, dVl.n);  // J Fb
                if (i == n - 1) {
                    F.f = add3(F.f, Fh.f);
                    F.n = add3(F.n, Fh.n);
                    dVb = dVl;
                } else {
                    F = dh_carry(Rn, bn, F, Fh);
                    dVb = dh_carry(Rn, bn, dVb, dVl);
                }
                oqdd.v[j] = dVb.n.z;
                tm_put(i, 2, dot_ez_cross(dVb.f, x.v) + dot_ez_cross(dVb.n, x.w));
                tm_put(i, 3, dot_ez_cross(dVb.f, x.a) + dot_ez_cross(dVb.n, x.al));
                tm_put(i, 4, dot_ez_cross(F.f, fbv) + dot_ez_cross(F.n, fbw));
                Rn = R;
                bn = L.b;
            }
            if (live) st_chunk<float, true>(gqdd + row, i0, n, oqdd);
        }
    } else {
        Wrench<float> Vb;  // adjoint of V_{i+1}
        float qdn = 0.0f;
        Chunk<float> cqd, nqd = {};
        ld_row_chunk(qdr, n - 4, cqd);
        for (int i0 = n - 4; i0 >= 0; i0 -= 4) {
            if (i0 > 0) ld_row_chunk(qdr, i0 - 4, nqd);
#pragma unroll
            for (int j = 3; j >= 0; --j) {
                const int i = i0 + j;
                DhLink<float> L;
                load_dh(sc + i * kDhConsts, L);
                const V3<float> xv = mk3(st_get(i, 0), st_get(i, 1), st_get(i, 2));
                const V3<float> xw = mk3(st_get(i, 3), st_get(i, 4), st_get(i, 5));
                const V3<float> fbv = mk3(st_get(i, 12), st_get(i, 13), st_get(i, 14));
                const V3<float> fbw = mk3(st_get(i, 15), st_get(i, 16), st_get(i, 17));
                const float c = st_get(i, 18), s = st_get(i, 19);
                const DhRot<float> R = dh_rot(L.ca, L.sa, c, s);
                // local seeds from F_hat = J dV - ad^T_V (J V)
                Wrench<float> dVl, Vl;
                J_apply(L.m, L.c, L.I, fbv, fbw, dVl.f, dVl.n);           // J Fb
                V3<float> jvf, jvn;
                J_apply(L.m, L.c, L.I, xv, xw, jvf, jvn);                 // J V
                const V3<float> adv = cross_add(xv, fbw, cross3(xw, fbv)); // ad_V Fb
                const V3<float> adw = cross3(xw, fbw);
                V3<float> jaf, jan;
                J_apply(L.m, L.c, L.I, adv, adw, jaf, jan);               // J ad_V Fb
                Vl.f = sub3(scale3(-1.0f, cross3(fbw, jvf)), jaf);
                Vl.n = sub3(scale3(-1.0f, cross_add(fbv, jvf, cross3(fbw, jvn))), jan);
                if (i == n - 1) {
                    Vb = Vl;
                    dVb = dVl;
                } else {
                    Wrench<float> Yb = Vb;  // Vbar_{i+1} - ad^T_{S qd_{i+1}} dVbar_{i+1}
                    Yb.f.x = fma(-qdn, dVb.f.y, Yb.f.x);
                    Yb.f.y = fma(qdn, dVb.f.x, Yb.f.y);
                    Yb.n.x = fma(-qdn, dVb.n.y, Yb.n.x);
                    Yb.n.y = fma(qdn, dVb.n.x, Yb.n.y);
                    Vb = dh_carry(Rn, bn, Yb, Vl);
                    dVb = dh_carry(Rn, bn, dVb, dVl);
                }
                tm_put(i, 0, Vb.n.z);
                tm_put(i, 1, dot_ez_cross(Vb.f, xv) + dot_ez_cross(Vb.n, xw));
                Rn = R;
                bn = L.b;
                qdn = cqd.v[j];
            }
            cqd = nqd;
        }
    }
    __syncthreads();

    // ---- gradients from the terms: warp A gq, warp B gqd
    if (!live) return;
    for (int i0 = 0; i0 < n; i0 += 4) {
        Chunk<float> o;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int i = i0 + j;
            if (warp_a) o.v[j] = -tm_get(i, 1) - tm_get(i, 3) - tm_get(i, 4);
            else o.v[j] = tm_get(i, 0) - tm_get(i, 2);
        }
        st_chunk<float, true>((warp_a ? gq : gqd) + row, i0, n, o);
    }
}

}  // namespace rdyn
