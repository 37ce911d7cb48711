// rnea_vjp_pair.cuh -- the FP32 adjoint of rnea_vjp_dh.cuh (recompute mode)
// with each instance's work split between the two warps of a 64-thread block,
// for batches too small to give every scheduler a warp. The split shortens the
// work per warp, not the latency chain of the motion and wrench recursions,
// which stays on warp 0: it gains on long chains only (n = 100, B = 8192: 40.6
// against 44.8 us; n = 32: 13.2 against 12.8).
//
// Lane l of both warps serves instance 32 * blockIdx.x + l.
// * Sweep 1 (base -> tip). The motion recursion (V_i, dV_i of Eq. id-forward)
//   and the adjoint-weight recursion Fb_i = Ad_{f^-1} Fb_{i-1} + S w_i depend
//   on the link transforms only, not on each other: warp 0 runs the first,
//   warp 1 the second, each evaluating the joint's sin/cos itself. No exchange.
// * Sweep 2 (tip -> base). Warp 0 (producer) carries the wrench F_i of Eq.
//   (id-backward) and re-derives the motion by inverting the forward step;
//   per link it hands (V_i, dV_i, F_i, cos q_i, sin q_i) to warp 1 (consumer),
//   which forms the local seeds of F_hat = J dV - ad^T_V (J V), carries the
//   adjoints Vbar, dVbar, writes gq, gqd, gqdd and re-derives Fb_{i-1}.
// The hand-over goes through a two-slot ring in shared memory guarded by four
// named barriers: FULL[s] (producer arrives after writing slot s, consumer
// waits before reading it) and EMPTY[s] (consumer arrives after reading slot s,
// producer waits before writing it again two links later). Every arrive has
// exactly one matching wait: both warps run the same n links with
// warp-uniform control flow, the producer waits on EMPTY from its third link
// on and the consumer arrives on EMPTY on all but its last two. Lanes past the
// batch recompute the last row and store nothing, so no thread leaves early.
// For n % 4 == 0, n <= NMAX and 16-byte aligned rows.
#pragma once
#include "rnea_vjp_dh.cuh"

namespace rdyn {

constexpr int kVjpPairScalars = 20;  // V (6), dV (6), F (6), cos, sin
constexpr int kVjpPairBarFull = 1;   // named barriers 1, 2 (0 is __syncthreads)
constexpr int kVjpPairBarEmpty = 3;  // named barriers 3, 4

// Barrier ids as immediates (the callers' ids fold to constants once the link
// loop is unrolled), so that the kernel holds four barriers, not all sixteen.
__device__ __forceinline__ void pair_bar_sync(int id)
{
    if (id == 1) asm volatile("bar.sync 1, 64;" ::: "memory");
    else if (id == 2) asm volatile("bar.sync 2, 64;" ::: "memory");
    else if (id == 3) asm volatile("bar.sync 3, 64;" ::: "memory");
    else asm volatile("bar.sync 4, 64;" ::: "memory");
}

__device__ __forceinline__ void pair_bar_arrive(int id)
{
    if (id == 1) asm volatile("bar.arrive 1, 64;" ::: "memory");
    else if (id == 2) asm volatile("bar.arrive 2, 64;" ::: "memory");
    else if (id == 3) asm volatile("bar.arrive 3, 64;" ::: "memory");
    else asm volatile("bar.arrive 4, 64;" ::: "memory");
}

template <int NMAX, int TRIG>
__global__ void __launch_bounds__(64)
rnea_vjp_pair_kernel(const __grid_constant__ DhParamConsts<float, NMAX> pc, int n, int B,
                     const float *__restrict__ q, const float *__restrict__ qd,
                     const float *__restrict__ qdd, const float *__restrict__ wv,
                     float *__restrict__ gq, float *__restrict__ gqd, float *__restrict__ gqdd,
                     BaseParams<float> base)
{
    __shared__ float ring[2][kVjpPairScalars][32];
    const float *sc = pc.c;
    const int lane = threadIdx.x & 31;
    const bool producer = threadIdx.x < 32;
    const int b_raw = blockIdx.x * 32 + lane;
    const bool live = b_raw < B;
    const size_t row = (size_t)(live ? b_raw : B - 1) * (size_t)n;
    const float *qr = q + row, *qdr = qd + row, *qddr = qdd + row, *wr = wv + row;
    const int nchunks = n / 4;

    if (producer) {
        // ---- sweep 1: motion, base -> tip
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
                DhXf<float> X;
                load_dh_xf(sc + (i0 + j) * kDhConsts, X);
                float s, c;
                dh_trig<float, TRIG>(cq.v[j] + X.th0, &s, &c);
                x = dh_forward(dh_rot(X.ca, X.sa, c, s), X.b, cqd.v[j], cqdd.v[j], x);
            }
            cq = nq;
            cqd = nqd;
            cqdd = nqdd;
        }

        // ---- sweep 2: wrenches and motion, tip -> base, handed to warp 1
        Wrench<float> F;
        F.f = mk3(base.Fn[0], base.Fn[1], base.Fn[2]);
        F.n = mk3(base.Fn[3], base.Fn[4], base.Fn[5]);
        DhRot<float> Rn = dh_rot(1.0f, 0.0f, 1.0f, 0.0f);
        V3<float> bn = mk3(0.0f, 0.0f, 0.0f);
        const int last0 = n - 4;
        ld_row_chunk(qr, last0, cq);
        ld_row_chunk(qdr, last0, cqd);
        ld_row_chunk(qddr, last0, cqdd);
        for (int i0 = last0; i0 >= 0; i0 -= 4) {
            if (i0 > 0) {
                ld_row_chunk(qr, i0 - 4, nq);
                ld_row_chunk(qdr, i0 - 4, nqd);
                ld_row_chunk(qddr, i0 - 4, nqdd);
            }
#pragma unroll
            for (int j = 3; j >= 0; --j) {
                const int i = i0 + j;
                const int t = n - 1 - i;  // links handed over so far
                const int slot = (j + 1) & 1;  // = t & 1, as n and i0 are multiples of 4
                DhLink<float> L;
                load_dh(sc + i * kDhConsts, L);
                float s, c;
                dh_trig<float, TRIG>(cq.v[j] + L.th0, &s, &c);
                const DhRot<float> R = dh_rot(L.ca, L.sa, c, s);
                const Wrench<float> Fh = bias_wrench(L.m, L.c, L.I, x);
                if (i == n - 1) {
                    F.f = add3(F.f, Fh.f);
                    F.n = add3(F.n, Fh.n);
                } else {
                    F = dh_carry(Rn, bn, F, Fh);
                }
                if (t >= 2) pair_bar_sync(kVjpPairBarEmpty + slot);
                float *o = &ring[slot][0][lane];
                const float vals[kVjpPairScalars] = {x.v.x,  x.v.y,  x.v.z,  x.w.x,  x.w.y,
                                                     x.w.z,  x.a.x,  x.a.y,  x.a.z,  x.al.x,
                                                     x.al.y, x.al.z, F.f.x,  F.f.y,  F.f.z,
                                                     F.n.x,  F.n.y,  F.n.z,  c,      s};
#pragma unroll
                for (int k = 0; k < kVjpPairScalars; ++k) o[32 * k] = vals[k];
                pair_bar_arrive(kVjpPairBarFull + slot);
                if (i > 0) x = dh_recover(R, L.b, cqd.v[j], cqdd.v[j], x);
                Rn = R;
                bn = L.b;
            }
            cq = nq;
            cqd = nqd;
            cqdd = nqdd;
        }
        return;
    }

    // ---- warp 1, sweep 1: adjoint weights, base -> tip
    V3<float> fbv = mk3(0.0f, 0.0f, 0.0f), fbw = mk3(0.0f, 0.0f, 0.0f);
    {
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
                DhXf<float> X;
                load_dh_xf(sc + (i0 + j) * kDhConsts, X);
                float s, c;
                dh_trig<float, TRIG>(cq.v[j] + X.th0, &s, &c);
                fb_forward_dh(dh_rot(X.ca, X.sa, c, s), X.b, cw.v[j], fbv, fbw);
            }
            cq = nq;
            cw = nw;
        }
    }

    // ---- warp 1, sweep 2: adjoints and gradients, tip -> base
    Wrench<float> Vb, dVb;  // adjoints of V_{i+1}, dV_{i+1} (covectors)
    DhRot<float> Rn = dh_rot(1.0f, 0.0f, 1.0f, 0.0f);
    V3<float> bn = mk3(0.0f, 0.0f, 0.0f);
    float qdn = 0.0f;
    Chunk<float> cqd, cw, nqd = {}, nw = {};
    const int last0 = n - 4;
    ld_row_chunk(qdr, last0, cqd);
    ld_row_chunk(wr, last0, cw);
    for (int i0 = last0; i0 >= 0; i0 -= 4) {
        if (i0 > 0) {
            ld_row_chunk(qdr, i0 - 4, nqd);
            ld_row_chunk(wr, i0 - 4, nw);
        }
        Chunk<float> oq, oqd, oqdd;
#pragma unroll
        for (int j = 3; j >= 0; --j) {
            const int i = i0 + j;
            const int t = n - 1 - i;
            const int slot = (j + 1) & 1;  // = t & 1
            DhLink<float> L;
            load_dh(sc + i * kDhConsts, L);
            pair_bar_sync(kVjpPairBarFull + slot);
            const float *in = &ring[slot][0][lane];
            float v[kVjpPairScalars];
#pragma unroll
            for (int k = 0; k < kVjpPairScalars; ++k) v[k] = in[32 * k];
            if (t + 2 <= n - 1) pair_bar_arrive(kVjpPairBarEmpty + slot);
            Motion<float> x;
            x.v = mk3(v[0], v[1], v[2]);
            x.w = mk3(v[3], v[4], v[5]);
            x.a = mk3(v[6], v[7], v[8]);
            x.al = mk3(v[9], v[10], v[11]);
            Wrench<float> F;
            F.f = mk3(v[12], v[13], v[14]);
            F.n = mk3(v[15], v[16], v[17]);
            const DhRot<float> R = dh_rot(L.ca, L.sa, v[18], v[19]);
            // local seeds from F_hat = J dV - ad^T_V (J V)
            Wrench<float> dVl, Vl;
            J_apply(L.m, L.c, L.I, fbv, fbw, dVl.f, dVl.n);              // J Fb
            V3<float> jvf, jvn;
            J_apply(L.m, L.c, L.I, x.v, x.w, jvf, jvn);                  // J V
            const V3<float> adv = cross_add(x.v, fbw, cross3(x.w, fbv));  // ad_V Fb
            const V3<float> adw = cross3(x.w, fbw);
            V3<float> jaf, jan;
            J_apply(L.m, L.c, L.I, adv, adw, jaf, jan);                  // J ad_V Fb
            Vl.f = sub3(scale3(-1.0f, cross3(fbw, jvf)), jaf);
            Vl.n = sub3(scale3(-1.0f, cross_add(fbv, jvf, cross3(fbw, jvn))), jan);
            if (i == n - 1) {
                Vb = Vl;
                dVb = dVl;
            } else {
                Wrench<float> Yb = Vb;  // Vbar_{i+1} - ad^T_{S qd_{i+1}} dVbar_{i+1}
                Yb.f.x = fmaf(-qdn, dVb.f.y, Yb.f.x);
                Yb.f.y = fmaf(qdn, dVb.f.x, Yb.f.y);
                Yb.n.x = fmaf(-qdn, dVb.n.y, Yb.n.x);
                Yb.n.y = fmaf(qdn, dVb.n.x, Yb.n.y);
                Vb = dh_carry(Rn, bn, Yb, Vl);
                dVb = dh_carry(Rn, bn, dVb, dVl);
            }
            oqdd.v[j] = dVb.n.z;
            oqd.v[j] = Vb.n.z - (dot_ez_cross(dVb.f, x.v) + dot_ez_cross(dVb.n, x.w));
            oq.v[j] = -(dot_ez_cross(Vb.f, x.v) + dot_ez_cross(Vb.n, x.w)) -
                      (dot_ez_cross(dVb.f, x.a) + dot_ez_cross(dVb.n, x.al)) -
                      (dot_ez_cross(F.f, fbv) + dot_ez_cross(F.n, fbw));
            if (i > 0) fb_backward_dh(R, L.b, cw.v[j], fbv, fbw);
            Rn = R;
            bn = L.b;
            qdn = cqd.v[j];
        }
        if (live) {
            st_chunk<float, true>(gq + row, i0, n, oq);
            st_chunk<float, true>(gqd + row, i0, n, oqd);
            st_chunk<float, true>(gqdd + row, i0, n, oqdd);
        }
        cqd = nqd;
        cw = nw;
    }
}

}  // namespace rdyn
