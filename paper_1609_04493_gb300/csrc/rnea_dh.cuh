// rnea_dh.cuh -- one thread per instance, the two propagations of Sec. II-A
// (Eqs. id-forward, id-backward) as a serial recursion over the links, in the
// common-normal frames of spatial_dh.cuh. Same structure and state modes as
// rnea_serial.cuh (kStore keeps F_hat_i, cos and sin of every link in shared
// memory; kRecompute keeps nothing and inverts the forward step in the
// backward sweep), with cheaper link rotations and 16 constants per link.
#pragma once
#include "rnea_serial.cuh"
#include "spatial_dh.cuh"

namespace rdyn {

// Shared memory: n * 16 link constants, then (VEC) the staging ring, then the
// per-link state of the mode. Thread b of the grid evaluates instance b.
template <typename T, int BLOCK, int MODE, bool VEC, bool FAST>
__global__ void __launch_bounds__(BLOCK)
rnea_dh_kernel(const T *__restrict__ consts, int n, int B, const T *__restrict__ q,
               const T *__restrict__ qd, const T *__restrict__ qdd, T *__restrict__ tau,
               BaseParams<T> base)
{
    static_assert(MODE == kStore || MODE == kRecompute, "rnea_dh_kernel: state mode");
    extern __shared__ __align__(16) unsigned char smem[];
    T *sc = reinterpret_cast<T *>(smem);
    const int nc = n * kDhConsts;
    for (int k = threadIdx.x; k < nc; k += BLOCK) sc[k] = consts[k];
    unsigned char *ring = smem + (size_t)nc * sizeof(T);
    unsigned char *st = ring + (VEC ? (size_t)stage_bytes_per_thread<T>() * BLOCK : 0);
    __syncthreads();

    const int tid = threadIdx.x;
    const int b = blockIdx.x * BLOCK + tid;
    if (b >= B) return;
    const size_t row = (size_t)b * (size_t)n;
    const T *qr = q + row, *qdr = qd + row, *qddr = qdd + row;
    T *taur = tau + row;

    Motion<T> x;
    x.v = mk3(base.V0[0], base.V0[1], base.V0[2]);
    x.w = mk3(base.V0[3], base.V0[4], base.V0[5]);
    x.a = mk3(base.dV0[0], base.dV0[1], base.dV0[2]);
    x.al = mk3(base.dV0[3], base.dV0[4], base.dV0[5]);

    // ---- forward sweep: base -> tip, joint values staged ahead of use
    const int nchunks = (n + 3) / 4;
    Chunk<T> cq = {}, cqd = {}, cqdd = {};
    if constexpr (VEC) {
#pragma unroll
        for (int k = 0; k < kStages - 1; ++k) {
            if (k < nchunks) stage_chunk<T, BLOCK>(ring, k, tid, qr, qdr, qddr, 4 * k);
            __pipeline_commit();
        }
    } else {
        cq = ld_chunk<T, VEC>(qr, 0, n);
        cqd = ld_chunk<T, VEC>(qdr, 0, n);
        cqdd = ld_chunk<T, VEC>(qddr, 0, n);
    }
    for (int kc = 0; kc < nchunks; ++kc) {
        const int i0 = 4 * kc;
        Chunk<T> nq = cq, nqd = cqd, nqdd = cqdd;
        if constexpr (VEC) {
            const int ahead = kc + kStages - 1;
            if (ahead < nchunks) stage_chunk<T, BLOCK>(ring, ahead % kStages, tid, qr, qdr, qddr, 4 * ahead);
            __pipeline_commit();
            __pipeline_wait_prior(kStages - 1);
            read_chunk<T, BLOCK>(ring, kc % kStages, tid, cq, cqd, cqdd);
        } else {
            if (i0 + 4 < n) {
                nq = ld_chunk<T, VEC>(qr, i0 + 4, n);
                nqd = ld_chunk<T, VEC>(qdr, i0 + 4, n);
                nqdd = ld_chunk<T, VEC>(qddr, i0 + 4, n);
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int i = i0 + j;
            if (VEC || i < n) {
                T s, c;
                if constexpr (MODE == kStore) {
                    DhLink<T> L;
                    load_dh(sc + i * kDhConsts, L);
                    joint_trig<T, FAST>(cq.v[j] + L.th0, &s, &c);
                    x = dh_forward(dh_rot(L.ca, L.sa, c, s), L.b, cqd.v[j], cqdd.v[j], x);
                    LinkState<T> ls;
                    ls.Fh = bias_wrench(L.m, L.c, L.I, x);
                    ls.c = c;
                    ls.s = s;
                    put_state<T>(st, i, tid, BLOCK, ls);
                } else {
                    DhXf<T> X;
                    load_dh_xf(sc + i * kDhConsts, X);
                    joint_trig<T, FAST>(cq.v[j] + X.th0, &s, &c);
                    x = dh_forward(dh_rot(X.ca, X.sa, c, s), X.b, cqd.v[j], cqdd.v[j], x);
                }
            }
        }
        if constexpr (!VEC) {
            cq = nq;
            cqd = nqd;
            cqdd = nqdd;
        }
    }

    // ---- backward sweep: tip -> base
    Wrench<T> F;
    F.f = mk3(base.Fn[0], base.Fn[1], base.Fn[2]);
    F.n = mk3(base.Fn[3], base.Fn[4], base.Fn[5]);
    constexpr bool kNeedJoints = MODE != kStore;
    DhRot<T> Rn = dh_rot(T(1), T(0), T(1), T(0));  // rotation of link i+1
    V3<T> bn = mk3(T(0), T(0), T(0));
    const int last0 = ((n - 1) / 4) * 4;
    if (kNeedJoints) {
        if constexpr (VEC) {
#pragma unroll
            for (int k = 0; k < kStages - 1; ++k) {
                const int c = nchunks - 1 - k;
                if (c >= 0) stage_chunk<T, BLOCK>(ring, k, tid, qr, qdr, qddr, 4 * c);
                __pipeline_commit();
            }
        } else {
            cq = ld_chunk<T, VEC>(qr, last0, n);
            cqd = ld_chunk<T, VEC>(qdr, last0, n);
            cqdd = ld_chunk<T, VEC>(qddr, last0, n);
        }
    }
    for (int kb = 0; kb < nchunks; ++kb) {
        const int i0 = last0 - 4 * kb;
        Chunk<T> nq = cq, nqd = cqd, nqdd = cqdd;
        if (kNeedJoints) {
            if constexpr (VEC) {
                const int ahead = kb + kStages - 1;
                if (ahead < nchunks)
                    stage_chunk<T, BLOCK>(ring, ahead % kStages, tid, qr, qdr, qddr,
                                          last0 - 4 * ahead);
                __pipeline_commit();
                __pipeline_wait_prior(kStages - 1);
                read_chunk<T, BLOCK>(ring, kb % kStages, tid, cq, cqd, cqdd);
            } else {
                if (i0 > 0) {
                    nq = ld_chunk<T, VEC>(qr, i0 - 4, n);
                    nqd = ld_chunk<T, VEC>(qdr, i0 - 4, n);
                    nqdd = ld_chunk<T, VEC>(qddr, i0 - 4, n);
                }
            }
        }
        Chunk<T> ct;
#pragma unroll
        for (int j = 3; j >= 0; --j) {
            const int i = i0 + j;
            ct.v[j] = T(0);
            if (VEC || i < n) {
                if constexpr (MODE == kStore) {
                    LinkState<T> ls;
                    get_state<T>(st, i, tid, BLOCK, ls);
                    if (i == n - 1) {
                        F.f = add3(F.f, ls.Fh.f);
                        F.n = add3(F.n, ls.Fh.n);
                    } else {
                        F = dh_carry(Rn, bn, F, ls.Fh);
                    }
                    DhXf<T> X;
                    load_dh_xf(sc + i * kDhConsts, X);
                    Rn = dh_rot(X.ca, X.sa, ls.c, ls.s);
                    bn = X.b;
                } else {
                    DhLink<T> L;
                    load_dh(sc + i * kDhConsts, L);
                    T s, c;
                    joint_trig<T, FAST>(cq.v[j] + L.th0, &s, &c);
                    const DhRot<T> R = dh_rot(L.ca, L.sa, c, s);
                    const Wrench<T> Fh = bias_wrench(L.m, L.c, L.I, x);
                    if (i == n - 1) {
                        F.f = add3(F.f, Fh.f);
                        F.n = add3(F.n, Fh.n);
                    } else {
                        F = dh_carry(Rn, bn, F, Fh);
                    }
                    if (i > 0) x = dh_recover(R, L.b, cqd.v[j], cqdd.v[j], x);
                    Rn = R;
                    bn = L.b;
                }
                ct.v[j] = F.n.z;
            }
        }
        st_chunk<T, VEC>(taur, i0, n, ct);
        if (kNeedJoints && !VEC) {
            cq = nq;
            cqd = nqd;
            cqdd = nqdd;
        }
    }
}

}  // namespace rdyn
